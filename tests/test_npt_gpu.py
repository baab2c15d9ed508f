"""GPU parity of the Berendsen thermostat and barostat (md_set_npt) against the oracle's
oracle_run_ex: the same coupling (lambda, mu computed from each step's K, K_aa and the
Eq. 29 total virial, applied at the start of the next step), run through the C ABI.

The GPU keeps a skin list whose test allows for the box scaling since the build and
coarsens cell grids that became too fine; the oracle rebuilds from scratch every step in
the current box.  Bounds as for NVE trajectories: 1e-10 (metric of the parity tests) on
positions, velocities, the (U, K, J) series and the box."""
import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TRAJ_TOL = 1e-10


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03343_gb300 import _build, md as M
    _build.build()
    M.load()
    return M


def rel(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max())


def pos_err(p, p_ref, box, pbc):
    d = p - p_ref
    d -= np.round(d / box) * box * pbc
    return float(np.abs(d).max())


def check(md, s, steps, dt, cpl, skin=0.0, splits=None, eager=False, precision=0):
    """Run `steps` NPT steps on the GPU (as md_run calls of the sizes in `splits`) and
    compare with one oracle run of the same length."""
    with md.from_inputs(s, skin=skin, precision=precision) as g:
        if eager:
            md.md_set_graph_mode(g.ctx, False)
        g.set_npt(**cpl)
        parts = splits or [steps]
        ser = np.concatenate([g.run(k, dt) for k in parts])
        pos, vel = g.state()
        box = g.box()
        st = g.stats()
    p2, v2, ser2, b2 = O.run_npt(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt, **cpl)
    assert rel(box, b2) < TRAJ_TOL, (box, b2)
    assert pos_err(pos, p2, b2, s.pbc) < TRAJ_TOL
    assert rel(vel, v2) < TRAJ_TOL
    for c in range(5):
        assert rel(ser[:, c], ser2[:, c]) < TRAJ_TOL, c
    return box, st, (pos, vel, ser)


def test_tersoff_thermostat_and_barostat_match_oracle(md):
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0)
    cpl = dict(T0=300.0, P0=0.0, tau_T=20.0, tau_P=100.0, beta=0.02)
    box, _, _ = check(md, s, 40, 1.0, cpl)
    assert not np.allclose(box, s.box)          # the barostat moved the box


def test_sw_thermostat_and_barostat_match_oracle(md):
    s = I.si_diamond_sw(n=3, jitter_amp=0.05, temperature=500.0)
    cpl = dict(T0=300.0, P0=1.0, tau_T=30.0, tau_P=80.0, beta=0.02)
    check(md, s, 40, 1.0, cpl)


def test_thermostat_only_and_barostat_only(md):
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=900.0)
    box, _, _ = check(md, s, 30, 1.0, dict(T0=300.0, tau_T=10.0, tau_P=0.0))
    assert np.array_equal(box, s.box)
    check(md, s, 30, 1.0, dict(tau_T=0.0, tau_P=60.0, beta=0.02, couple=(1, 0, 1)))


def test_pending_scaling_carries_over_between_runs(md):
    """Runs of 13 + 8 + 19 steps continue one trajectory: the scaling computed at the
    end of each call is applied at the first step of the next."""
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0, seed_pos=5, seed_vel=6)
    cpl = dict(T0=300.0, P0=0.5, tau_T=25.0, tau_P=60.0, beta=0.02)
    check(md, s, 40, 1.0, cpl, splits=[13, 8, 19])


def test_compressed_crystal_expands_with_rebuilds(md):
    """Diamond Si compressed to a = 5.38 A relaxes towards 5.432 A: a 1% expansion over the
    run, several list rebuilds forced by the box scaling."""
    pos, box = I.diamond_positions(3, 5.38)
    s = I.System("si_compressed", pos=I.wrap(I.jitter(pos, 0.02, 3), box, np.array([1, 1, 1], np.int32)), vel=I.maxwell_boltzmann(len(pos), I.MASS_SI, 100.0, 4),
                 box=box, pbc=np.array([1, 1, 1], np.int32), kind=I.MD_TERSOFF, params=I.TERSOFF_SI_1989,
                 mass=I.MASS_SI)
    cpl = dict(T0=100.0, tau_T=50.0, tau_P=40.0, beta=0.05)
    b, st, _ = check(md, s, 80, 1.0, cpl, skin=0.2)
    assert b[0] > box[0] * 1.004
    assert st.n_rebuilds >= 3


def test_shrinking_box_coarsens_the_cell_grid(md):
    """Expanded Si (a = 5.47 A) shrinks.  The skin is chosen so that the first cells are
    barely wider than the list radius (five per edge): once the edge has shrunk by more
    than ~0.006 A five cells no longer fit, the device coarsens the grid to four, and the
    rebuilds that follow (a small skin at 600 K) use that grid; the lists stay exact."""
    a, n = 5.47, 3
    L = a * n
    skin = L / 5.0 - 3.0 - 1e-4 - 1e-3     # Tersoff-Si cutoff S = 3.0 A; cell edge = rl + fp32 margin
    pbc = np.array([1, 1, 1], np.int32)
    pos, box = I.diamond_positions(n, a)
    s = I.System("si_expanded", pos=I.wrap(I.jitter(pos, 0.02, 7), box, pbc),
                 vel=I.maxwell_boltzmann(len(pos), I.MASS_SI, 600.0, 8), box=box, pbc=pbc, kind=I.MD_TERSOFF,
                 params=I.TERSOFF_SI_1989, mass=I.MASS_SI)
    cpl = dict(T0=600.0, tau_T=50.0, tau_P=30.0, beta=0.05)
    b, st, _ = check(md, s, 60, 1.0, cpl, skin=skin)
    assert b[0] < L - 0.02                    # shrank well past five cell edges
    assert st.n_rebuilds >= 3


def test_graph_replay_matches_eager_bitwise(md):
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0)
    cpl = dict(T0=300.0, P0=0.0, tau_T=20.0, tau_P=100.0, beta=0.02)
    _, _, (p1, v1, s1) = check(md, s, 21, 1.0, cpl)
    _, _, (p2, v2, s2) = check(md, s, 21, 1.0, cpl, eager=True)
    assert np.array_equal(p1, p2) and np.array_equal(v1, v2) and np.array_equal(s1, s2)


def test_mixed_precision_npt_tracks_fp64(md):
    """The mixed path (fp32 pair arithmetic, fp64 integration, scaling and totals) follows
    the fp64 trajectory over 20 steps within the force-error scale."""
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0)
    cpl = dict(T0=300.0, P0=0.0, tau_T=20.0, tau_P=100.0, beta=0.02)
    out = []
    for prec in (0, 1):
        with md.from_inputs(s, precision=prec) as g:
            g.set_npt(**cpl)
            ser = g.run(20, 1.0)
            out.append((g.box(), g.state(), ser))
    (b0, (p0, v0), s0), (b1, (p1, v1), s1) = out
    assert rel(b1, b0) < 1e-7
    assert pos_err(p1, p0, b0, s.pbc) < 1e-5
    assert rel(s1[:, 1], s0[:, 1]) < 1e-4                     # kinetic energy


def test_npt_off_returns_to_nve(md):
    """After coupling is switched off the box stays where the barostat left it and the
    steps are plain NVE in that box (compared with the oracle's NVE run from that state)."""
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0)
    with md.from_inputs(s) as g:
        g.set_npt(T0=300.0, tau_T=20.0, tau_P=50.0, beta=0.03)
        g.run(15, 1.0)
        g.set_npt(off=True)
        b = g.box()
        p0, v0 = g.state()
        ser = g.run(20, 1.0)
        p, v = g.state()
        assert np.array_equal(g.box(), b)
    p2, v2, ser2 = O.run(p0, v0, s.mass, b, s.pbc, s.kind, s.params, 20, 1.0)
    assert pos_err(p, p2, b, s.pbc) < TRAJ_TOL and rel(v, v2) < TRAJ_TOL
    assert rel(ser, ser2) < TRAJ_TOL


def test_compute_after_npt_uses_the_scaled_box(md):
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0)
    cpl = dict(T0=300.0, tau_T=20.0, tau_P=40.0, beta=0.03)
    with md.from_inputs(s) as g:
        g.set_npt(**cpl)
        g.run(25, 1.0)
        out = g.compute()
        b = g.box()
    p2, v2, _, b2 = O.run_npt(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 25, 1.0, **cpl)
    assert rel(b, b2) < TRAJ_TOL
    ref = O.compute(p2, b2, s.pbc, s.kind, s.params, v2)
    for k in ("F", "U", "W", "J"):
        assert rel(out[k], ref[k]) < 1e-9, k


def test_pool_npt_systems_match_standalone_and_oracle(md):
    """A pool with two differently coupled Tersoff systems and one NVE system: each
    equals the same system run alone (bitwise) and the oracle (1e-10)."""
    mix = [
        (I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0, seed_pos=3, seed_vel=4),
         dict(T0=300.0, tau_T=20.0, tau_P=60.0, beta=0.02)),
        (I.si_diamond_tersoff(n=2, jitter_amp=0.05, temperature=300.0, seed_pos=5, seed_vel=6), None),
        (I.si_diamond_tersoff(n=4, jitter_amp=0.05, temperature=200.0, seed_pos=7, seed_vel=8),
         dict(T0=400.0, P0=2.0, tau_T=15.0, tau_P=40.0, beta=0.03, couple=(1, 1, 0))),
    ]
    steps, dt = 30, 1.0
    with md.Pool(5000, 4, I.MD_TERSOFF, [I.TERSOFF_SI_1989], [I.MASS_SI]) as pool:
        ids = []
        for s, cpl in mix:
            sid = pool.add(s.pos, s.vel, s.box, s.pbc)
            if cpl:
                pool.set_npt(sid, **cpl)
            ids.append(sid)
        ser = pool.run(steps, dt, record=True)
        for (s, cpl), sid in zip(mix, ids):
            p, v = pool.state(sid)
            b = pool.box(sid)
            with md.from_inputs(s) as g:
                if cpl:
                    g.set_npt(**cpl)
                ser1 = g.run(steps, dt)
                p1, v1 = g.state()
                assert np.array_equal(b, g.box())
            assert np.array_equal(p, p1) and np.array_equal(v, v1), s.name
            assert np.array_equal(ser[:, sid, :], ser1), s.name
            if cpl:
                p2, v2, ser2, b2 = O.run_npt(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt, **cpl)
            else:
                p2, v2, ser2 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt)
                b2 = s.box
            assert rel(b, b2) < TRAJ_TOL
            assert pos_err(p, p2, b2, s.pbc) < TRAJ_TOL and rel(v, v2) < TRAJ_TOL
            assert rel(ser[:, sid, :], ser2) < TRAJ_TOL


def test_box_below_the_minimum_is_reported(md):
    """A list radius chosen so that the periodic edge is only 0.06 A above its minimum of
    2 (rl + margin) + 0.01 A, and a bath pressure that compresses the box by ~0.7% in one
    step: md_run reports MD_ERR_BOX (the atoms stay 2.33 A apart, far from overlap)."""
    s = I.si_diamond_tersoff(n=2, jitter_amp=0.0, temperature=10.0)
    L = s.box[0]
    skin = (L - 0.07) / 2.0 - 3.0
    with md.from_inputs(s, skin=skin) as g:
        g.set_npt(T0=10.0, P0=20.0, tau_T=0.0, tau_P=10.0, beta=0.01)
        with pytest.raises(md.MDError) as e:
            g.run(2, 1.0)
        assert e.value.status == md.MD_ERR_BOX


def test_bad_npt_arguments_are_rejected(md):
    s = I.si_diamond_tersoff(n=2)
    with md.from_inputs(s) as g:
        for bad in (dict(T0=-1.0), dict(beta=-0.1), dict(tau_T=float("nan")), dict(couple=(2, 0, 0))):
            with pytest.raises(md.MDError) as e:
                g.set_npt(**bad)
            assert e.value.status == md.MD_ERR_ARG
        with pytest.raises(md.MDError):
            md.md_set_npt(g.ctx, 1)
