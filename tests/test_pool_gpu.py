"""Pools: many systems stepped together over one flattened atom index.  Each system's
results must equal those it has alone (bitwise: same kernels, same per-atom arithmetic,
same block composition) and the oracle's (1e-10 after the trajectory)."""
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
    a = np.asarray(a); b = np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max())


def tersoff_mix():
    """Si diamond and C graphene / diamond cells of uneven sizes (two parameter sets)."""
    return [
        (I.si_diamond_tersoff(n=3, jitter_amp=0.05, seed_pos=3, seed_vel=4), 0, 1.0),
        (I.c_graphene_tersoff(nx=6, ny=10, jitter_amp=0.02, seed_pos=5, seed_vel=6), 1, 0.5),
        (I.si_diamond_tersoff(n=4, jitter_amp=0.05, seed_pos=7, seed_vel=8), 0, 1.0),
        (I.c_diamond_tersoff(n=3, jitter_amp=0.02, seed_pos=9, seed_vel=10), 1, 0.5),
        (I.si_diamond_tersoff(n=2, jitter_amp=0.05, seed_pos=11, seed_vel=12), 0, 1.0),
    ]


def make_pool(md, precision=0, capacity=20000, max_systems=8):
    return md.Pool(capacity, max_systems, I.MD_TERSOFF, [I.TERSOFF_SI_1989, I.TERSOFF_C_1989],
                   [I.MASS_SI, I.MASS_C], precision=precision)


def types_for(s):
    return np.full(s.n, 0 if s.mass == I.MASS_SI else 1, np.int32)


def standalone(md, s, steps, dt, precision=0, damp=0.0):
    with md.from_inputs(s, precision=precision) as g:
        ser = g.run(steps, dt)
        return g.state(), ser


@pytest.mark.parametrize("precision", [0, 1])
def test_pool_systems_match_standalone_bitwise(md, precision):
    mix = tersoff_mix()
    dt = 0.5
    with make_pool(md, precision) as pool:
        ids = [pool.add(s.pos, s.vel, s.box, s.pbc, pset, types_for(s)) for s, pset, _ in mix]
        ser = pool.run(24, dt, record=True)
        for (s, pset, _), sid in zip(mix, ids):
            (p1, v1), ser1 = standalone(md, s, 24, dt, precision)
            p2, v2 = pool.state(sid)
            assert np.array_equal(p1, p2) and np.array_equal(v1, v2), s.name
            assert np.array_equal(ser[:, sid, :], ser1), s.name


def test_pool_systems_match_oracle(md):
    mix = tersoff_mix()
    dt = 0.5
    with make_pool(md) as pool:
        ids = [pool.add(s.pos, s.vel, s.box, s.pbc, pset, types_for(s)) for s, pset, _ in mix]
        ser = pool.run(20, dt, record=True)
        for (s, pset, _), sid in zip(mix, ids):
            p_ref, v_ref, ser_ref = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 20, dt)
            p, v = pool.state(sid)
            d = p - p_ref
            d -= np.round(d / s.box) * s.box * s.pbc
            assert np.abs(d).max() < TRAJ_TOL and rel(v, v_ref) < TRAJ_TOL
            assert rel(ser[:, sid, :], ser_ref) < TRAJ_TOL


def test_step_budgets_stop_each_system_on_the_device(md):
    mix = tersoff_mix()[:3]
    budgets = [5, 13, 24]
    dt = 0.5
    with make_pool(md) as pool:
        ids = [pool.add(s.pos, s.vel, s.box, s.pbc, pset, types_for(s), n_steps=b)
               for (s, pset, _), b in zip(mix, budgets)]
        pool.run(24, dt)
        active, left, _, _ = pool.status()
        for (s, pset, _), sid, b in zip(mix, ids, budgets):
            assert active[sid] == 0 and left[sid] == 0
            (p1, v1), _ = standalone(md, s, b, dt)
            p2, v2 = pool.state(sid)
            assert np.array_equal(p1, p2) and np.array_equal(v1, v2), (s.name, b)


def test_continuous_admission_and_removal(md):
    """Systems join and leave between runs; each one's result equals its standalone run
    of the steps it was present for."""
    mix = tersoff_mix()
    dt = 0.5
    A, B, C, D = mix[0], mix[1], mix[2], mix[3]
    with make_pool(md, capacity=6000, max_systems=4) as pool:
        ia = pool.add(A[0].pos, A[0].vel, A[0].box, A[0].pbc, A[1], types_for(A[0]))
        ib = pool.add(B[0].pos, B[0].vel, B[0].box, B[0].pbc, B[1], types_for(B[0]))
        pool.run(10, dt)
        ic = pool.add(C[0].pos, C[0].vel, C[0].box, C[0].pbc, C[1], types_for(C[0]))
        pool.run(10, dt)
        pA = pool.state(ia)
        pool.remove(ia)
        idd = pool.add(D[0].pos, D[0].vel, D[0].box, D[0].pbc, D[1], types_for(D[0]))
        pool.run(10, dt)
        for (s, _, _), sid, steps, got in ((A, ia, 20, pA), (B, ib, 30, None), (C, ic, 20, None),
                                           (D, idd, 10, None)):
            st = got if got is not None else pool.state(sid)
            (p1, v1), _ = standalone(md, s, steps, dt)
            assert np.array_equal(p1, st[0]) and np.array_equal(v1, st[1]), s.name


def test_pool_full_reports_out_of_memory(md):
    s = I.si_diamond_tersoff(n=3)
    with make_pool(md, capacity=300, max_systems=2) as pool:
        pool.add(s.pos, s.vel, s.box, s.pbc, 0, types_for(s))
        with pytest.raises(md.MDError) as e:
            pool.add(s.pos, s.vel, s.box, s.pbc, 0, types_for(s))
        assert e.value.status == -4


def test_damped_relaxation_matches_oracle(md):
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.1)
    with make_pool(md) as pool:
        sid = pool.add(s.pos, s.vel, s.box, s.pbc, 0, types_for(s), damp=0.01)
        pool.run(30, 1.0)
        p, v = pool.state(sid)
    p_ref, v_ref, _ = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 30, 1.0, damp=0.01)
    d = p - p_ref
    d -= np.round(d / s.box) * s.box
    assert np.abs(d).max() < TRAJ_TOL and rel(v, v_ref) < TRAJ_TOL


@pytest.mark.parametrize("precision", [0, 1])
def test_sw_pool_with_deferred_atoms_matches_standalone(md, precision):
    """Hot, jittered SW cells whose heaviest atoms go to the full-capacity pass (one warp per
    atom, in a pool over the flattened index): bit for bit what each system gives alone."""
    systems = [I.si_diamond_sw(n=4, jitter_amp=0.12, temperature=900.0, seed_pos=k, seed_vel=k + 1)
               for k in (11, 13)]
    systems.append(I.si_diamond_sw(n=3, jitter_amp=0.12, temperature=900.0, seed_pos=15, seed_vel=16))
    with md.from_inputs(systems[0], precision=precision) as g:
        g.compute()
        assert g.stats().pair_deferred > 0
    with md.Pool(4000, 4, I.MD_SW, [I.SW_SI_1985], [I.MASS_SI], precision=precision) as pool:
        ids = [pool.add(s.pos, s.vel, s.box, s.pbc) for s in systems]
        pool.run(12, 1.0)
        for s, sid in zip(systems, ids):
            (p1, v1), _ = standalone(md, s, 12, 1.0, precision=precision)
            p2, v2 = pool.state(sid)
            assert np.array_equal(p1, p2) and np.array_equal(v1, v2)


def test_sw_pool_matches_standalone(md):
    systems = [I.si_diamond_sw(n=3, jitter_amp=0.05, seed_pos=k, seed_vel=k + 1) for k in (1, 3)]
    systems.append(I.si_diamond_sw(n=4, jitter_amp=0.05, seed_pos=5, seed_vel=6))
    with md.Pool(4000, 4, I.MD_SW, [I.SW_SI_1985], [I.MASS_SI]) as pool:
        ids = [pool.add(s.pos, s.vel, s.box, s.pbc) for s in systems]
        pool.run(16, 1.0)
        for s, sid in zip(systems, ids):
            (p1, v1), _ = standalone(md, s, 16, 1.0)
            p2, v2 = pool.state(sid)
            assert np.array_equal(p1, p2) and np.array_equal(v1, v2)
