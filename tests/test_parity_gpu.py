"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by
element, on the same seeded inputs.

Error metric (per-atom fields): max_i |a_i - b_i|_inf / max_i |b_i|_inf; scalars |a-b|/|b|.
Bounds: fp64 path 1e-12 on F, U_i, W_i, J_i and totals; trajectories 1e-10 after 50
steps; mixed path (fp32 pair arithmetic) 1e-5 on forces.
"""
import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
TRAJ_TOL = 1e-10
MIXED_TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    if b.size == 0:
        return 0.0
    den = np.abs(b).max()
    if den == 0.0:
        return float(np.abs(a).max())
    return float(np.abs(a - b).max() / den)


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03343_gb300 import _build, md as M
    _build.build()
    M.load()
    return M


def compare_compute(md, sysm, tol=FP64_TOL, precision=0, **kw):
    ref = O.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, sysm.params, sysm.vel)
    with md.from_inputs(sysm, precision=precision, **kw) as g:
        out = g.compute()
    errs = {k: rel(out[k], ref[k]) for k in ("F", "U", "W", "J")}
    errs["totals"] = rel(out["totals"], ref["totals"])
    for k, e in errs.items():
        assert e < tol, (sysm.name, k, e, errs)
    return errs


CASES = [
    ("tersoff_si_1728", lambda: I.si_diamond_tersoff(n=6)),
    ("tersoff_si_1000_ragged", lambda: I.si_diamond_tersoff(n=5, jitter_amp=0.1, seed_pos=3)),
    ("sw_si_216", lambda: I.si_diamond_sw(n=3, jitter_amp=0.1)),
    ("sw_si_4096_300K", lambda: I.si_diamond_sw(n=8, jitter_amp=0.08)),
    ("tersoff_c_graphene_960", lambda: I.c_graphene_tersoff(nx=10, ny=24)),
    ("tersoff_c_diamond_512", lambda: I.c_diamond_tersoff(n=4)),
    ("tersoff_cluster", lambda: I.cluster(I.si_diamond_tersoff(n=4, jitter_amp=0.1), 7.0)),
    ("sw_cluster", lambda: I.cluster(I.si_diamond_sw(n=4, jitter_amp=0.1), 7.0)),
    ("tersoff_tight_box", lambda: I.random_cell(14, [6.95, 7.0, 7.05], 2.0, I.MD_TERSOFF,
                                                I.TERSOFF_SI_1989, I.MASS_SI, 31)),
    ("sw_tight_box", lambda: I.random_cell(20, [8.7, 8.8, 8.9], 2.0, I.MD_SW, I.SW_SI_1985,
                                           I.MASS_SI, 33)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_compute_fp64_matches_oracle(md, name, make):
    compare_compute(md, make())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("lattice", ["jittered", "compressed"])
def test_atoms_with_many_bonds_take_the_full_capacity_pass(md, precision, lattice):
    """Atoms with more in-cutoff bonds than the common-case pass stages (SW: 8) are deferred
    to the full-capacity pass (one warp per atom).  Jittered SW silicon puts up to 10
    neighbours inside the cutoff (some atoms deferred, the rest in the common pass: every
    bond between the two passes must be seen from both ends); silicon compressed to
    a = 5.1 A brings the 12-atom second shell (3.61 A) inside the 3.77 A cutoff, 16 bonds
    per atom (all atoms deferred)."""
    if lattice == "jittered":
        s = I.si_diamond_sw(n=5, jitter_amp=0.1)
    else:
        s = I.si_diamond_sw(n=5, a=5.1, jitter_amp=0.05)
    ref = O.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
    with md.from_inputs(s, precision=precision) as g:
        out = g.compute()
        st = g.stats()
    if lattice == "jittered":
        assert 10 < st.pair_deferred < s.n // 2
    else:
        assert st.pair_deferred == s.n
    tol = FP64_TOL if precision == 0 else MIXED_TOL
    for k in ("F", "U", "W", "J"):
        assert rel(out[k], ref[k]) < tol, k
    # Newton's third law across the two passes: a bond seen from one end only would leave a
    # residue of the order of one bond's force; fp32 per-atom sums leave ~1e-7 of it
    newton = 1e-11 if precision == 0 else MIXED_TOL
    assert np.abs(out["F"].sum(axis=0)).max() < newton * np.abs(out["F"]).max()


def test_trajectory_with_deferred_atoms_matches_oracle(md):
    """NVE steps of hot SW silicon in which a few atoms per step go to the full-capacity
    pass: positions, velocities and the U, K, J series against the oracle."""
    s = I.si_diamond_sw(n=5, jitter_amp=0.1, temperature=900.0, seed_pos=7, seed_vel=8)
    steps, dt = 30, 1.0
    with md.from_inputs(s) as g:
        g.compute()
        assert g.stats().pair_deferred > 0
        ser = g.run(steps, dt)
        pos, vel = g.state()
    p2, v2, ser2 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt)
    d = pos - p2
    d -= np.round(d / s.box) * s.box * s.pbc
    assert np.abs(d).max() < TRAJ_TOL
    assert rel(vel, v2) < TRAJ_TOL
    for c in range(5):
        assert rel(ser[:, c], ser2[:, c]) < TRAJ_TOL, c


@pytest.mark.parametrize("name,make", CASES[:6], ids=[c[0] for c in CASES[:6]])
def test_compute_mixed_force_error(md, name, make):
    sysm = make()
    ref = O.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, sysm.params, sysm.vel)
    with md.from_inputs(sysm, precision=md.MD_MIXED) as g:
        out = g.compute()
    assert rel(out["F"], ref["F"]) < MIXED_TOL
    assert rel(out["U"], ref["U"]) < MIXED_TOL
    assert rel(out["W"], ref["W"]) < 1e-4
    assert rel(out["J"], ref["J"]) < 1e-4
    assert rel(out["totals"][:1], ref["totals"][:1]) < 1e-6


def test_empty_system(md):
    box = np.array([20.0, 20.0, 20.0])
    g = md.System(box, [1, 1, 1], 0, I.MD_TERSOFF, I.TERSOFF_SI_1989, I.MASS_SI)
    g.set_positions(np.zeros((0, 3)))
    g.set_velocities(np.zeros((0, 3)))
    out = g.compute()
    assert np.all(out["totals"] == 0.0)
    ser = g.run(3, 1.0)
    assert ser.shape == (3, 5) and np.all(ser == 0.0)
    g.close()


def test_single_atom_and_dimer(md):
    box = np.array([20.0, 20.0, 20.0])
    for pos in (np.array([[5.0, 5.0, 5.0]]), np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 7.35]]),
                np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 7.85]])):   # inside the f_C switch
        sysm = I.System("few", pos, box, np.array([0, 0, 0], np.int32), I.MD_TERSOFF,
                        I.TERSOFF_SI_1989, I.MASS_SI, np.zeros_like(pos))
        compare_compute(md, sysm)


def test_bitwise_deterministic(md):
    s = I.si_diamond_sw(n=5, jitter_amp=0.08)
    outs = []
    for _ in range(2):
        with md.from_inputs(s) as g:
            o = g.compute()
            ser = g.run(20, 1.0)
            outs.append((o["F"].copy(), o["W"].copy(), ser.copy(), g.state()[0]))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("make,steps,dt", [
    (lambda: I.si_diamond_tersoff(n=6), 50, 1.0),
    (lambda: I.si_diamond_sw(n=4, jitter_amp=0.05), 50, 1.0),
    (lambda: I.c_graphene_tersoff(nx=8, ny=14, jitter_amp=0.02), 40, 0.5),
], ids=["tersoff_si_1728", "sw_si_512", "graphene_448"])
def test_trajectory_matches_oracle(md, make, steps, dt):
    """50 NVE velocity-Verlet steps (the GPU keeps a skin list and rebuilds on the
    skin/2 rule; the oracle rebuilds from scratch every step)."""
    s = make()
    with md.from_inputs(s) as g:
        ser = g.run(steps, dt)
        pos, vel = g.state()
        st = g.stats()
    p2, v2, ser2 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt)
    d = pos - p2
    d -= np.round(d / s.box) * s.box * s.pbc
    assert np.abs(d).max() < TRAJ_TOL
    assert rel(vel, v2) < TRAJ_TOL
    for c in range(5):
        assert rel(ser[:, c], ser2[:, c]) < TRAJ_TOL, c
    assert st.steps_done == steps


MIXED_TRAJ = [
    ("tersoff_si_1728", lambda: I.si_diamond_tersoff(n=6), 1.0),
    ("tersoff_c_graphene_960", lambda: I.c_graphene_tersoff(nx=10, ny=24), 0.5),
    ("sw_si_1000", lambda: I.si_diamond_sw(n=5, jitter_amp=0.05), 1.0),
]


@pytest.mark.parametrize("name,make,dt", MIXED_TRAJ, ids=[c[0] for c in MIXED_TRAJ])
def test_mixed_trajectory_matches_oracle(md, name, make, dt):
    """Mixed path over 50 NVE steps against the fp64 oracle.  Bounds, from the force bound:
    a relative force error e < 1e-5 on forces of ~1 eV/A moves an atom of mass m by at most
    about (e/m) t^2/2 (acceleration unit 9.65e-3 A/fs^2 per eV/(A amu)), below 1e-5 A after
    50 fs for m >= 12 amu, so positions within 1e-4 A; the per-step energies carry fp32 sums
    of per-atom terms (relative 1e-7 each), so U and K within 1e-5 eV per atom; the heat
    current J = sum_i M_i v_i within 1e-3 of the series' largest |J| (fp32 per-atom products,
    and velocities that follow the slightly different forces)."""
    s = make()
    steps = 50
    with md.from_inputs(s, precision=1) as g:
        ser = g.run(steps, dt)
        pos, vel = g.state()
    p2, v2, ser2 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt)
    d = pos - p2
    d -= np.round(d / s.box) * s.box * s.pbc
    assert np.abs(d).max() < 1e-4
    for c in (0, 1):
        assert np.abs(ser[:, c] - ser2[:, c]).max() / s.n < 1e-5, c
    assert rel(ser[:, 2:5], ser2[:, 2:5]) < 1e-3


def test_rebuilds_happen_and_stay_exact(md):
    """A hot, small-skin run forces several list rebuilds; results still match."""
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=1500.0)
    with md.from_inputs(s, skin=0.1) as g:
        ser = g.run(60, 1.0)
        pos, _ = g.state()
        st = g.stats()
    assert st.n_rebuilds >= 3
    p2, v2, ser2 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 60, 1.0)
    d = pos - p2
    d -= np.round(d / s.box) * s.box
    assert np.abs(d).max() < TRAJ_TOL
    assert rel(ser, ser2) < TRAJ_TOL


def test_compute_after_run_continues_the_trajectory(md):
    """md_compute after md_run evaluates the state the run reached (graph-replayed steps
    leave positions unwrapped between list builds): compare with the oracle's own
    end state of the same trajectory."""
    s = I.si_diamond_tersoff(n=4, jitter_amp=0.05, temperature=900.0)
    with md.from_inputs(s, skin=0.2) as g:
        g.run(37, 1.0)
        out = g.compute()
    p2, v2, _ = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 37, 1.0)
    ref = O.compute(p2, s.box, s.pbc, s.kind, s.params, v2)
    for k in ("F", "U", "W", "J"):
        assert rel(out[k], ref[k]) < 1e-9, k


def test_list_overflow_is_reported(md):
    s = I.si_diamond_sw(n=3)
    with md.from_inputs(s, max_neigh=8) as g:     # SW lists hold 16 (4 + 12 second nbrs)
        with pytest.raises(md.MDError) as e:
            g.compute()
        assert e.value.status == -3


def test_device_io_matches_host_io(md):
    import torch
    s = I.si_diamond_tersoff(n=4)
    with md.from_inputs(s) as g:
        host = g.compute()
    g = md.System(s.box, s.pbc, s.n, s.kind, s.params, s.mass, io=md.MD_IO_DEVICE)
    g.set_positions(torch.tensor(s.pos, device="cuda"))
    g.set_velocities(torch.tensor(s.vel, device="cuda"))
    dev = g.compute()
    for k in ("F", "U", "W", "J"):
        assert np.array_equal(dev[k].cpu().numpy(), host[k])
    g.close()


FULL = [
    ("sw_si_512000", lambda j: I.si_diamond_sw(n=40, jitter_amp=j), 1.0),
    ("tersoff_c_graphene_1M", lambda j: I.c_graphene_tersoff(jitter_amp=j), 0.5),
]


@pytest.mark.parametrize("name,make,dt", FULL, ids=[f[0] for f in FULL])
def test_full_size_compute(md, name, make, dt):
    """Full-size workloads in the benchmark's launch configuration, jittered by
    +-0.02 A so that every per-atom field is non-trivial."""
    compare_compute(md, make(0.02))


def test_full_size_perfect_lattice_sw(md):
    """The unjittered 512,000-atom SW crystal at a = 5.431 A sits at the energy minimum:
    U_i = -2 epsilon to 1e-12 on both sides and every force vanishes to round-off."""
    s = I.si_diamond_sw(n=40)
    ref = O.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
    with md.from_inputs(s) as g:
        out = g.compute()
    assert rel(out["U"], ref["U"]) < FP64_TOL
    assert np.abs(out["F"]).max() < 1e-10 and np.abs(ref["F"]).max() < 1e-10


@pytest.mark.parametrize("name,make,dt", FULL, ids=[f[0] for f in FULL])
def test_full_size_trajectory(md, name, make, dt):
    """10 velocity-Verlet steps of the full-size benchmark workload, GPU (graph-replayed
    steps, skin list) against the oracle (list rebuilt every step)."""
    s = make(0.0 if name.startswith("sw") else 0.02)
    steps = 10
    with md.from_inputs(s) as g:
        ser = g.run(steps, dt)
        pos, vel = g.state()
    p2, v2, ser2 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt)
    d = pos - p2
    d -= np.round(d / s.box) * s.box * s.pbc
    assert np.abs(d).max() < TRAJ_TOL
    assert rel(vel, v2) < TRAJ_TOL
    for c in range(5):
        assert rel(ser[:, c], ser2[:, c]) < TRAJ_TOL, c


def test_profiling_records_every_kernel_class(md):
    """Per-kernel CUDA-event timing over graph-replayed (8) and eager (2) steps."""
    s = I.si_diamond_tersoff(n=4)
    with md.from_inputs(s) as g:
        md.md_set_profiling(g.ctx, True)
        g.run(10, 1.0)
        kt = md.md_kernel_times(g.ctx)
        st = g.stats()
    assert set(kt) == {"kick_drift", "rebuild", "pair", "gather", "reduce"}
    for name, (n, ms) in kt.items():
        assert n == 10 and ms > 0.0, (name, n, ms)
    assert st.kernel_launches_per_step >= 5


def test_eager_launches_match_graph_replay_bitwise(md):
    s = I.si_diamond_tersoff(n=4, jitter_amp=0.05, temperature=900.0)
    outs = []
    for graphs in (True, False):
        with md.from_inputs(s, skin=0.2) as g:
            md.md_set_graph_mode(g.ctx, graphs)
            ser = g.run(21, 1.0)
            pos, vel = g.state()
            st = g.stats()
            outs.append((ser, pos, vel, st.n_rebuilds))
    assert outs[0][3] == outs[1][3] and outs[0][3] >= 2
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert np.array_equal(a, b)
