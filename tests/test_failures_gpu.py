"""Failure paths and state handling that run safely on a GPU: every failure here is a
value the kernels report (a non-finite number, an overlong list) or a host-side limit (an
allocation budget, a deadline) -- nothing traps, faults or hangs.

- coincident atoms give a zero-length bond, whose 1/r is +inf: the forces turn non-finite
  and the call returns MD_ERR_NAN; the context is usable again after new positions;
- a non-finite position or velocity is reported as MD_ERR_NAN (a NaN position has no bond
  inside the cutoff, so its force alone would be a silent zero);
- an hbm_budget below the footprint fails with MD_ERR_OOM and leaks nothing;
- a checkpoint restored into a fresh context continues bitwise like the uninterrupted run;
- md_server_wait_timeout returns MD_ERR_TIMEOUT for a job that is not done in time;
- in a pool or the server, one failing system fails alone: the others end bitwise as they
  would without it.
"""
import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MD_ERR_NAN, MD_ERR_OOM, MD_ERR_ARG, MD_ERR_TIMEOUT = -7, -4, -1, -6


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


def coincident(s, i=5, j=6):
    """s with atom j moved onto atom i."""
    pos = s.pos.copy()
    pos[j] = pos[i]
    return pos


# ------------------------------------------------------------------ non-finite values
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("make", [lambda: I.si_diamond_tersoff(n=3), lambda: I.si_diamond_sw(n=3, jitter_amp=0.05)],
                         ids=["tersoff", "sw"])
def test_coincident_atoms_report_nan_and_the_context_recovers(md, precision, make):
    s = make()
    with md.from_inputs(s, precision=precision) as g:
        g.set_positions(coincident(s))
        with pytest.raises(md.MDError) as e:
            g.compute()
        assert e.value.status == MD_ERR_NAN
        with pytest.raises(md.MDError) as e:
            g.run(5, 1.0)
        assert e.value.status == MD_ERR_NAN
        # new positions: the context computes again
        g.set_positions(s.pos)
        g.set_velocities(s.vel)
        out = g.compute()
    if precision == 0:
        ref = O.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
        for k in ("F", "U", "W", "J"):
            assert rel(out[k], ref[k]) < FP64_TOL, k


@pytest.mark.parametrize("field", ["position", "velocity"])
def test_nonfinite_input_reports_nan(md, field):
    s = I.si_diamond_tersoff(n=3)
    with md.from_inputs(s) as g:
        if field == "position":
            pos = s.pos.copy()
            pos[17, 1] = np.nan
            g.set_positions(pos)
        else:
            vel = s.vel.copy()
            vel[23, 2] = np.inf
            g.set_velocities(vel)
        with pytest.raises(md.MDError) as e:
            g.compute()
        assert e.value.status == MD_ERR_NAN


# ------------------------------------------------------------------ allocation budget
def test_hbm_budget_below_the_footprint_fails_without_leaking(md):
    import torch
    s = I.si_diamond_tersoff(n=30)     # 216,000 atoms: a leak would show in free memory
    with md.from_inputs(s) as g:
        need = g.stats().device_bytes
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        with pytest.raises(md.MDError) as e:
            md.System(s.box, s.pbc, s.n, s.kind, s.params, s.mass, hbm_budget=need - 1)
        assert e.value.status == MD_ERR_OOM
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < need // 4, (free0, free1, need)
    # exactly the footprint: creation and steps fit, the per-atom W and J of md_compute do not
    with md.System(s.box, s.pbc, s.n, s.kind, s.params, s.mass, hbm_budget=need) as g:
        g.set_positions(s.pos)
        g.set_velocities(s.vel)
        g.run(3, 1.0)
        with pytest.raises(md.MDError) as e:
            g.compute()
        assert e.value.status == MD_ERR_OOM
        assert g.stats().device_bytes <= need
        g.run(3, 1.0)                    # still usable


# ------------------------------------------------------------------ checkpoint / resume
CK_CASES = {
    "tersoff_fp64": (lambda: I.si_diamond_tersoff(n=4, jitter_amp=0.08), 0, 1.0, {}),
    "tersoff_mixed": (lambda: I.si_diamond_tersoff(n=4, jitter_amp=0.08), 1, 1.0, {}),
    "sw_fp64": (lambda: I.si_diamond_sw(n=4, jitter_amp=0.08), 0, 1.0, {}),
    "graphene_eager": (lambda: I.c_graphene_tersoff(nx=8, ny=12), 0, 0.5, {"eager": True}),
    "tersoff_npt": (lambda: I.si_diamond_tersoff(n=4, jitter_amp=0.08), 0, 1.0, {"npt": True}),
}


@pytest.mark.parametrize("case", list(CK_CASES), ids=list(CK_CASES))
def test_checkpoint_resume_is_bitwise(md, case):
    make, precision, dt, opts = CK_CASES[case]
    s = make()
    kw = dict(precision=precision, skin=0.12)     # a thin skin: rebuilds on both sides of the cut

    def new():
        g = md.System(s.box, s.pbc, s.n, s.kind, s.params, s.mass, **kw)
        if opts.get("eager"):
            md.md_set_graph_mode(g.ctx, False)
        return g

    with new() as a:
        a.set_positions(s.pos)
        a.set_velocities(s.vel)
        if opts.get("npt"):
            a.set_npt(T0=300.0, P0=0.0, tau_T=50.0, tau_P=500.0, beta=0.01)
        a.run(37, dt)
        image = a.checkpoint()
        r0 = a.stats().n_rebuilds
        ser_a = a.run(45, dt)
        assert a.stats().n_rebuilds > r0          # the continuation rebuilt its list
        xa, va = a.state()
        box_a = a.box()
        # the same context rewound to the checkpoint repeats the continuation
        a.restore(image)
        ser_a2 = a.run(45, dt)
        assert np.array_equal(ser_a, ser_a2)
    with new() as b:
        b.restore(image)
        ser_b = b.run(45, dt)
        xb, vb = b.state()
        assert np.array_equal(box_a, b.box())
    assert np.array_equal(ser_a, ser_b)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_checkpoint_rejects_a_different_context(md):
    s = I.si_diamond_tersoff(n=3)
    with md.from_inputs(s) as a:
        image = a.checkpoint()
    other = I.si_diamond_tersoff(n=4)
    for kw in (dict(), dict(precision=1)):
        src = other if not kw else s
        with md.System(src.box, src.pbc, src.n, src.kind, src.params, src.mass, **kw) as b:
            with pytest.raises(md.MDError) as e:
                b.restore(image)
            assert e.value.status == MD_ERR_ARG
    with md.System(s.box, s.pbc, s.n, s.kind, s.params, s.mass) as b:
        with pytest.raises(md.MDError) as e:
            b.restore(image[: len(image) // 2])
        assert e.value.status == MD_ERR_ARG


# ------------------------------------------------------------------ pools and serving
TSETS = [I.TERSOFF_SI_1989, I.TERSOFF_C_1989]
TMASS = [I.MASS_SI, I.MASS_C]


def pool_run(md, members, steps, precision):
    """members: (system, positions) pairs added to one pool in order; returns the pool's
    per-slot errors and each member's final state (None for a failed one)."""
    with md.Pool(12000, 8, I.MD_TERSOFF, TSETS, TMASS, precision=precision) as pool:
        ids = [pool.add(pos, s.vel, s.box, s.pbc, 0, np.zeros(s.n, np.int32), n_steps=steps)
               for s, pos in members]
        pool.run(steps, 1.0)
        err = pool.errors()
        active, _, _, _ = pool.status()
        states = [None if err[k] else pool.state(k) for k in ids]
        return [int(err[k]) for k in ids], [int(active[k]) for k in ids], states


@pytest.mark.parametrize("precision", [0, 1])
def test_pool_system_with_coincident_atoms_fails_alone(md, precision):
    good = [I.si_diamond_tersoff(n=3, jitter_amp=0.05, seed_pos=20 + k, seed_vel=40 + k) for k in range(3)]
    bad = I.si_diamond_tersoff(n=3, jitter_amp=0.05, seed_pos=30, seed_vel=31)
    steps = 24
    err, active, states = pool_run(md, [(good[0], good[0].pos), (bad, coincident(bad)), (good[1], good[1].pos),
                                        (good[2], good[2].pos)], steps, precision)
    assert err == [0, MD_ERR_NAN, 0, 0]
    assert active[1] == 0
    for k, s in ((0, good[0]), (2, good[1]), (3, good[2])):
        _, _, ref = pool_run(md, [(s, s.pos)], steps, precision)
        assert np.array_equal(states[k][0], ref[0][0]) and np.array_equal(states[k][1], ref[0][1])


def test_pool_rejects_nonfinite_input_at_admission(md):
    s = I.si_diamond_tersoff(n=2)
    pos = s.pos.copy()
    pos[3, 0] = np.nan
    with md.Pool(2000, 4, I.MD_TERSOFF, TSETS, TMASS) as pool:
        with pytest.raises(md.MDError) as e:
            pool.add(pos, s.vel, s.box, s.pbc, 0, np.zeros(s.n, np.int32))
        assert e.value.status == MD_ERR_NAN
        assert (pool.status()[0] == -1).all()       # nothing was admitted


def test_served_job_with_bad_input_fails_alone(md):
    """Among good jobs, one with coincident atoms (found on the device) and one with a NaN
    position (rejected at admission) fail with MD_ERR_NAN; every other job ends bitwise as
    the same job run alone."""
    good = [I.si_diamond_tersoff(n=2 + k % 2, jitter_amp=0.05, seed_pos=60 + k, seed_vel=70 + k) for k in range(5)]
    bad_dev = I.si_diamond_tersoff(n=3, jitter_amp=0.05, seed_pos=80, seed_vel=81)
    bad_host = I.si_diamond_tersoff(n=2, jitter_amp=0.05, seed_pos=82, seed_vel=83)
    host_pos = bad_host.pos.copy()
    host_pos[1, 2] = np.nan
    jobs = [(s, s.pos, 30 + 4 * k) for k, s in enumerate(good)]
    jobs.insert(2, (bad_dev, coincident(bad_dev), 25))
    jobs.insert(4, (bad_host, host_pos, 25))
    with md.Server(precision=1, tersoff_atoms=6000, max_jobs_per_pool=8, tersoff_dt=1.0, tersoff_sets=TSETS,
                   tersoff_masses=TMASS) as srv:
        ids = [srv.submit(I.MD_TERSOFF, pos, s.vel, s.box, s.pbc, steps, 0, np.zeros(s.n, np.int32))
               for s, pos, steps in jobs]
        results = [srv.wait(j) for j in ids]
        st = srv.stats()
    assert st.failed == 2 and st.completed == len(jobs) - 2
    for (s, pos, steps), (r, state) in zip(jobs, results):
        assert r.done == 1
        if s is bad_dev or s is bad_host:
            assert r.status == MD_ERR_NAN
            continue
        assert r.status == 0
        with md.Pool(s.n + 128, 1, I.MD_TERSOFF, TSETS, TMASS, precision=1) as pool:
            sid = pool.add(s.pos, s.vel, s.box, s.pbc, 0, np.zeros(s.n, np.int32), n_steps=steps)
            pool.run(steps, 1.0)
            ref = pool.state(sid)
        assert np.array_equal(state[0], ref[0]) and np.array_equal(state[1], ref[1])


def test_server_wait_timeout(md):
    s = I.si_diamond_tersoff(n=6)
    with md.Server(precision=1, tersoff_atoms=4000, max_jobs_per_pool=2, tersoff_dt=1.0, tersoff_sets=TSETS,
                   tersoff_masses=TMASS) as srv:
        jid = srv.submit(I.MD_TERSOFF, s.pos, s.vel, s.box, s.pbc, 4000, 0, np.zeros(s.n, np.int32))
        st, r = md.md_server_wait_timeout(srv.srv, jid, 0.0)
        assert st == MD_ERR_TIMEOUT and r.done == 0
        st, r = md.md_server_wait_timeout(srv.srv, jid, 120.0)
        assert st == 0 and r.done == 1 and r.status == 0
        srv.wait(jid)
