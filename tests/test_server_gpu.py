"""Serving: jobs admitted into running pools as they arrive (continuous batching).
Each job's result must equal the same job run alone (bitwise), whatever else shared
the device with it."""
import time

import numpy as np
import pytest

from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03343_gb300 import _build, md as M
    _build.build()
    M.load()
    return M


TSETS = [I.TERSOFF_SI_1989, I.TERSOFF_C_1989]
TMASS = [I.MASS_SI, I.MASS_C]
DT = {I.MD_TERSOFF: 0.5, I.MD_SW: 1.0}


def jobs():
    out = []
    rng = np.random.default_rng(4)
    makers = [
        lambda k: (I.MD_TERSOFF, 0, I.si_diamond_tersoff(n=2 + k % 3, jitter_amp=0.05, seed_pos=k, seed_vel=k + 50)),
        lambda k: (I.MD_TERSOFF, 1, I.c_graphene_tersoff(nx=3 + k % 4, ny=5 + k % 3, jitter_amp=0.02, seed_pos=k,
                                                         seed_vel=k + 50)),
        lambda k: (I.MD_SW, 0, I.si_diamond_sw(n=2 + k % 2, jitter_amp=0.05, seed_pos=k, seed_vel=k + 50)),
    ]
    for k in range(12):
        kind, pset, s = makers[k % 3](k)
        steps = int(rng.integers(10, 60))
        damp = 0.01 if k % 4 == 3 else 0.0
        out.append((kind, pset, s, steps, damp))
    return out


def alone(md, precision, kind, pset, s, steps, damp):
    if kind == I.MD_TERSOFF:
        pool = md.Pool(s.n + 128, 1, kind, TSETS, TMASS, precision=precision)
        types = np.full(s.n, pset, np.int32)
    else:
        pool = md.Pool(s.n + 128, 1, kind, [I.SW_SI_1985], [I.MASS_SI], precision=precision)
        types = None
    with pool:
        sid = pool.add(s.pos, s.vel, s.box, s.pbc, pset, types, n_steps=steps, damp=damp)
        pool.run(steps, DT[kind])
        return pool.state(sid)


@pytest.mark.parametrize("precision", [1, 0])
def test_served_jobs_equal_their_standalone_runs(md, precision):
    js = jobs()
    with md.Server(precision=precision, tersoff_atoms=3000, sw_atoms=1200, max_jobs_per_pool=8,
                   tersoff_dt=DT[I.MD_TERSOFF], sw_dt=DT[I.MD_SW], tersoff_sets=TSETS, tersoff_masses=TMASS,
                   sw_set=[I.SW_SI_1985], sw_mass=[I.MASS_SI]) as srv:
        ids = []
        for k, (kind, pset, s, steps, damp) in enumerate(js):
            types = np.full(s.n, pset, np.int32) if kind == I.MD_TERSOFF else None
            ids.append(srv.submit(kind, s.pos, s.vel, s.box, s.pbc, steps, pset, types, damp))
            if k % 3 == 2:
                time.sleep(0.02)    # later jobs arrive while earlier ones run
        results = [srv.wait(j) for j in ids]
        st = srv.stats()
    assert st.completed == len(js) and st.failed == 0
    assert abs(st.atom_steps - sum(s.n * steps for _, _, s, steps, _ in js)) < 1e-6
    for (kind, pset, s, steps, damp), (r, state) in zip(js, results):
        assert r.status == 0 and r.done == 1
        assert r.t_submit <= r.t_admit <= r.t_done
        p_ref, v_ref = alone(md, precision, kind, pset, s, steps, damp)
        assert np.array_equal(state[0], p_ref) and np.array_equal(state[1], v_ref), (s.name, steps, damp)


def test_job_larger_than_its_pool_fails_cleanly(md):
    s = I.si_diamond_tersoff(n=4)   # 512 atoms
    with md.Server(precision=1, tersoff_atoms=256, max_jobs_per_pool=2, tersoff_sets=TSETS,
                   tersoff_masses=TMASS) as srv:
        jid = srv.submit(I.MD_TERSOFF, s.pos, s.vel, s.box, s.pbc, 5, 0, np.zeros(s.n, np.int32))
        r, _ = srv.wait(jid)
        assert r.done == 1 and r.status == -4
