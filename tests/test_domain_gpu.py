"""Spatial decomposition on the GPU: one system in slabs over 2-4 ranks, each rank with its
ghost shell, against the undivided system and the oracle.

- one force evaluation: per-atom F, U, W, J (by atom id) and the summed totals equal the
  oracle's at the fp64 bound 1e-12 (only the order of the bonds in the sums differs);
- trajectories with list rebuilds and atoms migrating between slabs equal the oracle's at
  the trajectory bound 1e-10;
- the ranks as separate processes with a gloo transport (host-staged messages) give, bit for
  bit, the run of all ranks held in one process (the same per-rank arithmetic).
Every rank's kernels read only that rank's memory; ranks never wait on one another inside a
kernel (all messages pass through the host between launches)."""
import json
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FP64_TOL = 1e-12
TRAJ_TOL = 1e-10
MIXED_TOL = 1e-5


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


CASES = {
    "tersoff_si_2": (lambda: I.si_diamond_tersoff(n=6, jitter_amp=0.08), 0, 2),
    "tersoff_si_3_y": (lambda: I.si_diamond_tersoff(n=8, jitter_amp=0.08), 1, 3),
    "graphene_4": (lambda: I.c_graphene_tersoff(nx=12, ny=24), 0, 4),
    "sw_si_2_z": (lambda: I.si_diamond_sw(n=7, jitter_amp=0.08), 2, 2),
}


@pytest.mark.parametrize("case", list(CASES), ids=list(CASES))
def test_decomposed_compute_matches_oracle(md, case):
    make, axis, ranks = CASES[case]
    s = make()
    ref = O.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
    with md.DomainGroup(s.box, s.pbc, axis, ranks, s.n, s.kind, s.params, s.mass) as grp:
        grp.start(s.pos, s.vel)
        out = grp.compute(s.n)
        owned = [len(md.md_domain_owned(d)[0]) for d in grp.doms]
    assert sum(owned) == s.n and min(owned) > 0
    for k in ("F", "U", "W", "J"):
        assert not np.isnan(out[k]).any(), k
        assert rel(out[k], ref[k]) < FP64_TOL, (k, rel(out[k], ref[k]))
    assert rel(out["totals"], ref["totals"]) < FP64_TOL


def test_decomposed_mixed_precision_forces(md):
    s = I.c_graphene_tersoff(nx=12, ny=24)
    ref = O.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
    with md.DomainGroup(s.box, s.pbc, 0, 3, s.n, s.kind, s.params, s.mass, precision=md.MD_MIXED) as grp:
        grp.start(s.pos, s.vel)
        out = grp.compute(s.n)
    assert rel(out["F"], ref["F"]) < MIXED_TOL


TRAJ = {
    "tersoff_si_2": (lambda: I.si_diamond_tersoff(n=6, jitter_amp=0.1, temperature=600.0), 0, 2, 1.0, 0.2),
    "graphene_3": (lambda: I.c_graphene_tersoff(nx=12, ny=24, temperature=600.0), 0, 3, 0.5, 0.12),
    "sw_si_2": (lambda: I.si_diamond_sw(n=7, jitter_amp=0.08, temperature=600.0), 1, 2, 1.0, 0.2),
}


@pytest.mark.parametrize("case", list(TRAJ), ids=list(TRAJ))
def test_decomposed_trajectory_with_migrations_matches_oracle(md, case):
    make, axis, ranks, dt, skin = TRAJ[case]
    s = make()
    steps = 60
    with md.DomainGroup(s.box, s.pbc, axis, ranks, s.n, s.kind, s.params, s.mass, skin=skin) as grp:
        grp.start(s.pos, s.vel)
        owners0 = [set(md.md_domain_owned(d)[0].tolist()) for d in grp.doms]
        ser = grp.run(steps, dt)
        x, v = grp.state(s.n)
        owners1 = [set(md.md_domain_owned(d)[0].tolist()) for d in grp.doms]
        rebuilds = grp.rebuilds
    assert rebuilds >= 2
    assert owners0 != owners1, "no atom changed slab: the migration path was not exercised"
    p2, v2, ser2 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, steps, dt)
    d = x - p2
    d -= np.round(d / s.box) * s.box * s.pbc
    assert np.abs(d).max() < TRAJ_TOL
    assert rel(v, v2) < TRAJ_TOL
    for c in range(5):
        assert rel(ser[:, c], ser2[:, c]) < TRAJ_TOL, c


def test_decomposition_rejects_thin_slabs_and_open_axes(md):
    s = I.si_diamond_tersoff(n=6)
    with pytest.raises(md.MDError) as e:      # 3 slabs of 10.9 A < 2 x 6.9 A ghost shells
        md.DomainGroup(s.box, s.pbc, 0, 3, s.n, s.kind, s.params, s.mass)
    assert e.value.status == -2
    with pytest.raises(md.MDError) as e:
        md.DomainGroup(s.box, np.array([0, 1, 1]), 0, 2, s.n, s.kind, s.params, s.mass)
    assert e.value.status == -1


def test_capacity_overflow_is_reported(md):
    s = I.si_diamond_tersoff(n=6)
    with md.DomainGroup(s.box, s.pbc, 0, 2, 900, s.kind, s.params, s.mass) as grp:   # 864 owned + ghosts
        with pytest.raises(md.MDError) as e:
            grp.start(s.pos, s.vel)
        assert e.value.status == -4


# -------------------------------------------------------------- ranks as processes
def free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, out_dir, steps):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1610_03343_gb300 import inputs, md as M
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    s = inputs.si_diamond_tersoff(n=6, jitter_amp=0.1, temperature=600.0)
    with M.Domain(M.DistTransport(), s.box, s.pbc, 0, s.n, s.kind, s.params, s.mass, skin=0.2) as dom:
        dom.start(s.pos, s.vel)
        ser = dom.run(steps, 1.0)
        ids, x, v = dom.owned()
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), ser=ser, ids=ids, x=x, v=v, rebuilds=dom.rebuilds)
    dist.barrier()
    dist.destroy_process_group()


def test_ranks_as_processes_match_the_in_process_group(md, tmp_path):
    import torch.multiprocessing as mp
    steps = 40
    mp.start_processes(_rank, args=(2, free_port(), str(tmp_path), steps), nprocs=2, start_method="spawn")
    s = I.si_diamond_tersoff(n=6, jitter_amp=0.1, temperature=600.0)
    with md.DomainGroup(s.box, s.pbc, 0, 2, s.n, s.kind, s.params, s.mass, skin=0.2) as grp:
        grp.start(s.pos, s.vel)
        ser = grp.run(steps, 1.0)
        x, v = grp.state(s.n)
    xs = np.full_like(x, np.nan)
    vs = np.full_like(v, np.nan)
    for r in range(2):
        z = np.load(tmp_path / f"r{r}.npz")
        assert np.array_equal(z["ser"], ser)
        xs[z["ids"]] = z["x"]
        vs[z["ids"]] = z["v"]
        assert int(z["rebuilds"]) == grp.rebuilds
    assert np.array_equal(xs, x) and np.array_equal(vs, v)
