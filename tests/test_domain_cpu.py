"""Spatial decomposition, host side: how messages travel between slab ranks.  A rank sends
one message to its left neighbour and one to its right; it must receive, as `from_left`, what
its left neighbour sent right and, as `from_right`, what its right neighbour sent left --
also when both neighbours are the same rank (two ranks).  Checked for the in-memory routing
and for the torch.distributed transport on 2 and 3 gloo ranks (CPU), together with the
transport's OR and rank-ordered sum."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def label(src, direction):
    return np.frombuffer(f"{src}:{direction}".encode(), dtype=np.uint8).copy()


def decode(a):
    return bytes(np.asarray(a, dtype=np.uint8)).decode()


@pytest.mark.parametrize("n", [2, 3, 5])
def test_route_pairs_neighbours(n):
    from paper_1610_03343_gb300.md import domain_route
    inbox = domain_route([(label(r, "L"), label(r, "R")) for r in range(n)])
    for r, (fl, fr) in enumerate(inbox):
        assert decode(fl) == f"{(r - 1) % n}:R"
        assert decode(fr) == f"{(r + 1) % n}:L"


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1610_03343_gb300.md import DistTransport
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t = DistTransport()
    res = {}
    for mode in (0, 1, 2):
        # messages of different lengths in the two directions
        fl, fr = t.exchange(mode, label(rank, f"L{mode}"), label(rank, f"R{mode}" + "x" * rank))
        res[f"m{mode}"] = [decode(fl), decode(fr)]
    res["any0"] = t.any(False)
    res["any1"] = t.any(rank == world - 1)
    res["sum"] = t.sum(np.array([1.0 + rank, 10.0 ** rank])).tolist()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_dist_transport_on_gloo_ranks(tmp_path, world):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        res = json.load(open(tmp_path / f"r{r}.json"))
        left, right = (r - 1) % world, (r + 1) % world
        for mode in (0, 1, 2):
            assert res[f"m{mode}"][0] == f"{left}:R{mode}" + "x" * left
            assert res[f"m{mode}"][1] == f"{right}:L{mode}"
        assert res["any0"] is False and res["any1"] is True
        want = [sum(1.0 + q for q in range(world)), sum(10.0 ** q for q in range(world))]
        assert res["sum"] == want
