"""bench.py's multi-GPU path (one replica per rank, launched under torchrun) on two gloo
ranks on the CPU: the max-over-ranks reduction of the timed region, the whole-job value, and
the reference arm, which rank 0 alone runs and prints while the other rank exits without
work.  (The replicas themselves need GPUs; every box here has one, so the CUDA side of the
N > 1 path is tested only through these host pieces.)"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    vals = bench.reduce_max_over_ranks([1.0 + rank, 10.0 - rank, 3.0], world, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(vals, f)
    dist.barrier()
    dist.destroy_process_group()


def _reference_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    sys.argv = ["bench.py", "--impl", "reference", "--gpus", str(world), "--steps", "1", "--warmup", "0"]
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.main()
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as f:
        f.write(buf.getvalue())


def _spawn(fn, world, tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mp.spawn(fn, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)


def test_max_over_two_gloo_ranks(tmp_path):
    _spawn(_reduce_worker, 2, tmp_path)
    for r in range(2):
        assert json.load(open(tmp_path / f"r{r}.json")) == [2.0, 10.0, 3.0]


def test_job_value_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(1, 1000, 10, 1.0) == pytest.approx(1.0e7)
    assert bench.job_value(4, 1000, 10, 2.0) == pytest.approx(2.0e7)   # 4 replicas, slowest 2 ms
    assert bench.reduce_max_over_ranks([1.5, 2.5], 1, "cpu") == [1.5, 2.5]


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    _spawn(_reference_worker, 2, tmp_path)
    out0 = (tmp_path / "ref0.txt").read_text().strip().splitlines()
    out1 = (tmp_path / "ref1.txt").read_text().strip()
    assert len(out0) == 1 and out1 == ""
    line = json.loads(out0[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["unit"] == "atom-steps/s" and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
