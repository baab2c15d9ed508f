"""bench.py's host-side bookkeeping for the roofline: the in-cutoff bond statistics that
scale the pair pass's per-bond and per-bond-pair flop counts.  Pinned to lattices whose
neighbour shells are known exactly (diamond: 4 nearest neighbours at a sqrt(3)/4, 12 next at
a/sqrt(2); honeycomb: 3 at a_cc, 6 next at sqrt(3) a_cc), and to a brute-force count over
all periodic images on a small jittered cell."""
import itertools
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1610_03343_gb300 import inputs as I  # noqa: E402

pytest.importorskip("scipy")
import bench  # noqa: E402


def test_diamond_first_shell_only():
    pos, box = I.diamond_positions(3, 5.431)
    m, mm = bench.bond_statistics(pos, box, np.array([1, 1, 1]), 3.77118)
    assert (m, mm) == (4.0, 12.0)


def test_diamond_compressed_second_shell_inside():
    # a = 5.1: second shell at 3.606 A inside 3.77 A, third at 4.23 A outside
    pos, box = I.diamond_positions(3, 5.1)
    m, mm = bench.bond_statistics(pos, box, np.array([1, 1, 1]), 3.77118)
    assert (m, mm) == (16.0, 240.0)


def test_honeycomb_sheet_with_open_axis():
    pos, box = I.graphene_positions(6, 6, 1.42, 20.0)
    for pbc in ([1, 1, 1], [1, 1, 0]):
        m, mm = bench.bond_statistics(pos, box, np.array(pbc), 2.1)
        assert (m, mm) == (3.0, 6.0), pbc
    # open in-plane axis: the atoms on the cut edge lose their bonds across it
    m, _ = bench.bond_statistics(pos, box, np.array([0, 1, 1]), 2.1)
    assert m < 3.0


def test_matches_brute_force_over_images():
    rng = np.random.Generator(np.random.PCG64(5))
    pos, box = I.diamond_positions(2, 5.3)
    pos = pos + rng.uniform(-0.25, 0.25, pos.shape)     # some atoms outside [0, L)
    rc = 3.77118
    n = pos.shape[0]
    cnt = np.zeros(n)
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            for s in itertools.product((-1, 0, 1), repeat=3):
                d = pos[j] + np.array(s) * box - pos[i]
                if d @ d < rc * rc:
                    cnt[i] += 1
    m, mm = bench.bond_statistics(pos, box, np.array([1, 1, 1]), rc)
    assert m == pytest.approx(cnt.mean(), abs=0)
    assert mm == pytest.approx((cnt * (cnt - 1)).mean(), abs=0)


def test_flop_model_reproduces_the_counted_launches():
    """The roofline's per-bond and per-bond-pair FP64 flops and issue slots are solved from ncu
    instruction counts of two states each (profiles/pair_*_fp64_*.md); they must give those
    counts back (flop = DADD + DMUL + 2 DFMA; slots = warp instructions x 32, per atom)."""
    I_T, I_S = bench.I.MD_TERSOFF, bench.I.MD_SW
    for kind, bonds, pairs, flop, fp64, issue in [
        (I_T, 3.0, 6.0, 143.012, 3.482252 * 32, 180.557976 * 32),                 # C sheet
        (I_T, 4.0, 12.0, 203.167, 4.958065 * 32, 276.845213 * 32),                # Si diamond
        (I_S, 4.0, 12.0, 196.250, 5.241750 * 32, (243.885 + 0.418) * 32),          # SW lattice
        (I_S, 5.1028, 21.8819, 253.673, (9.282328 + 0.318531) * 32, (584.584 + 3.086) * 32),  # SW, 300 K
    ]:
        assert bench.pair_flops(kind, bonds, pairs) == pytest.approx(flop, abs=0.02)
        s64, sall = bench.pair_slots(kind, bonds, pairs)
        assert s64 == pytest.approx(fp64, abs=0.05)
        assert sall == pytest.approx(issue, abs=0.5)


def test_pipe_model_takes_the_slower_pipe():
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 64.0}
    pm = bench.pipe_model(bench.I.MD_TERSOFF, 3.0, 6.0, 1_000_000, peaks)
    s64, sall = bench.pair_slots(bench.I.MD_TERSOFF, 3.0, 6.0)
    assert pm["t_fp64_pipe_us"] == pytest.approx(s64 * 1e6 / 0.5e12 * 1e6)
    assert pm["t_issue_us"] == pytest.approx(sall * 1e6 / 32 / 1e12 * 1e6)
    assert pm["t_model_us"] == max(pm["t_fp64_pipe_us"], pm["t_issue_us"])
    assert pm["bound_pipe"] == ("fp64" if pm["t_fp64_pipe_us"] >= pm["t_issue_us"] else "issue")
