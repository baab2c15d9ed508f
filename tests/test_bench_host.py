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
    """The roofline's per-bond and per-bond-pair FP64 flops are solved from ncu instruction
    counts of two states each (profiles/pair_*_fp64_*.md); they must give those counts back."""
    I_T, I_S = bench.I.MD_TERSOFF, bench.I.MD_SW
    for kind, bonds, pairs, counted in [
        (I_T, 3.0, 6.0, 551.449),        # C sheet
        (I_T, 4.0, 12.0, 822.266),       # Si diamond
        (I_S, 4.0, 12.0, 620.215),       # SW lattice
        (I_S, 5.0726, 21.5767, 947.165),  # SW after 100 fs at 300 K
    ]:
        assert bench.pair_flops(kind, bonds, pairs) == pytest.approx(counted, abs=0.02)
