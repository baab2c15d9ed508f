"""The seeded synthetic inputs have the shapes of the paper's workloads (Sec. 3)."""
import numpy as np

from paper_1610_03343_gb300 import inputs as I


def test_diamond_counts_and_box():
    s = I.si_diamond_tersoff(n=6)
    assert s.n == 1728 and np.allclose(s.box, 6 * 5.432)
    assert np.all(s.pos >= 0) and np.all(s.pos < s.box)


def test_graphene_counts_and_box():
    s = I.c_graphene_tersoff(nx=5, ny=7)
    assert s.n == 4 * 35
    assert np.allclose(s.box, [5 * 3 * 1.42, 7 * np.sqrt(3) * 1.42, 20.0])


def test_maxwell_boltzmann_exact_temperature_zero_momentum():
    v = I.maxwell_boltzmann(1000, I.MASS_SI, 300.0, 4)
    assert np.abs(v.sum(axis=0)).max() < 1e-12
    ke = 0.5 * I.MASS_SI * np.sum(v * v) / I.EV_PER_A_AMU_TO_A_PER_FS2
    t = 2 * ke / ((3 * 1000 - 3) * I.KB_EV_PER_K)
    assert abs(t - 300.0) < 1e-9


def test_seeded_reproducible():
    a = I.si_diamond_tersoff(n=2, seed_pos=5)
    b = I.si_diamond_tersoff(n=2, seed_pos=5)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)


def test_batch_sizes_admissible():
    sizes = I.batch_sizes(512, 64, 20000, 7)
    tot = sum(s[3] for s in sizes)
    assert 0.8e6 < tot < 3.5e6
    for kind, a, b, n in sizes:
        assert n == (8 * a ** 3 if kind == "si_diamond" else 4 * a * b)
