"""Pins of the Green-Kubo oracle (oracle/green_kubo.py) against results fixed by the
mathematics rather than by its own formula: closed forms of constant and periodic
series, the Wiener-Khinchin route through numpy's FFT, exactness of the trapezoid rule
on a linear integrand, the decay integral of an exponential HCACF, and the unit
conversion redone in SI units."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import green_kubo as GK


def test_constant_series_closed_form():
    T = 50
    j = np.tile([0.3, -1.5, 2.0], (T, 1))
    c = O.hcacf(j, 20)
    assert np.allclose(c, np.tile([0.09, 2.25, 4.0], (20, 1)), rtol=1e-14, atol=0)
    k = O.running_kappa(c, 0.5, 1000.0, 300.0)
    pref = GK.EV_PER_FS_A_K_TO_W_PER_M_K / (GK.K_B * 300.0 ** 2 * 1000.0)
    m = np.arange(20)[:, None]
    assert np.allclose(k, pref * np.array([0.09, 2.25, 4.0]) * m * 0.5, rtol=1e-13, atol=0)


def test_periodic_series_closed_form():
    """cos(2 pi t / 8): the cross term sum_{t<n} cos(w(2t+m)) vanishes when n = T - m is a
    multiple of 4, leaving C(m) = cos(w m) / 2 exactly."""
    P, T = 8, 64
    t = np.arange(T)
    j = np.zeros((T, 3))
    j[:, 0] = np.cos(2 * math.pi * t / P)
    j[:, 1] = 2.0 * np.sin(2 * math.pi * t / P)
    c = O.hcacf(j, T)
    for m in range(T):
        if (T - m) % 4 == 0:
            assert abs(c[m, 0] - 0.5 * math.cos(2 * math.pi * m / P)) < 1e-14
            assert abs(c[m, 1] - 2.0 * math.cos(2 * math.pi * m / P)) < 1e-13
    assert np.all(c[:, 2] == 0.0)


def test_matches_wiener_khinchin_fft():
    rng = np.random.default_rng(5)
    T = 301
    j = rng.normal(size=(T, 3)).cumsum(axis=0) * 0.1 + rng.normal(size=(T, 3))
    c = O.hcacf(j, T)
    n = 1 << (2 * T - 1).bit_length()
    f = np.fft.rfft(j, n=n, axis=0)
    raw = np.fft.irfft(f * np.conj(f), n=n, axis=0)[:T]
    ref = raw / (T - np.arange(T))[:, None]
    assert np.abs(c - ref).max() / np.abs(ref).max() < 1e-12


def test_lag_direction_and_origin_count():
    """An impulse at t0 and another at t1 > t0 correlate only at lag t1 - t0, with one
    origin out of T - (t1 - t0)."""
    T = 40
    j = np.zeros((T, 3))
    j[5, 2] = 2.0
    j[17, 2] = 3.0
    c = O.hcacf(j, T)
    expect = np.zeros(T)
    expect[0] = (4.0 + 9.0) / T
    expect[12] = 6.0 / (T - 12)
    assert np.allclose(c[:, 2], expect, rtol=1e-15, atol=0)


def test_trapezoid_exact_on_linear_hcacf():
    m = np.arange(30, dtype=float)
    c = np.stack([2.0 - 0.1 * m, 0.5 + 0.0 * m, -1.0 + 0.3 * m], axis=1)
    dt, V, T = 0.25, 500.0, 200.0
    k = O.running_kappa(c, dt, V, T)
    pref = GK.EV_PER_FS_A_K_TO_W_PER_M_K / (GK.K_B * T * T * V)
    a = np.array([2.0, 0.5, -1.0])
    b = np.array([-0.1, 0.0, 0.3])
    exact = pref * (a * (m * dt)[:, None] + b * (m * m * dt / 2.0)[:, None])
    assert np.allclose(k, exact, rtol=1e-12, atol=1e-12 * np.abs(exact).max())


def test_exponential_decay_integral():
    """C(t) = C0 exp(-t / tau): kappa(inf) = C0 tau / (k_B T^2 V), trapezoid error
    C0 dt^2 / (12 tau) to leading order."""
    dt, tau, C0 = 0.5, 40.0, 3.0
    m = np.arange(4000)
    c = np.repeat((C0 * np.exp(-m * dt / tau))[:, None], 3, axis=1)
    k = O.running_kappa(c, dt, 1.0, 1.0)
    pref = GK.EV_PER_FS_A_K_TO_W_PER_M_K / GK.K_B
    assert abs(k[-1, 0] / pref - C0 * tau) < 1.1 * C0 * dt * dt / (12 * tau)


def test_units_through_si():
    """kappa from the same C computed in SI units: J [eV A/fs] -> J m/s, V -> m^3,
    k_B = 1.380649e-23 J/K."""
    c = np.array([[1.7, 0.2, 0.9], [1.1, 0.1, 0.4]])
    dt, V, T = 0.5, 1234.5, 310.0
    k = O.running_kappa(c, dt, V, T)
    e, kb_si = 1.602176634e-19, 1.380649e-23
    j_unit = e * 1e-10 / 1e-15                       # eV A / fs in J m / s
    c_si = c * j_unit ** 2
    integral = 0.5 * (c_si[0] + c_si[1]) * dt * 1e-15
    ref = integral / (kb_si * T * T * V * 1e-30)
    assert np.allclose(k[1], ref, rtol=1e-9)        # k_B in eV/K is quoted to 10 digits


def test_rejects_bad_lag_count():
    with pytest.raises(ValueError):
        O.hcacf(np.zeros((5, 3)), 6)
    with pytest.raises(ValueError):
        O.hcacf(np.zeros((5, 3)), 0)
