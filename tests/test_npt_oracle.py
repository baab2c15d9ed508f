"""Pins of the oracle's Berendsen thermostat and barostat (oracle_run_ex) against results
fixed elsewhere: the exact geometric relaxation of a free gas's temperature, the closed
form of the box scaling of a free gas, the pressure recovered from a box change against
-dE/dV by finite differences of the energy, and relaxation of a compressed silicon
crystal to the lattice constant the Tersoff parameters were fitted to."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "published_properties.json")))
KB = 8.617333262e-5
GPA = 160.2176634
ACC = 9.648533215665328e-3


def free_gas(n=60, L=60.0, seed=3, T=500.0):
    """Atoms on a coarse grid far beyond the Tersoff cutoff: no interactions at all."""
    g = int(np.ceil(n ** (1 / 3)))
    idx = np.array([(i, j, k) for i in range(g) for j in range(g) for k in range(g)][:n], dtype=float)
    pos = (idx + 0.5) * (L / g)
    vel = I.maxwell_boltzmann(n, I.MASS_SI, T, seed)
    return pos, vel, np.array([L, L, L]), np.array([1, 1, 1], np.int32)


def temperature(K, n):
    return 2.0 * K / (KB * (3 * n - 3))


def test_couplings_off_is_nve_bitwise():
    s = I.si_diamond_tersoff(n=2, jitter_amp=0.05)
    p0, v0, s0 = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 6, 1.0)
    p1, v1, s1, b = O.run_npt(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 6, 1.0, tau_T=0.0, tau_P=0.0)
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1) and np.array_equal(s0, s1)
    assert np.array_equal(b, s.box)


def test_free_gas_temperature_relaxes_geometrically():
    """No forces: K changes only by lambda^2, so T_{s+1} - T0 = (1 - dt/tau)(T_s - T0)."""
    pos, vel, box, pbc = free_gas()
    dt, tau, T0 = 1.0, 20.0, 300.0
    _, _, ser, _ = O.run_npt(pos, vel, I.MASS_SI, box, pbc, I.MD_TERSOFF, I.TERSOFF_SI_1989, 40, dt,
                             T0=T0, tau_T=tau, tau_P=0.0)
    T = temperature(ser[:, 1], pos.shape[0])
    expect = T0 + (T[0] - T0) * (1.0 - dt / tau) ** np.arange(40)
    assert np.abs(T - expect).max() < 1e-10 * T0
    assert np.all(ser[:, 0] == 0.0)


def test_free_gas_box_scaling_closed_form():
    """No forces: P_aa = 2 K_aa / V, and one step later each edge is scaled by
    mu_a = (1 - beta dt / tau_P (P0 - P_aa))^(1/3)."""
    pos, vel, box, pbc = free_gas(T=2000.0)
    dt, tauP, beta, P0 = 1.0, 50.0, 0.5, 0.0
    p2, _, _, b = O.run_npt(pos, vel, I.MASS_SI, box, pbc, I.MD_TERSOFF, I.TERSOFF_SI_1989, 2, dt,
                            tau_T=0.0, tau_P=tauP, beta=beta, P0=P0)
    Kaa = 0.5 * I.MASS_SI * (vel ** 2).sum(axis=0) / ACC      # free flight keeps v
    P = 2.0 * Kaa / np.prod(box) * GPA
    mu = np.cbrt(1.0 - beta * dt / tauP * (P0 - P))
    assert np.allclose(b, box * mu, rtol=1e-14, atol=0)
    assert np.all(mu > 1.0)                                   # a gas at P > P0 expands
    # coordinates scale with the box: x2 = mu (x0 + v dt) + v dt, wrapped into the new box
    x2 = mu * np.mod(pos + vel * dt, box) + vel * dt
    d = p2 - x2
    d -= np.round(d / b) * b
    assert np.abs(d).max() < 1e-12


def test_crystal_pressure_matches_energy_derivative():
    """Perfect compressed diamond at T = 0 (forces vanish by symmetry): the barostat's
    pressure, read back from the box change of one step, equals -dE/dV by central
    differences of the oracle's total energy under uniform strain."""
    a, n = 5.40, 2
    pos, box = I.diamond_positions(n, a)
    pbc = np.array([1, 1, 1], np.int32)
    zero = np.zeros_like(pos)
    dt, tauP, beta = 1.0, 100.0, 0.01
    _, _, _, b = O.run_npt(pos, zero, I.MASS_SI, box, pbc, I.MD_TERSOFF, I.TERSOFF_SI_1989, 2, dt,
                           tau_T=0.0, tau_P=tauP, beta=beta, P0=0.0)
    mu = b[0] / box[0]
    P_baro = (mu ** 3 - 1.0) * tauP / (beta * dt)             # from mu^3 = 1 - beta dt/tau (0 - P)

    def energy(scale):
        p2, b2 = I.diamond_positions(n, a * scale)
        return O.compute(p2, b2, pbc, I.MD_TERSOFF, I.TERSOFF_SI_1989)["totals"][0]
    h = 1e-5
    dE = energy(1 + h) - energy(1 - h)
    V = np.prod(box)
    dV = V * ((1 + h) ** 3 - (1 - h) ** 3)
    P_fd = -dE / dV * GPA
    assert P_fd > 1.0                                          # compressed: positive pressure
    assert abs(P_baro - P_fd) < 1e-6 * abs(P_fd)


def test_compressed_crystal_relaxes_to_fitted_lattice_constant():
    g = GOLDEN["tersoff_si_1989"]
    n = 2
    pos, box = I.diamond_positions(n, 5.38)
    pbc = np.array([1, 1, 1], np.int32)
    _, _, _, b = O.run_npt(pos, np.zeros_like(pos), I.MASS_SI, box, pbc, I.MD_TERSOFF, I.TERSOFF_SI_1989, 150, 1.0,
                           tau_T=0.0, tau_P=50.0, beta=0.04, P0=0.0)
    a = b / n
    assert np.all(np.abs(a - g["lattice_constant_A"]) < g["lattice_tol_A"]), a


def test_thermostat_and_barostat_together_stay_finite_and_near_targets():
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.05, temperature=600.0)
    _, _, ser, b = O.run_npt(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 300, 1.0,
                             T0=300.0, tau_T=20.0, tau_P=200.0, beta=0.01)
    T = temperature(ser[:, 1], s.n)
    assert np.all(np.isfinite(ser)) and np.all(np.isfinite(b))
    assert abs(T[-50:].mean() - 300.0) < 60.0
    assert np.all(np.abs(b / s.box - 1.0) < 0.02)
