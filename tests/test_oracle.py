"""Pins for the CPU oracle, against facts fixed outside the oracle itself:
published fitted properties of the parameter sets, finite differences of the energy,
the paper's own identities (Eqs. 12-16, 17-21, 23-27), symmetry invariants, brute
force on tiny inputs, and integrator properties.  A plausible slip anywhere in oracle.c
(a dropped term, a sign, a transposed index) fails at least one of these."""
import json
import math
import os

import numpy as np
import pytest

from paper_1610_03343_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "published_properties.json")))


def energy(O, kind, params, pos, box, pbc):
    rc = O.cutoff(kind, params)
    NN, NL = O.neighbors(pos, box, pbc, rc, 32, "brute")
    if kind == O.TERSOFF:
        U, F, _, _ = O.tersoff_conventional(pos, box, pbc, params, NN, NL)
    else:
        U, F, _ = O.sw_conventional(pos, box, pbc, params, NN, NL)
    return U, F


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def small_systems():
    """Small jittered cells of every workload family + non-periodic clusters."""
    si = I.si_diamond_tersoff(n=3, jitter_amp=0.1, seed_pos=11, seed_vel=12)
    sw = I.si_diamond_sw(n=3, jitter_amp=0.1, seed_pos=13, seed_vel=14)
    gr = I.c_graphene_tersoff(nx=3, ny=5, jitter_amp=0.05, seed_pos=15, seed_vel=16)
    cd = I.c_diamond_tersoff(n=3, jitter_amp=0.05, seed_pos=17, seed_vel=18)
    si_cl = I.cluster(I.si_diamond_tersoff(n=3, jitter_amp=0.1, seed_pos=19, seed_vel=20), 6.0)
    sw_cl = I.cluster(I.si_diamond_sw(n=3, jitter_amp=0.1, seed_pos=21, seed_vel=22), 6.0)
    # periodic cells barely wider than twice the cutoff: the minimum image is exercised
    # on pairs whose raw separation is just over half a box
    tight_t = I.random_cell(14, [6.15, 6.2, 6.3], 2.0, I.MD_TERSOFF, I.TERSOFF_SI_1989, I.MASS_SI, 31)
    tight_s = I.random_cell(18, [7.7, 7.8, 7.9], 2.0, I.MD_SW, I.SW_SI_1985, I.MASS_SI, 33)
    return [si, sw, gr, cd, si_cl, sw_cl, tight_t, tight_s]


SYSTEMS = small_systems()
IDS = [s.name for s in SYSTEMS]


# ------------------------------------------------------------- published pins
@pytest.mark.parametrize("key,params", [("tersoff_si_1989", I.TERSOFF_SI_1989),
                                        ("tersoff_c_1989", I.TERSOFF_C_1989)])
def test_tersoff_diamond_cohesive_energy_and_lattice(oracle, key, params):
    g = GOLD[key]
    a0 = g["lattice_constant_A"]

    def e(a):
        pos, box = I.diamond_positions(2, a)
        U, F = energy(oracle, oracle.TERSOFF, params, pos, box, [1, 1, 1])
        return U.sum() / len(U), F

    e0, F0 = e(a0)
    assert abs(-e0 - g["cohesive_energy_eV_per_atom"]) < g["energy_tol_eV"]
    # perfect lattice: every force vanishes by symmetry
    assert np.abs(F0).max() < 1e-10
    # a0 is the minimum of E(a) to within the tolerance of the published constant
    grid = np.linspace(a0 - 0.02, a0 + 0.02, 41)
    es = [e(a)[0] for a in grid]
    amin = grid[int(np.argmin(es))]
    assert abs(amin - a0) <= g["lattice_tol_A"]


def test_sw_pair_minimum_dimer(oracle):
    """SW 1985 construction: two atoms at 2^(1/6) sigma have energy -epsilon, and that
    distance is the minimum (zero force)."""
    g = GOLD["sw_si_1985"]
    eps, sig = I.SW_SI_1985[0], I.SW_SI_1985[1]
    r0 = g["pair_minimum_r_over_sigma"] * sig
    box = np.array([30.0, 30.0, 30.0])

    def dimer(r):
        pos = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        return energy(oracle, oracle.SW, I.SW_SI_1985, pos, box, [0, 0, 0])

    U, F = dimer(r0)
    assert abs(U.sum() / eps - g["pair_minimum_depth_over_epsilon"]) < g["rel_tol"]
    assert np.abs(F).max() < 1e-6
    assert dimer(r0 * 0.99)[0].sum() > U.sum() and dimer(r0 * 1.01)[0].sum() > U.sum()


def test_sw_diamond_energy_is_minus_two_epsilon(oracle):
    g = GOLD["sw_si_1985"]
    eps, sig = I.SW_SI_1985[0], I.SW_SI_1985[1]
    a = 4.0 * g["pair_minimum_r_over_sigma"] * sig / math.sqrt(3.0)
    pos, box = I.diamond_positions(2, a)
    U, F = energy(oracle, oracle.SW, I.SW_SI_1985, pos, box, [1, 1, 1])
    assert abs(U.sum() / len(U) / eps - g["diamond_energy_over_epsilon"]) < g["rel_tol"]
    assert np.abs(F).max() < 1e-6


def test_tersoff_c_graphene_bond_length_minimum(oracle):
    """The 1989 carbon set is known to put the graphene/graphite bond length near
    1.46 Angstrom (longer than the experimental 1.42)."""
    def e(acc):
        pos, box = I.graphene_positions(3, 2, acc, 20.0)
        U, _ = energy(oracle, oracle.TERSOFF, I.TERSOFF_C_1989, pos, box, [1, 1, 1])
        return U.sum() / len(U)
    grid = np.linspace(1.40, 1.52, 121)
    amin = grid[int(np.argmin([e(a) for a in grid]))]
    assert 1.455 <= amin <= 1.467


# ------------------------------------------------------------ special cases
def test_tersoff_dimer_reduces_to_pair_form(oracle):
    """With a single neighbour zeta = 0 and b = 1: each atom's energy is 1/2 of
    f_C (A e^{-lambda r} - B e^{-mu r}), including inside the cutoff switch."""
    A, B, lam, mu = I.TERSOFF_SI_1989[:4]
    R, S = I.TERSOFF_SI_1989[9:11]
    box = np.array([30.0, 30.0, 30.0])
    for r in (2.3, 2.5, 2.85, 2.99, 3.01):
        pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0 + r, 10.0]])
        U, F = energy(oracle, oracle.TERSOFF, I.TERSOFF_SI_1989, pos, box, [0, 0, 0])
        fc = 1.0 if r < R else (0.0 if r >= S else 0.5 + 0.5 * math.cos(math.pi * (r - R) / (S - R)))
        want = fc * (A * math.exp(-lam * r) - B * math.exp(-mu * r))
        assert abs(U.sum() - want) <= 1e-12 * max(abs(want), 1.0)
        assert np.all(np.isfinite(F))


# ------------------------------------------------------------ finite differences
@pytest.mark.parametrize("sysm", SYSTEMS, ids=IDS)
def test_forces_match_energy_finite_difference(oracle, sysm):
    rng = np.random.default_rng(5)
    U, F = energy(oracle, sysm.kind, sysm.params, sysm.pos, sysm.box, sysm.pbc)
    h = 1e-5
    fmax = np.abs(F).max()
    for _ in range(12):
        i = int(rng.integers(sysm.n)); a = int(rng.integers(3))
        p1 = sysm.pos.copy(); p1[i, a] += h
        p2 = sysm.pos.copy(); p2[i, a] -= h
        e1 = energy(oracle, sysm.kind, sysm.params, p1, sysm.box, sysm.pbc)[0].sum()
        e2 = energy(oracle, sysm.kind, sysm.params, p2, sysm.box, sysm.pbc)[0].sum()
        fd = -(e1 - e2) / (2 * h)
        assert abs(fd - F[i, a]) < 2e-7 * max(fmax, 1.0), (i, a, fd, F[i, a])


@pytest.mark.parametrize("sysm", SYSTEMS, ids=IDS)
def test_dUi_drij_matches_per_atom_energy_finite_difference(oracle, sysm):
    """dU_i/dr_ij (the building block of Eqs. 14, 28-30) against a central difference of
    the single-atom energy U_i when only atom j moves (each pair occurs once in the
    minimum image, so moving r_j moves r_ij alone)."""
    rc = oracle.cutoff(sysm.kind, sysm.params)
    NN, NL = oracle.neighbors(sysm.pos, sysm.box, sysm.pbc, rc, 32, "brute")
    Ud, D = oracle.dUdr(sysm.kind, sysm.pos, sysm.box, sysm.pbc, sysm.params, NN, NL)
    rng = np.random.default_rng(7)
    h = 1e-5
    dmax = np.abs(D).max()
    checked = 0
    while checked < 10:
        i = int(rng.integers(sysm.n))
        if NN[i] == 0:
            continue
        m = int(rng.integers(NN[i])); j = int(NL[m, i]); a = int(rng.integers(3))
        p1 = sysm.pos.copy(); p1[j, a] += h
        p2 = sysm.pos.copy(); p2[j, a] -= h
        u1 = energy(oracle, sysm.kind, sysm.params, p1, sysm.box, sysm.pbc)[0][i]
        u2 = energy(oracle, sysm.kind, sysm.params, p2, sysm.box, sysm.pbc)[0][i]
        fd = (u1 - u2) / (2 * h)
        assert abs(fd - D[a, m, i]) < 2e-7 * max(dmax, 1.0), (i, j, a, fd, D[a, m, i])
        checked += 1


# ------------------------------------------------------------ the paper's identities
@pytest.mark.parametrize("sysm", SYSTEMS, ids=IDS)
def test_conventional_equals_pairwise_forces(oracle, sysm):
    """Eqs. 12-16: Algorithm 1's forces equal sum_j (dU_i/dr_ij - dU_j/dr_ji)."""
    r = oracle.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, sysm.params, sysm.vel)
    assert rel(r["F_pair"], r["F"]) < 1e-13
    assert rel(r["U_d"], r["U"]) < 1e-14


@pytest.mark.parametrize("sysm", SYSTEMS, ids=IDS)
def test_newton_third_law_and_virial_totals(oracle, sysm):
    r = oracle.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, sysm.params, sysm.vel)
    F = r["F"]
    scale = np.abs(F).max() * math.sqrt(sysm.n)
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * max(scale, 1.0)
    Wsum = r["W"].sum(axis=0)                     # Eq. 29 summed (Eq. 19)
    assert rel(Wsum, r["W_total_conv"]) < 1e-12   # Algorithm 1's total virial
    if r["W_lammps"] is not None:                 # Eq. 22 summed: same total
        assert rel(r["W_lammps"].sum(axis=0), Wsum) < 1e-12
    if not np.any(sysm.pbc):
        # cluster: W = sum_i r_i (x) F_i (Eq. 17), symmetric, zero torque
        Wabs = np.einsum("ia,ib->ab", sysm.pos, F).ravel()
        assert rel(Wsum, Wabs) < 1e-11
        W9 = Wsum.reshape(3, 3)
        assert np.abs(W9 - W9.T).max() < 1e-11 * np.abs(W9).max()
        torque = np.cross(sysm.pos, F).sum(axis=0)
        assert np.abs(torque).max() < 1e-11 * max(scale * np.abs(sysm.pos).max(), 1.0)


@pytest.mark.parametrize("sysm", SYSTEMS, ids=IDS)
def test_virial_matches_strain_derivative(oracle, sysm):
    """W_ab = -dU/d eps_ba under the homogeneous strain r -> (1 + eps) r (Eqs. 17-21).
    Periodic cells: diagonal strains (box scaled too); clusters: all nine."""
    r = oracle.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, sysm.params, sysm.vel)
    W = r["W"].sum(axis=0).reshape(3, 3)
    h = 1e-6
    comps = [(a, a) for a in range(3)] if np.any(sysm.pbc) else [(a, b) for a in range(3) for b in range(3)]
    wmax = max(np.abs(W).max(), 1.0)
    for (a, b) in comps:
        def u(e):
            eps = np.zeros((3, 3)); eps[b, a] = e
            M = np.eye(3) + eps
            pos = sysm.pos @ M.T
            box = sysm.box * np.diag(M) if np.any(sysm.pbc) else sysm.box
            return energy(oracle, sysm.kind, sysm.params, pos, box, sysm.pbc)[0].sum()
        fd = -(u(h) - u(-h)) / (2 * h)
        assert abs(fd - W[a, b]) < 1e-6 * wmax, (a, b, fd, W[a, b])


def test_perfect_diamond_has_zero_virial(oracle):
    pos, box = I.diamond_positions(2, 5.432)
    # zero only at the exact minimum; 5.432 is within 0.001 of it, so |W| is small
    r = oracle.compute(pos, box, [1, 1, 1], oracle.TERSOFF, I.TERSOFF_SI_1989)
    W = r["W"].sum(axis=0).reshape(3, 3)
    assert np.abs(W - np.diag(np.diag(W))).max() < 1e-10     # cubic: no shear
    assert abs(W[0, 0] - W[1, 1]) < 1e-10 and abs(W[0, 0] - W[2, 2]) < 1e-10
    assert abs(W[0, 0]) / len(pos) < 2e-3


@pytest.mark.parametrize("sysm", [s for s in SYSTEMS if not np.any(s.pbc)],
                         ids=[s.name for s in SYSTEMS if not np.any(s.pbc)])
def test_heat_current_matches_energy_flux_definition(oracle, sysm):
    """Eq. 25 rewritten for a non-periodic cluster: J_pot = sum_i r_i (F_i . v_i + dU_i/dt),
    with dU_i/dt taken by central difference of U_i along the velocities."""
    r = oracle.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, sysm.params, sysm.vel)
    J = r["J"].sum(axis=0)
    v = sysm.vel
    e = 1e-4
    Up = energy(oracle, sysm.kind, sysm.params, sysm.pos + e * v, sysm.box, sysm.pbc)[0]
    Um = energy(oracle, sysm.kind, sysm.params, sysm.pos - e * v, sysm.box, sysm.pbc)[0]
    dUdt = (Up - Um) / (2 * e)
    Jref = (sysm.pos * ((r["F"] * v).sum(axis=1) + dUdt)[:, None]).sum(axis=0)
    assert rel(J, Jref) < 1e-6, (J, Jref)


def _pair_limit(sysm):
    p = list(sysm.params)
    if sysm.kind == I.MD_TERSOFF:
        p[4] = 0.0      # beta = 0  ->  b_ij = 1: a pair potential
    else:
        p[3] = 0.0      # lambda = 0: no three-body term
    return tuple(p)


@pytest.mark.parametrize("sysm", SYSTEMS[:4], ids=IDS[:4])
def test_stress_based_heat_current_only_valid_for_pair_potentials(oracle, sysm):
    """Eqs. 23-24 vs Eqs. 25-27: J_i = W_i . v_i holds per atom for a pair potential
    and fails for the many-body one (Sec. 2.3)."""
    for params, should_match in ((_pair_limit(sysm), True), (sysm.params, False)):
        r = oracle.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, params, sysm.vel)
        W = r["W"].reshape(-1, 3, 3)
        Jstress = np.einsum("iab,ib->ia", W, sysm.vel)
        err = rel(Jstress, r["J"])
        if should_match:
            assert err < 1e-12
        else:
            assert err > 1e-3


@pytest.mark.parametrize("sysm", [s for s in SYSTEMS if s.kind == I.MD_TERSOFF],
                         ids=[s.name for s in SYSTEMS if s.kind == I.MD_TERSOFF])
def test_lammps_per_atom_virial_differs_unless_pairwise(oracle, sysm):
    """Eq. 22 equals Eq. 21 per atom only when b_ij = b_ji trivially (pair limit)."""
    for params, should_match in ((_pair_limit(sysm), True), (sysm.params, False)):
        r = oracle.compute(sysm.pos, sysm.box, sysm.pbc, sysm.kind, params, sysm.vel)
        err = rel(r["W_lammps"], r["W"])
        if should_match:
            assert err < 1e-12
        else:
            assert err > 1e-3


# ------------------------------------------------------------ invariances
@pytest.mark.parametrize("sysm", [s for s in SYSTEMS if not np.any(s.pbc)],
                         ids=[s.name for s in SYSTEMS if not np.any(s.pbc)])
def test_rotation_and_translation_invariance(oracle, sysm):
    U0, F0 = energy(oracle, sysm.kind, sysm.params, sysm.pos, sysm.box, sysm.pbc)
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    c = sysm.pos.mean(axis=0)
    pos = (sysm.pos - c) @ q.T + c + np.array([0.3, -0.2, 0.1])
    U1, F1 = energy(oracle, sysm.kind, sysm.params, pos, sysm.box + 2.0, sysm.pbc)
    assert rel(U1, U0) < 1e-12
    assert rel(F1, F0 @ q.T) < 1e-11


def test_periodic_translation_invariance(oracle):
    s = SYSTEMS[0]
    U0, F0 = energy(oracle, s.kind, s.params, s.pos, s.box, s.pbc)
    pos = I.wrap(s.pos + np.array([1.7, -3.1, 0.4]), s.box, s.pbc)
    U1, F1 = energy(oracle, s.kind, s.params, pos, s.box, s.pbc)
    assert rel(U1, U0) < 1e-12 and rel(F1, F0) < 1e-11


# ------------------------------------------------------------ neighbour lists
@pytest.mark.parametrize("n,rc,pbc", [(2, 3.0, [1, 1, 1]), (3, 3.5, [1, 1, 1]), (4, 4.27, [1, 1, 1]),
                                      (3, 3.0, [1, 0, 1]), (3, 2.6, [0, 0, 0]),
                                      (2, 4.27, [1, 1, 1]), (1, 2.6, [1, 1, 1]), (2, 5.0, [1, 0, 1])])
def test_cell_list_equals_brute_force(oracle, n, rc, pbc):
    s = I.si_diamond_tersoff(n=n, jitter_amp=0.15, seed_pos=n)
    pos = s.pos.copy()
    box = s.box.copy()
    for a in range(3):
        if not pbc[a]:
            box[a] += 6.0
            pos[:, a] += 3.0
    NNb, NLb = oracle.neighbors(pos, box, pbc, rc, 48, "brute")
    NNc, NLc = oracle.neighbors(pos, box, pbc, rc, 48, "cells")
    assert np.array_equal(NNb, NNc)
    assert np.array_equal(NLb, NLc)
    # symmetric: j in NL_i <=> i in NL_j
    for i in range(len(NNb)):
        for m in range(NNb[i]):
            j = NLb[m, i]
            assert i in NLb[:NNb[j], j]


def test_graphene_has_three_neighbours_diamond_four(oracle):
    s = I.c_graphene_tersoff(nx=4, ny=6, jitter_amp=0.0)
    NN, _ = oracle.neighbors(s.pos, s.box, s.pbc, 2.1, 8)
    assert NN.min() == 3 and NN.max() == 3
    s = I.si_diamond_tersoff(n=3, jitter_amp=0.0)
    NN, _ = oracle.neighbors(s.pos, s.box, s.pbc, 3.0, 8)
    assert NN.min() == 4 and NN.max() == 4


# ------------------------------------------------------------ integrator
def _total_energy(series):
    return series[:, 0] + series[:, 1]


def test_nve_energy_conservation_and_dt_squared(oracle):
    s = I.si_diamond_tersoff(n=2, jitter_amp=0.05, temperature=300.0)
    _, _, s1 = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 400, 1.0)
    _, _, s2 = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 800, 0.5)
    e1 = _total_energy(s1); e2 = _total_energy(s2)
    assert np.abs(e1 - e1[0]).max() / s.n < 1e-4        # bounded drift, eV/atom
    # velocity Verlet: fluctuation of the conserved energy scales as dt^2
    ratio = np.std(e1) / np.std(e2)
    assert 3.0 < ratio < 5.5, ratio


def test_time_reversibility(oracle):
    s = I.si_diamond_sw(n=2, jitter_amp=0.05, temperature=300.0)
    p1, v1, _ = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 100, 1.0)
    p2, v2, _ = oracle.run(p1, -v1, s.mass, s.box, s.pbc, s.kind, s.params, 100, 1.0)
    d = p2 - s.pos
    d -= np.round(d / s.box) * s.box
    assert np.abs(d).max() < 1e-9
    assert np.abs(v2 + s.vel).max() < 1e-11


def test_run_series_matches_direct_evaluation(oracle):
    """The run's recorded U, K and J equal a fresh evaluation at the final state."""
    s = I.si_diamond_tersoff(n=2, jitter_amp=0.05)
    p, v, ser = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 5, 1.0)
    r = oracle.compute(p, s.box, s.pbc, s.kind, s.params, v)
    assert abs(ser[-1, 0] - r["U"].sum()) < 1e-10
    assert abs(ser[-1, 1] - oracle.kinetic_energy(v, s.mass)) < 1e-12
    assert rel(ser[-1, 2:], r["J"].sum(axis=0)) < 1e-12


@pytest.mark.parametrize("kind,params", [(I.MD_TERSOFF, I.TERSOFF_SI_1989), (I.MD_SW, I.SW_SI_1985)])
def test_per_atom_force_virial_heat_current_brute_force(oracle, kind, params):
    """Tiny cluster: every dU_i/dr_ij by central differences of U_i (moving atom j only),
    then Eqs. 28-30 assembled by hand; the oracle's per-atom F_i, W_i (as r_ij (x) F_ij,
    component (a,b) = r_a F_b) and J_i must agree."""
    rng = np.random.default_rng(9)
    base = np.array([[0, 0, 0], [2.3, 0.2, 0.1], [-0.6, 2.2, -0.3], [0.4, -0.5, 2.25],
                     [-2.2, -0.7, -0.4]], dtype=np.float64) + 10.0
    pos = base + rng.uniform(-0.05, 0.05, size=base.shape)
    vel = rng.normal(0, 0.01, size=base.shape)
    box = np.array([30.0, 30.0, 30.0]); pbc = [0, 0, 0]
    n = len(pos)
    h = 1e-5
    d = np.zeros((n, n, 3))                      # d[i, j] = dU_i / dr_ij
    for j in range(n):
        for a in range(3):
            p1 = pos.copy(); p1[j, a] += h
            p2 = pos.copy(); p2[j, a] -= h
            dU = (energy(oracle, kind, params, p1, box, pbc)[0] -
                  energy(oracle, kind, params, p2, box, pbc)[0]) / (2 * h)
            for i in range(n):
                if i != j:
                    d[i, j, a] = dU[i]
    F = np.zeros((n, 3)); W = np.zeros((n, 3, 3)); J = np.zeros((n, 3))
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            rij = pos[j] - pos[i]
            Fij = d[i, j] - d[j, i]
            F[i] += Fij
            W[i] += -0.5 * np.outer(rij, Fij)
            J[i] += rij * np.dot(d[j, i], vel[i])
    r = oracle.compute(pos, box, pbc, kind, params, vel)
    assert rel(r["F"], F) < 1e-7
    assert rel(r["W"].reshape(n, 3, 3), W) < 1e-7
    assert rel(r["J"], J) < 1e-7
    # the per-atom virial is genuinely non-symmetric here, so orientation is pinned
    Wo = r["W"].reshape(n, 3, 3)
    assert np.abs(Wo - Wo.transpose(0, 2, 1)).max() > 1e-4 * np.abs(Wo).max()


def test_damped_step_scales_velocities_after_the_second_half_kick(oracle):
    """Damped relaxation (reading: v <- v (1 - gamma dt) after the second half-kick):
    one damped step leaves positions unchanged and scales the undamped velocities."""
    s = I.si_diamond_tersoff(n=2, jitter_amp=0.05)
    p0, v0, _ = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 1, 1.0)
    p1, v1, _ = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 1, 1.0, damp=0.01)
    assert np.array_equal(p0, p1)
    assert np.array_equal(v1, v0 * (1.0 - 0.01 * 1.0))
    _, _, ser = oracle.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 200, 1.0, damp=0.01)
    e = ser[:, 0] + ser[:, 1]
    assert e[-1] < e[0] - 0.5 * ser[0, 1]      # most of the kinetic energy is removed
