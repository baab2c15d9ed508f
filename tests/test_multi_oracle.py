"""Pins for the oracle's multi-element Tersoff (Tersoff 1989 multicomponent form: mixed
radial parameters, element-i angular and bond-order parameters, chi per element pair),
against facts fixed outside it: the zincblende SiC lattice constant and cohesive energy
reported for the model, exact reduction to the pinned single-element oracle, finite
differences of the energy, the paper's identities (Eqs. 12-16 force equivalence, Eq. 29
virial = strain derivative), Newton's third law, invariance under relabelling the
elements, and a three-atom closed form written out below from the published form."""
import json
import math
import os

import numpy as np
import pytest

from paper_1610_03343_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "published_properties.json")))


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def lists(O, s, rc=None):
    return O.neighbors(s.pos, s.box, s.pbc, rc or O.multi_cutoff(s.params), 32, "brute")


def energy(O, pos, box, pbc, types, params, chi):
    rc = O.multi_cutoff(params)
    NN, NL = O.neighbors(pos, box, pbc, rc, 32, "brute")
    U, F, W = O.tersoff_multi_conventional(pos, box, pbc, types, params, chi, NN, NL)
    return U, F, W


def alloy(seed=0):
    return I.sic_substituted_diamond(n=2, a=5.2, c_fraction=0.35, jitter_amp=0.08, seed_types=5 + seed,
                                     seed_pos=6 + seed, seed_vel=7 + seed)


# ------------------------------------------------------------- published pins
def test_sic_zincblende_lattice_constant_and_cohesive_energy(oracle):
    g = GOLD["tersoff_sic_1989"]
    pbc = np.array([1, 1, 1], np.int32)
    types = np.tile(np.array([0, 0, 0, 0, 1, 1, 1, 1], np.int32), 8)

    def e(a):
        pos, box = I.diamond_positions(2, a)
        U, _, _ = energy(oracle, pos, box, pbc, types, I.TERSOFF_SIC_1989, I.CHI_SIC_1989)
        return U.sum() / len(pos)
    grid = np.arange(4.25, 4.40, 0.001)
    es = np.array([e(a) for a in grid])
    k = int(np.argmin(es))
    assert 0 < k < len(grid) - 1
    assert abs(grid[k] - g["lattice_constant_A"]) < g["lattice_tol_A"]
    assert abs(-es[k] - g["cohesive_energy_eV_per_atom"]) < g["energy_tol_eV"]


def test_sic_perfect_crystal_has_no_forces(oracle):
    pos, box = I.diamond_positions(2, 4.32)
    types = np.tile(np.array([0, 0, 0, 0, 1, 1, 1, 1], np.int32), 8)
    _, F, _ = energy(oracle, pos, box, np.array([1, 1, 1], np.int32), types, I.TERSOFF_SIC_1989, I.CHI_SIC_1989)
    assert np.abs(F).max() < 1e-10


# ---------------------------------------------------- reduction to one element
def test_two_labels_of_one_element_reduce_to_the_single_element_oracle(oracle):
    """Both 'elements' Si with chi = 1: every mixed parameter equals the element's own, so
    the multi-element routines must reproduce the pinned single-element ones."""
    s = I.si_diamond_tersoff(n=2, jitter_amp=0.1, seed_pos=3)
    rng = np.random.Generator(np.random.PCG64(9))
    types = rng.integers(0, 2, size=s.n).astype(np.int32)
    params = (I.TERSOFF_SI_1989, I.TERSOFF_SI_1989)
    chi = ((1.0, 1.0), (1.0, 1.0))
    NN, NL = oracle.neighbors(s.pos, s.box, s.pbc, 3.0, 32, "brute")
    U1, F1, _, W1 = oracle.tersoff_conventional(s.pos, s.box, s.pbc, s.params, NN, NL)
    U2, F2, W2 = oracle.tersoff_multi_conventional(s.pos, s.box, s.pbc, types, params, chi, NN, NL)
    Ud1, D1 = oracle.dUdr(oracle.TERSOFF, s.pos, s.box, s.pbc, s.params, NN, NL)
    Ud2, D2 = oracle.tersoff_multi_dUdr(s.pos, s.box, s.pbc, types, params, chi, NN, NL)
    assert rel(U2, U1) < 1e-14 and rel(F2, F1) < 1e-14 and rel(W2, W1) < 1e-14
    assert rel(Ud2, Ud1) < 1e-14 and rel(D2, D1) < 1e-14


def test_relabelling_the_elements_changes_nothing(oracle):
    s = alloy()
    swap_params = (s.params[1], s.params[0])
    swap_chi = ((s.chi[1][1], s.chi[1][0]), (s.chi[0][1], s.chi[0][0]))
    a = oracle.compute_multi(s.pos, s.box, s.pbc, s.types, s.params, s.chi, s.vel)
    b = oracle.compute_multi(s.pos, s.box, s.pbc, 1 - s.types, swap_params, swap_chi, s.vel)
    for k in ("U", "F", "W", "J"):
        assert rel(b[k], a[k]) < 1e-14, k


# ------------------------------------------------------ finite differences
def test_forces_are_minus_the_energy_gradient(oracle):
    s = alloy()
    _, F, _ = energy(oracle, s.pos, s.box, s.pbc, s.types, s.params, s.chi)
    h = 1e-5
    rng = np.random.Generator(np.random.PCG64(4))
    for i in rng.choice(s.n, size=10, replace=False):
        for a in range(3):
            p1 = s.pos.copy(); p1[i, a] += h
            p2 = s.pos.copy(); p2[i, a] -= h
            e1 = energy(oracle, p1, s.box, s.pbc, s.types, s.params, s.chi)[0].sum()
            e2 = energy(oracle, p2, s.box, s.pbc, s.types, s.params, s.chi)[0].sum()
            fd = -(e1 - e2) / (2 * h)
            assert abs(F[i, a] - fd) < 2e-7 * max(1.0, abs(fd)), (i, a, F[i, a], fd)


def test_dUi_drij_matches_finite_differences_of_Ui(oracle):
    s = alloy(1)
    NN, NL = lists(oracle, s)
    U, D = oracle.tersoff_multi_dUdr(s.pos, s.box, s.pbc, s.types, s.params, s.chi, NN, NL)
    h = 1e-5
    for i in (0, 5, 17, 40):
        for m in range(NN[i]):
            j = NL[m, i]
            for a in range(3):
                p1 = s.pos.copy(); p1[j, a] += h
                p2 = s.pos.copy(); p2[j, a] -= h
                u1 = oracle.tersoff_multi_dUdr(p1, s.box, s.pbc, s.types, s.params, s.chi, NN, NL)[0][i]
                u2 = oracle.tersoff_multi_dUdr(p2, s.box, s.pbc, s.types, s.params, s.chi, NN, NL)[0][i]
                fd = (u1 - u2) / (2 * h)
                assert abs(D[a, m, i] - fd) < 2e-7 * max(1.0, abs(fd)), (i, m, a)


# ------------------------------------------------------------ paper identities
def test_algorithm1_forces_equal_the_pairwise_forces(oracle):
    """Eqs. 12-16: the conventional partial forces sum to the explicit pairwise form."""
    for seed in (0, 1, 2):
        s = alloy(seed)
        out = oracle.compute_multi(s.pos, s.box, s.pbc, s.types, s.params, s.chi, s.vel)
        assert rel(out["F_pair"], out["F"]) < 1e-12
        assert rel(out["U_d"], out["U"]) < 1e-14
        assert np.abs(out["F"].sum(axis=0)).max() < 1e-10 * np.abs(out["F"]).max()


def test_virial_is_the_strain_derivative(oracle):
    """sum_i W_i (Eq. 29) = Algorithm 1's total virial = -dU/d(epsilon) (homogeneous strain)."""
    s = alloy(2)
    out = oracle.compute_multi(s.pos, s.box, s.pbc, s.types, s.params, s.chi, s.vel)
    Wsum = out["W"].sum(axis=0)
    assert rel(Wsum, out["W_total_conv"]) < 1e-12
    h = 1e-6
    for a in range(3):
        for b in range(3):
            eps = np.zeros((3, 3)); eps[a, b] = h
            if a != b:
                continue   # orthorhombic box: only the normal strains keep it orthorhombic
            def e(sign):
                M = np.eye(3) + sign * eps
                return energy(oracle, s.pos @ M.T, s.box * np.diag(M), s.pbc, s.types, s.params, s.chi)[0].sum()
            dUde = (e(1) - e(-1)) / (2 * h)
            assert abs(Wsum[3 * a + b] + dUde) < 1e-6 * max(1.0, abs(dUde)), (a, b)


# ------------------------------------------------------------ closed form
def test_trimer_closed_form_with_mixed_cutoffs(oracle):
    """Si at the origin bonded to a C atom at 2.35 A (inside the Si-C switching shell
    sqrt(R_Si R_C) .. sqrt(S_Si S_C) = 2.205 .. 2.510 A) and to a Si atom at 2.30 A (inside
    the Si-Si core), 100 degrees apart; the C-Si' distance (3.58 A) is beyond every cutoff.
    The energy is written out here from the published form, term by term."""
    Si, C = I.TERSOFF_SI_1989, I.TERSOFF_C_1989
    chi = 0.9776
    th = math.radians(100.0)
    pos = np.array([[10.0, 10.0, 10.0],
                    [10.0 + 2.35, 10.0, 10.0],
                    [10.0 + 2.30 * math.cos(th), 10.0 + 2.30 * math.sin(th), 10.0]])
    types = np.array([0, 1, 0], np.int32)
    box = np.array([30.0, 30.0, 30.0]); pbc = np.array([0, 0, 0], np.int32)

    def mix(p, q):
        A, B, lam, mu, R, S = (math.sqrt(p[0] * q[0]), math.sqrt(p[1] * q[1]), (p[2] + q[2]) / 2,
                               (p[3] + q[3]) / 2, math.sqrt(p[9] * q[9]), math.sqrt(p[10] * q[10]))
        return A, B, lam, mu, R, S

    def fc(r, R, S):
        return 1.0 if r < R else (0.0 if r >= S else 0.5 + 0.5 * math.cos(math.pi * (r - R) / (S - R)))

    def g(e, cs):
        c, d, h = e[6], e[7], e[8]
        return 1.0 + c * c / (d * d) - c * c / (d * d + (h - cs) ** 2)

    def b(e, z, x):
        beta, n = e[4], e[5]
        return x * (1.0 + (beta * z) ** n) ** (-1.0 / (2.0 * n)) if z > 0 else x

    def Uij(pp, r, bij):
        A, B, lam, mu, R, S = pp
        return fc(r, R, S) * (A * math.exp(-lam * r) - bij * B * math.exp(-mu * r))

    sic, sisi = mix(Si, C), mix(Si, Si)
    cs = math.cos(th)
    # atom 0 (Si): bonds to C (1) and Si (2); each bond order sees the other bond
    z01 = fc(2.30, sisi[4], sisi[5]) * g(Si, cs)
    z02 = fc(2.35, sic[4], sic[5]) * g(Si, cs)
    u0 = 0.5 * (Uij(sic, 2.35, b(Si, z01, chi)) + Uij(sisi, 2.30, b(Si, z02, 1.0)))
    # atom 1 (C): one bond, to Si (0), zeta = 0; atom 2 (Si): one bond, to Si (0)
    u1 = 0.5 * Uij(sic, 2.35, chi)
    u2 = 0.5 * Uij(sisi, 2.30, 1.0)
    assert fc(2.35, sic[4], sic[5]) < 1.0                # the bond sits in the switching shell
    U, _, _ = energy(oracle, pos, box, pbc, types, I.TERSOFF_SIC_1989, I.CHI_SIC_1989)
    assert abs(U[0] - u0) < 1e-13 * abs(u0)
    assert abs(U[1] - u1) < 1e-13 * abs(u1)
    assert abs(U[2] - u2) < 1e-13 * abs(u2)


# ------------------------------------------------------------ integrator
def test_multi_element_nve_conserves_energy(oracle):
    s = I.sic_zincblende(n=2, jitter_amp=0.03, temperature=300.0)
    m = s.atom_masses
    _, _, ser = oracle.run_multi(s.pos, s.vel, m, s.box, s.pbc, s.types, s.params, s.chi, 200, 0.5)
    E = ser[:, 0] + ser[:, 1]
    assert np.abs(E - E[0]).max() / s.n < 2e-4
