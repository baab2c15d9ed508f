"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds *inputs only*: lattice geometries, random jitter, Maxwell-Boltzmann
velocities, and the published potential parameter sets as plain numbers.  It contains
none of the force method's arithmetic (no cutoff functions, no bond order, no forces),
so the oracle and the GPU path can both be fed from it without sharing any of the
computation they are compared on.

Workloads follow the paper's test system (Sec. 3: silicon crystal in a cubic periodic
domain with N = 8 n^3 atoms, 300 K) and the graphene-like carbon sheets the paper's
applications use.

Units: Angstrom, eV, amu, fs, K.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Unit conversion: 1 eV/(Angstrom*amu) expressed in Angstrom/fs^2, built from the exact
# elementary charge and the CODATA-2018 atomic mass constant.
#   eV/(A amu) = 1.602176634e-19 J / (1e-10 m * 1.66053906660e-27 kg)   [m/s^2]
#   m/s^2 -> A/fs^2: * 1e10 * 1e-30                         = 9.648533215665328e-3
EV_PER_A_AMU_TO_A_PER_FS2 = 9.648533215665328e-3
KB_EV_PER_K = 8.617333262e-5  # Boltzmann constant, eV/K

MASS_SI = 28.0855
MASS_C = 12.011

# ---------------------------------------------------------------------------
# Potential parameter sets (published values; the paper names the potentials,
# Sec. 2.1 and Ref. tersoff1989 / stillinger1985, but prints no parameters).
# Packed layouts match include/md.h.
# ---------------------------------------------------------------------------
MD_TERSOFF = 1
MD_SW = 2

# Tersoff, Phys. Rev. B 39, 5566 (1989), silicon:
#   A, B, lambda, mu, beta, n, c, d, h, R, S
TERSOFF_SI_1989 = (1830.8, 471.18, 2.4799, 1.7322, 1.1e-6, 0.78734,
                   1.0039e5, 16.217, -0.59825, 2.7, 3.0)
# Tersoff, Phys. Rev. B 39, 5566 (1989), carbon.
TERSOFF_C_1989 = (1393.6, 346.74, 3.4879, 2.2119, 1.5724e-7, 0.72751,
                  38049.0, 4.3484, -0.57058, 1.8, 2.1)
# Tersoff, Phys. Rev. B 39, 5566 (1989): the Si-C system, element 0 = Si, element 1 = C
# (per-element parameters as above) and the Si-C bond-order factor chi.
TERSOFF_SIC_1989 = (TERSOFF_SI_1989, TERSOFF_C_1989)
CHI_SIC_1989 = ((1.0, 0.9776), (0.9776, 1.0))
# Stillinger & Weber, Phys. Rev. B 31, 5262 (1985), silicon:
#   epsilon, sigma, a, lambda, gamma, A, B, p, q
SW_SI_1985 = (2.1683, 2.0951, 1.80, 21.0, 1.20, 7.049556277, 0.6022245584, 4.0, 0.0)


def cutoff(kind: int, params) -> float:
    """Interaction cutoff of a parameter set (Tersoff: S; SW: a*sigma)."""
    if kind == MD_TERSOFF:
        return float(params[10])
    if kind == MD_SW:
        return float(params[1] * params[2])
    raise ValueError(kind)


@dataclass
class System:
    """A synthetic MD system: SoA-friendly (N,3) arrays plus box and potential."""
    name: str
    pos: np.ndarray            # (N,3) float64, wrapped into [0, L) on periodic axes
    box: np.ndarray            # (3,) float64, orthorhombic edge lengths
    pbc: np.ndarray            # (3,) int32, 1 = periodic
    kind: int                  # MD_TERSOFF or MD_SW
    params: tuple              # packed parameters
    mass: float                # amu (single-element systems)
    vel: np.ndarray = field(default=None)  # (N,3) float64, Angstrom/fs
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def types(self) -> np.ndarray:
        return np.zeros(self.n, dtype=np.int32)


# ---------------------------------------------------------------------------
# Lattices
# ---------------------------------------------------------------------------
_DIAMOND_BASIS = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


def diamond_positions(n: int, a: float, ny: int | None = None, nz: int | None = None):
    """Cubic diamond, n x ny x nz conventional cells (8 atoms each), cell-major order."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + _DIAMOND_BASIS[None, :, :]).reshape(-1, 3) * a
    box = np.array([n * a, ny * a, nz * a], dtype=np.float64)
    return pos, box


def graphene_positions(nx: int, ny: int, a_cc: float, lz: float):
    """Flat honeycomb sheet in the xy plane, rectangular 4-atom cells (3 a_cc x sqrt3 a_cc).

    The sheet sits at z = lz/2; lz is the periodic length along z (vacuum + sheet).
    """
    s3 = math.sqrt(3.0)
    basis = np.array([[0.0, 0.0], [1.0, 0.0], [1.5, 0.5 * s3], [2.5, 0.5 * s3]]) * a_cc
    lx, ly = 3.0 * a_cc, s3 * a_cc
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    org = np.stack([ix.ravel() * lx, iy.ravel() * ly], axis=1)
    xy = (org[:, None, :] + basis[None, :, :]).reshape(-1, 2)
    pos = np.concatenate([xy, np.full((xy.shape[0], 1), 0.5 * lz)], axis=1)
    box = np.array([nx * lx, ny * ly, lz], dtype=np.float64)
    return pos, box


def wrap(pos: np.ndarray, box: np.ndarray, pbc: np.ndarray) -> np.ndarray:
    out = pos.copy()
    for d in range(3):
        if pbc[d]:
            out[:, d] = np.mod(out[:, d], box[d])
            out[:, d] = np.where(out[:, d] >= box[d], out[:, d] - box[d], out[:, d])
    return out


def jitter(pos: np.ndarray, amp: float, seed: int) -> np.ndarray:
    """Independent uniform displacement in [-amp, amp] per component."""
    if amp == 0.0:
        return pos.copy()
    rng = np.random.Generator(np.random.PCG64(seed))
    return pos + rng.uniform(-amp, amp, size=pos.shape)


def maxwell_boltzmann(n: int, mass: float, temperature: float, seed: int) -> np.ndarray:
    """Gaussian velocities at `temperature`, zero total momentum, rescaled so that the
    kinetic temperature with 3N-3 degrees of freedom equals `temperature` exactly."""
    if n == 0 or temperature == 0.0:
        return np.zeros((n, 3))
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma = math.sqrt(KB_EV_PER_K * temperature / mass * EV_PER_A_AMU_TO_A_PER_FS2)
    v = rng.normal(0.0, sigma, size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0, keepdims=True)
        ke = 0.5 * mass * np.sum(v * v) / EV_PER_A_AMU_TO_A_PER_FS2
        dof = 3 * n - 3
        t_now = 2.0 * ke / (dof * KB_EV_PER_K)
        v *= math.sqrt(temperature / t_now)
    return v


# ---------------------------------------------------------------------------
# Named workloads (shapes of the paper's test systems)
# ---------------------------------------------------------------------------
def si_diamond_tersoff(n: int = 6, a: float = 5.432, jitter_amp: float = 0.05,
                       temperature: float = 300.0, seed_pos: int = 1, seed_vel: int = 2) -> System:
    """Tersoff-1989 Si diamond, n^3 conventional cells (default 6^3 = 1728 atoms)."""
    pos, box = diamond_positions(n, a)
    pbc = np.array([1, 1, 1], dtype=np.int32)
    pos = wrap(jitter(pos, jitter_amp, seed_pos), box, pbc)
    vel = maxwell_boltzmann(pos.shape[0], MASS_SI, temperature, seed_vel)
    return System(f"tersoff_si_diamond_{n}", pos, box, pbc, MD_TERSOFF, TERSOFF_SI_1989,
                  MASS_SI, vel, dict(n_cells=n, a=a, jitter=jitter_amp, T=temperature))


def si_diamond_sw(n: int = 40, a: float = 5.431, jitter_amp: float = 0.0,
                  temperature: float = 300.0, seed_pos: int = 1, seed_vel: int = 2) -> System:
    """Stillinger-Weber Si diamond, n^3 conventional cells (default 40^3 = 512,000 atoms).

    a = 5.431 Angstrom is the lattice constant at which the SW two-body term sits at
    its minimum (nearest-neighbour distance 2^(1/6) sigma)."""
    pos, box = diamond_positions(n, a)
    pbc = np.array([1, 1, 1], dtype=np.int32)
    pos = wrap(jitter(pos, jitter_amp, seed_pos), box, pbc)
    vel = maxwell_boltzmann(pos.shape[0], MASS_SI, temperature, seed_vel)
    return System(f"sw_si_diamond_{n}", pos, box, pbc, MD_SW, SW_SI_1985, MASS_SI, vel,
                  dict(n_cells=n, a=a, jitter=jitter_amp, T=temperature))


def c_graphene_tersoff(nx: int = 500, ny: int = 500, a_cc: float = 1.42, lz: float = 20.0,
                       jitter_amp: float = 0.02, temperature: float = 300.0,
                       seed_pos: int = 1, seed_vel: int = 2) -> System:
    """Tersoff-1989 C honeycomb sheet, 4 nx ny atoms (default 10^6), periodic in-plane,
    periodic along z with lz = 20 Angstrom (sheet + vacuum)."""
    pos, box = graphene_positions(nx, ny, a_cc, lz)
    pbc = np.array([1, 1, 1], dtype=np.int32)
    pos = wrap(jitter(pos, jitter_amp, seed_pos), box, pbc)
    vel = maxwell_boltzmann(pos.shape[0], MASS_C, temperature, seed_vel)
    return System(f"tersoff_c_graphene_{nx}x{ny}", pos, box, pbc, MD_TERSOFF, TERSOFF_C_1989,
                  MASS_C, vel, dict(nx=nx, ny=ny, a_cc=a_cc, lz=lz, jitter=jitter_amp,
                                    T=temperature))


def c_diamond_tersoff(n: int = 4, a: float = 3.566, jitter_amp: float = 0.02,
                      temperature: float = 300.0, seed_pos: int = 1, seed_vel: int = 2) -> System:
    pos, box = diamond_positions(n, a)
    pbc = np.array([1, 1, 1], dtype=np.int32)
    pos = wrap(jitter(pos, jitter_amp, seed_pos), box, pbc)
    vel = maxwell_boltzmann(pos.shape[0], MASS_C, temperature, seed_vel)
    return System(f"tersoff_c_diamond_{n}", pos, box, pbc, MD_TERSOFF, TERSOFF_C_1989,
                  MASS_C, vel, dict(n_cells=n, a=a, jitter=jitter_amp, T=temperature))


def cluster(base: System, radius: float, vacuum: float = 12.0) -> System:
    """Non-periodic spherical cluster cut from `base` (all pbc = 0), centred in a box
    with `vacuum` of empty space on every side."""
    c = base.box * 0.5
    d = base.pos - c
    keep = np.sum(d * d, axis=1) < radius * radius
    pos = d[keep]
    lo = pos.min(axis=0) - vacuum
    pos = pos - lo
    box = pos.max(axis=0) + vacuum
    vel = None if base.vel is None else base.vel[keep].copy()
    return System(base.name + f"_cluster_r{radius:g}", pos, box, np.zeros(3, dtype=np.int32),
                  base.kind, base.params, base.mass, vel, dict(base.meta, radius=radius))


def random_cell(n: int, box, dmin: float, kind: int, params, mass: float, seed: int,
                temperature: float = 300.0, pbc=(1, 1, 1)) -> System:
    """n atoms placed uniformly at random in an orthorhombic box, rejecting any closer
    than dmin to an already placed atom (minimum image on periodic axes)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    box = np.asarray(box, dtype=np.float64)
    pbc = np.asarray(pbc, dtype=np.int32)
    pos = np.zeros((0, 3))
    tries = 0
    while pos.shape[0] < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("random_cell: could not place atoms")
        p = rng.uniform(0.0, 1.0, size=3) * box
        if pos.shape[0]:
            d = pos - p
            d -= np.round(d / box) * box * pbc
            if np.min(np.sum(d * d, axis=1)) < dmin * dmin:
                continue
        pos = np.vstack([pos, p])
    vel = maxwell_boltzmann(n, mass, temperature, seed + 1)
    return System(f"random_cell_{n}", pos, box, pbc, kind, tuple(params), mass, vel,
                  dict(dmin=dmin, seed=seed))


# Batched workload: atom counts drawn log-uniform, snapped to the nearest admissible
# lattice (8 n^3 for diamond, 4 nx ny for a square-ish graphene patch).
def batch_sizes(n_sys: int, lo: int, hi: int, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    target = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_sys))
    kinds = rng.integers(0, 2, size=n_sys)  # 0 = Si diamond, 1 = C graphene
    out = []
    for t, k in zip(target, kinds):
        if k == 0:
            n = max(2, int(round((t / 8.0) ** (1.0 / 3.0))))
            out.append(("si_diamond", n, n, 8 * n ** 3))
        else:
            # graphene rectangular cells are 4.26 x 2.46 Angstrom: take ny ~ 1.73 nx for a
            # near-square patch, with at least 3 cells per side along each axis
            nx = max(3, int(round(math.sqrt(t / 4.0 / 1.732))))
            ny = max(3, int(round(1.732 * nx)))
            out.append(("c_graphene", nx, ny, 4 * nx * ny))
    return out


# ---------------------------------------------------------------------------
# Several elements (multi-element Tersoff)
# ---------------------------------------------------------------------------
@dataclass
class MultiSystem:
    """A synthetic system of several elements: per-atom element index `types`, a
    parameter row per element (`params`, n_types x 11), the bond-order factors `chi`
    (n_types x n_types) and a mass per element."""
    name: str
    pos: np.ndarray
    box: np.ndarray
    pbc: np.ndarray
    types: np.ndarray          # (N,) int32
    params: tuple              # n_types rows of 11
    chi: tuple                 # n_types x n_types
    masses: tuple              # amu per element
    vel: np.ndarray = field(default=None)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def atom_masses(self) -> np.ndarray:
        return np.asarray(self.masses, dtype=np.float64)[self.types]


def maxwell_boltzmann_per_atom(masses: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Gaussian velocities for per-atom masses, zero total momentum, rescaled so that the
    kinetic temperature with 3N-3 degrees of freedom equals `temperature` exactly."""
    m = np.asarray(masses, dtype=np.float64)
    n = m.shape[0]
    if n == 0 or temperature == 0.0:
        return np.zeros((n, 3))
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma = np.sqrt(KB_EV_PER_K * temperature / m * EV_PER_A_AMU_TO_A_PER_FS2)
    v = rng.normal(0.0, 1.0, size=(n, 3)) * sigma[:, None]
    if n > 1:
        v -= (m[:, None] * v).sum(axis=0, keepdims=True) / m.sum()
        ke = 0.5 * np.sum(m[:, None] * v * v) / EV_PER_A_AMU_TO_A_PER_FS2
        t_now = 2.0 * ke / ((3 * n - 3) * KB_EV_PER_K)
        v *= math.sqrt(temperature / t_now)
    return v


def sic_zincblende(n: int = 4, a: float = 4.32, jitter_amp: float = 0.03, temperature: float = 300.0,
                   seed_pos: int = 1, seed_vel: int = 2) -> MultiSystem:
    """3C-SiC (zincblende): Si on the fcc sites, C on the fcc sites shifted by a(1,1,1)/4;
    n^3 conventional cells of 8 atoms, Tersoff 1989 Si-C parameters."""
    pos, box = diamond_positions(n, a)
    pbc = np.array([1, 1, 1], dtype=np.int32)
    types = np.tile(np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.int32), n ** 3)
    pos = wrap(jitter(pos, jitter_amp, seed_pos), box, pbc)
    masses = (MASS_SI, MASS_C)
    vel = maxwell_boltzmann_per_atom(np.asarray(masses)[types], temperature, seed_vel)
    return MultiSystem(f"tersoff_sic_zincblende_{n}", pos, box, pbc, types, TERSOFF_SIC_1989, CHI_SIC_1989,
                       masses, vel, dict(n_cells=n, a=a, jitter=jitter_amp, T=temperature))


def sic_substituted_diamond(n: int = 4, a: float = 5.2, c_fraction: float = 0.3, jitter_amp: float = 0.08,
                            temperature: float = 300.0, seed_types: int = 5, seed_pos: int = 6,
                            seed_vel: int = 7) -> MultiSystem:
    """Diamond lattice with a random fraction of the sites carbon, the rest silicon: every
    element pair meets (Si-Si, Si-C, C-C), and at a = 5.2 A the 2.25 A bonds fall inside
    the Si-Si core, the Si-C switching shell and beyond the C-C cutoff."""
    pos, box = diamond_positions(n, a)
    pbc = np.array([1, 1, 1], dtype=np.int32)
    rng = np.random.Generator(np.random.PCG64(seed_types))
    types = (rng.uniform(0.0, 1.0, size=pos.shape[0]) < c_fraction).astype(np.int32)
    pos = wrap(jitter(pos, jitter_amp, seed_pos), box, pbc)
    masses = (MASS_SI, MASS_C)
    vel = maxwell_boltzmann_per_atom(np.asarray(masses)[types], temperature, seed_vel)
    return MultiSystem(f"tersoff_sic_substituted_{n}", pos, box, pbc, types, TERSOFF_SIC_1989, CHI_SIC_1989,
                       masses, vel, dict(n_cells=n, a=a, c_fraction=c_fraction, jitter=jitter_amp, T=temperature))
