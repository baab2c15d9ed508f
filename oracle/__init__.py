"""CPU oracle for many-body MD (Tersoff, Stillinger-Weber) -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs may
import this package.  The CUDA product path never does, and this package imports
nothing from the CUDA package.  The arithmetic lives in oracle.c (plain C, fp64, no
fast-math, no FMA contraction); this module compiles it with gcc and marshals numpy
arrays through ctypes.

Functions follow the paper (arXiv:1610.03343) as documented in oracle.c:
  neighbors            Sec. 2.1 neighbour list (brute force or linked-list cells)
  tersoff_conventional Algorithm 1 with Eqs. 7-11 (U_i, F_i, Eq. 22 virial, total W)
  tersoff_dUdr         dU_i/dr_ij per list slot (the quantity of Eqs. 14, 28-30)
  sw_conventional / sw_dUdr   the same two routes for Stillinger-Weber
  manybody_fwj         Eqs. 28-30 (F_i, W_i, J_i) from dU_i/dr_ij
  run                  velocity Verlet with per-step U, K, J
  run_npt              the same with the Berendsen thermostat and barostat (NPT)
  tersoff_multi_conventional / tersoff_multi_dUdr / compute_multi / run_multi
                       multi-element Tersoff (Tersoff 1989 mixing rules and chi)
  hcacf, running_kappa Green-Kubo HCACF and thermal conductivity from a J series
                       (green_kubo.py, numpy)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .green_kubo import hcacf, running_kappa  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

TERSOFF = 1
SW = 2

_CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_neighbors_brute.argtypes = [I64, P, P, P, P, P, D, I, P, P]
        lib.oracle_neighbors_cells.argtypes = [I64, P, P, P, P, P, D, I, P, P]
        lib.oracle_tersoff_conventional.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_tersoff_dUdr.argtypes = [I64, P, P, P, P, P, P, I, P, P, P, P]
        lib.oracle_sw_conventional.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_sw_dUdr.argtypes = [I64, P, P, P, P, P, P, I, P, P, P, P]
        lib.oracle_manybody_fwj.argtypes = [I64, P, P, P, P, P, I, P, P, P, P, P, P, P, P, P]
        lib.oracle_run.argtypes = [I64, P, P, P, P, P, P, P, P, P, I, P, I, I64, D, D, P]
        lib.oracle_run_ex.argtypes = [I64, P, P, P, P, P, P, P, P, P, I, P, I, I64, D, D, P, P]
        lib.oracle_tersoff_multi_conventional.argtypes = [I64, P, P, P, P, P, P, I, P, P, P, P, P, P, P]
        lib.oracle_tersoff_multi_dUdr.argtypes = [I64, P, P, P, P, P, P, I, P, P, I, P, P, P, P]
        lib.oracle_run_multi.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, I, P, P, I, I64, D, D, P, P]
        for f in ("oracle_neighbors_brute", "oracle_neighbors_cells", "oracle_tersoff_conventional",
                  "oracle_tersoff_dUdr", "oracle_sw_conventional", "oracle_sw_dUdr",
                  "oracle_manybody_fwj", "oracle_run", "oracle_run_ex", "oracle_tersoff_multi_conventional",
                  "oracle_tersoff_multi_dUdr", "oracle_run_multi"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _soa(pos):
    pos = np.asarray(pos, dtype=np.float64)
    return (np.ascontiguousarray(pos[:, 0]), np.ascontiguousarray(pos[:, 1]),
            np.ascontiguousarray(pos[:, 2]))


def _box(box, pbc):
    return (np.ascontiguousarray(box, dtype=np.float64),
            np.ascontiguousarray(pbc, dtype=np.int32))


def neighbors(pos, box, pbc, rc, cap=32, method="auto"):
    """Neighbour list within rc: NN (N,), NL (cap, N) sorted ascending.  Raises on overflow."""
    lib = _load()
    x, y, z = _soa(pos)
    b, p = _box(box, pbc)
    n = x.shape[0]
    NN = np.zeros(max(n, 1), dtype=np.int32)
    NL = np.full((cap, max(n, 1)), -1, dtype=np.int32)
    if method == "auto":
        method = "brute" if n <= 4096 else "cells"
    fn = lib.oracle_neighbors_brute if method == "brute" else lib.oracle_neighbors_cells
    maxc = fn(n, _p(x), _p(y), _p(z), _p(b), _p(p), float(rc), int(cap), _p(NN), _p(NL))
    if maxc < 0:
        raise MemoryError("oracle neighbour build failed")
    if maxc > cap:
        raise OverflowError(f"neighbour list overflow: {maxc} > cap {cap}")
    return NN[:n], NL[:, :n].copy()


def tersoff_conventional(pos, box, pbc, params, NN, NL):
    """Algorithm 1: returns U (N,), F (N,3), W_lammps (N,9) [Eq. 22], W_total (9,)."""
    lib = _load()
    x, y, z = _soa(pos)
    b, p = _box(box, pbc)
    n = x.shape[0]
    prm = np.ascontiguousarray(params, dtype=np.float64)
    U = np.zeros(n)
    F = np.zeros(3 * n)
    W = np.zeros(9 * n)
    Wt = np.zeros(9)
    NN = np.ascontiguousarray(NN, dtype=np.int32)
    NL = np.ascontiguousarray(NL, dtype=np.int32)
    lib.oracle_tersoff_conventional(n, _p(x), _p(y), _p(z), _p(b), _p(p), _p(prm), _p(NN), _p(NL),
                                    _p(U), _p(F), _p(W), _p(Wt))
    return U, F.reshape(3, n).T.copy(), W.reshape(9, n).T.copy(), Wt


def sw_conventional(pos, box, pbc, params, NN, NL):
    """Conventional SW: returns U (N,), F (N,3), W_total (9,)."""
    lib = _load()
    x, y, z = _soa(pos)
    b, p = _box(box, pbc)
    n = x.shape[0]
    prm = np.ascontiguousarray(params, dtype=np.float64)
    U = np.zeros(n)
    F = np.zeros(3 * n)
    Wt = np.zeros(9)
    NN = np.ascontiguousarray(NN, dtype=np.int32)
    NL = np.ascontiguousarray(NL, dtype=np.int32)
    lib.oracle_sw_conventional(n, _p(x), _p(y), _p(z), _p(b), _p(p), _p(prm), _p(NN), _p(NL),
                               _p(U), _p(F), _p(Wt))
    return U, F.reshape(3, n).T.copy(), Wt


def dUdr(kind, pos, box, pbc, params, NN, NL):
    """Per-slot dU_i/dr_ij: returns U (N,), D (3, cap, N)."""
    lib = _load()
    x, y, z = _soa(pos)
    b, p = _box(box, pbc)
    n = x.shape[0]
    NL = np.ascontiguousarray(NL, dtype=np.int32)
    cap = NL.shape[0]
    prm = np.ascontiguousarray(params, dtype=np.float64)
    U = np.zeros(n)
    D = np.zeros(3 * cap * n)
    NN = np.ascontiguousarray(NN, dtype=np.int32)
    fn = lib.oracle_tersoff_dUdr if kind == TERSOFF else lib.oracle_sw_dUdr
    fn(n, _p(x), _p(y), _p(z), _p(b), _p(p), _p(prm), cap, _p(NN), _p(NL), _p(U), _p(D))
    return U, D.reshape(3, cap, n)


def manybody_fwj(pos, box, pbc, NN, NL, D, vel=None):
    """Eqs. 28-30: F (N,3), W (N,9), J (N,3) (J is None without velocities)."""
    lib = _load()
    x, y, z = _soa(pos)
    b, p = _box(box, pbc)
    n = x.shape[0]
    NL = np.ascontiguousarray(NL, dtype=np.int32)
    cap = NL.shape[0]
    NN = np.ascontiguousarray(NN, dtype=np.int32)
    D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1)
    F = np.zeros(3 * n)
    W = np.zeros(9 * n)
    J = np.zeros(3 * n)
    if vel is not None:
        vx, vy, vz = _soa(vel)
    else:
        vx = vy = vz = None
    rc = lib.oracle_manybody_fwj(n, _p(x), _p(y), _p(z), _p(b), _p(p), cap, _p(NN), _p(NL), _p(D),
                                 _p(vx), _p(vy), _p(vz), _p(F), _p(W), _p(J))
    if rc != 0:
        raise RuntimeError("asymmetric neighbour list")
    return (F.reshape(3, n).T.copy(), W.reshape(9, n).T.copy(),
            None if vel is None else J.reshape(3, n).T.copy())


def cutoff(kind, params):
    return float(params[10]) if kind == TERSOFF else float(params[1] * params[2])


def compute(pos, box, pbc, kind, params, vel=None, cap=32):
    """Everything one force evaluation defines, from positions (and velocities):
    U_i and F_i by the conventional loop (Algorithm 1), W_i (Eq. 29) and J_i (Eq. 30)
    from dU_i/dr_ij, and system totals.  Returns a dict of numpy arrays."""
    rc = cutoff(kind, params)
    NN, NL = neighbors(pos, box, pbc, rc, cap)
    if kind == TERSOFF:
        U, F, Wlmp, Wtot_conv = tersoff_conventional(pos, box, pbc, params, NN, NL)
    else:
        U, F, Wtot_conv = sw_conventional(pos, box, pbc, params, NN, NL)
        Wlmp = None
    Ud, D = dUdr(kind, pos, box, pbc, params, NN, NL)
    Fp, W, J = manybody_fwj(pos, box, pbc, NN, NL, D, vel)
    out = dict(U=U, F=F, W=W, J=J, F_pair=Fp, U_d=Ud, W_lammps=Wlmp, W_total_conv=Wtot_conv,
               NN=NN, NL=NL, D=D)
    out["totals"] = np.concatenate([[U.sum()], W.sum(axis=0),
                                    J.sum(axis=0) if J is not None else np.zeros(3)])
    return out


def run(pos, vel, masses, box, pbc, kind, params, n_steps, dt, cap=32, damp=0.0):
    """Velocity Verlet for n_steps (optionally damped, v *= 1 - damp dt after each step):
    returns (pos, vel, series[n_steps, 5] = U, K, Jx, Jy, Jz)."""
    lib = _load()
    x, y, z = _soa(pos)
    vx, vy, vz = _soa(vel)
    n = x.shape[0]
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(masses, dtype=np.float64), (n,)))
    b, p = _box(box, pbc)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    series = np.zeros(5 * max(n_steps, 1))
    rc = lib.oracle_run(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), _p(m), _p(b), _p(p),
                        int(kind), _p(prm), int(cap), int(n_steps), float(dt), float(damp), _p(series))
    if rc != 0:
        raise RuntimeError(f"oracle_run failed: {rc}")
    return (np.stack([x, y, z], axis=1), np.stack([vx, vy, vz], axis=1),
            series[:5 * n_steps].reshape(n_steps, 5))


def run_npt(pos, vel, masses, box, pbc, kind, params, n_steps, dt, T0=300.0, P0=0.0, tau_T=100.0, tau_P=1000.0,
            beta=0.01, couple=(1, 1, 1), cap=32, damp=0.0):
    """Velocity Verlet with the Berendsen thermostat and barostat (oracle.c,
    oracle_run_ex): returns (pos, vel, series[n_steps, 5], box).  The scaling computed at
    the last step is left pending, as the library leaves it for its next run."""
    lib = _load()
    x, y, z = _soa(pos)
    vx, vy, vz = _soa(vel)
    n = x.shape[0]
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(masses, dtype=np.float64), (n,)))
    b, p = _box(box, pbc)
    b = np.array(b, dtype=np.float64)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    npt = np.array([T0, P0, tau_T, tau_P, beta, *[float(c) for c in couple]], dtype=np.float64)
    series = np.zeros(5 * max(n_steps, 1))
    rc = lib.oracle_run_ex(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), _p(m), _p(b), _p(p), int(kind),
                           _p(prm), int(cap), int(n_steps), float(dt), float(damp), _p(npt), _p(series))
    if rc != 0:
        raise RuntimeError(f"oracle_run_ex failed: {rc}")
    return (np.stack([x, y, z], axis=1), np.stack([vx, vy, vz], axis=1),
            series[:5 * n_steps].reshape(n_steps, 5), b)


def kinetic_energy(vel, masses):
    """Sum 1/2 m v^2 in eV."""
    v = np.asarray(vel)
    m = np.broadcast_to(np.asarray(masses, dtype=np.float64), (v.shape[0],))
    return float(0.5 * np.sum(m[:, None] * v * v) / 9.648533215665328e-3)


# ---------------------------------------------------------------- multi-element Tersoff
def _multi_args(types, params, chi):
    params = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1, 11))
    nt = params.shape[0]
    chi = np.ascontiguousarray(np.asarray(chi, dtype=np.float64).reshape(nt, nt))
    types = np.ascontiguousarray(types, dtype=np.int32)
    return types, nt, params.reshape(-1).copy(), chi.reshape(-1).copy()


def multi_cutoff(params):
    """Largest mixed cutoff sqrt(S_a S_b) of a multi-element parameter table."""
    S = np.asarray(params, dtype=np.float64).reshape(-1, 11)[:, 10]
    return float(np.sqrt(np.outer(S, S)).max())


def tersoff_multi_conventional(pos, box, pbc, types, params, chi, NN, NL):
    """Algorithm 1 for multi-element Tersoff: U (N,), F (N,3), W_total (9,)."""
    lib = _load()
    x, y, z = _soa(pos)
    b, p = _box(box, pbc)
    n = x.shape[0]
    t, nt, prm, ch = _multi_args(types, params, chi)
    U = np.zeros(n)
    F = np.zeros(3 * n)
    Wt = np.zeros(9)
    NN = np.ascontiguousarray(NN, dtype=np.int32)
    NL = np.ascontiguousarray(NL, dtype=np.int32)
    rc = lib.oracle_tersoff_multi_conventional(n, _p(x), _p(y), _p(z), _p(b), _p(p), _p(t), nt, _p(prm), _p(ch),
                                               _p(NN), _p(NL), _p(U), _p(F), _p(Wt))
    if rc != 0:
        raise ValueError("bad multi-element parameters")
    return U, F.reshape(3, n).T.copy(), Wt


def tersoff_multi_dUdr(pos, box, pbc, types, params, chi, NN, NL):
    """Per-slot dU_i/dr_ij for multi-element Tersoff: U (N,), D (3, cap, N)."""
    lib = _load()
    x, y, z = _soa(pos)
    b, p = _box(box, pbc)
    n = x.shape[0]
    t, nt, prm, ch = _multi_args(types, params, chi)
    NL = np.ascontiguousarray(NL, dtype=np.int32)
    cap = NL.shape[0]
    NN = np.ascontiguousarray(NN, dtype=np.int32)
    U = np.zeros(n)
    D = np.zeros(3 * cap * n)
    rc = lib.oracle_tersoff_multi_dUdr(n, _p(x), _p(y), _p(z), _p(b), _p(p), _p(t), nt, _p(prm), _p(ch), cap,
                                       _p(NN), _p(NL), _p(U), _p(D))
    if rc != 0:
        raise ValueError("bad multi-element parameters")
    return U, D.reshape(3, cap, n)


def compute_multi(pos, box, pbc, types, params, chi, vel=None, cap=32):
    """compute() for multi-element Tersoff: U_i, F_i by Algorithm 1, W_i and J_i (Eqs.
    29-30) from dU_i/dr_ij, totals."""
    rc = multi_cutoff(params)
    NN, NL = neighbors(pos, box, pbc, rc, cap)
    U, F, Wtot_conv = tersoff_multi_conventional(pos, box, pbc, types, params, chi, NN, NL)
    Ud, D = tersoff_multi_dUdr(pos, box, pbc, types, params, chi, NN, NL)
    Fp, W, J = manybody_fwj(pos, box, pbc, NN, NL, D, vel)
    out = dict(U=U, F=F, W=W, J=J, F_pair=Fp, U_d=Ud, W_total_conv=Wtot_conv, NN=NN, NL=NL, D=D)
    out["totals"] = np.concatenate([[U.sum()], W.sum(axis=0),
                                    J.sum(axis=0) if J is not None else np.zeros(3)])
    return out


def run_multi(pos, vel, masses, box, pbc, types, params, chi, n_steps, dt, cap=32, damp=0.0):
    """Velocity Verlet with multi-element Tersoff (masses per atom): (pos, vel, series)."""
    lib = _load()
    x, y, z = _soa(pos)
    vx, vy, vz = _soa(vel)
    n = x.shape[0]
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(masses, dtype=np.float64), (n,)))
    b, p = _box(box, pbc)
    b = np.array(b, dtype=np.float64)
    t, nt, prm, ch = _multi_args(types, params, chi)
    series = np.zeros(5 * max(n_steps, 1))
    rc = lib.oracle_run_multi(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), _p(m), _p(b), _p(p), _p(t), nt,
                              _p(prm), _p(ch), int(cap), int(n_steps), float(dt), float(damp), None, _p(series))
    if rc != 0:
        raise RuntimeError(f"oracle_run_multi failed: {rc}")
    return (np.stack([x, y, z], axis=1), np.stack([vx, vy, vz], axis=1),
            series[:5 * n_steps].reshape(n_steps, 5))
