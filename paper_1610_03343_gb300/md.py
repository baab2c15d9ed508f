"""Thin Python binding of libmd.so (include/md.h) -- argument marshalling only.

Every computation runs in the CUDA library.  The functions below carry the C names
(md_create, md_set_positions, md_compute, md_run, md_get_state, ...) and take numpy
arrays (host I/O) or torch CUDA tensors (device I/O); `System` is a small convenience
wrapper over one context.  Loading fails loudly if the library has not been built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

MD_OK = 0
MD_TERSOFF = 1
MD_SW = 2
MD_FP64 = 0
MD_MIXED = 1
MD_IO_HOST = 0
MD_IO_DEVICE = 1
MD_ERR_ARG, MD_ERR_BOX, MD_ERR_NEIGH_OVERFLOW, MD_ERR_OOM = -1, -2, -3, -4
MD_ERR_CUDA, MD_ERR_TIMEOUT, MD_ERR_NAN, MD_ERR_STATE = -5, -6, -7, -8
MD_DOMAIN_POSITIONS, MD_DOMAIN_MIGRATE, MD_DOMAIN_GHOSTS = 0, 1, 2

STATUS = {0: "MD_OK", -1: "MD_ERR_ARG", -2: "MD_ERR_BOX", -3: "MD_ERR_NEIGH_OVERFLOW",
          -4: "MD_ERR_OOM", -5: "MD_ERR_CUDA", -6: "MD_ERR_TIMEOUT", -7: "MD_ERR_NAN",
          -8: "MD_ERR_STATE"}


class MDError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class md_params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_types", ctypes.c_int), ("p", ctypes.POINTER(ctypes.c_double))]


class md_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skin", ctypes.c_double), ("max_neigh", ctypes.c_int),
                ("max_active", ctypes.c_int), ("io", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("hbm_budget", ctypes.c_size_t), ("device", ctypes.c_int)]


class md_batch_options(ctypes.Structure):
    _fields_ = [("max_box", ctypes.c_double), ("cell_capacity", ctypes.c_int64)]


class md_system(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("pbc", ctypes.c_int * 3), ("n_atoms", ctypes.c_int64),
                ("types", ctypes.c_void_p), ("param_set", ctypes.c_int),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p),
                ("n_steps", ctypes.c_int64), ("damp", ctypes.c_double)]


class md_server_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tersoff_atoms", ctypes.c_int64), ("sw_atoms", ctypes.c_int64),
                ("max_jobs_per_pool", ctypes.c_int), ("tersoff_dt", ctypes.c_double), ("sw_dt", ctypes.c_double),
                ("chunk_steps", ctypes.c_int), ("device", ctypes.c_int)]


class md_job(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("param_set", ctypes.c_int), ("box", ctypes.c_double * 3),
                ("pbc", ctypes.c_int * 3), ("n_atoms", ctypes.c_int64), ("types", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("vz", ctypes.c_void_p),
                ("n_steps", ctypes.c_int64), ("damp", ctypes.c_double),
                ("x_out", ctypes.c_void_p), ("v_out", ctypes.c_void_p)]


class md_job_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("U", ctypes.c_double),
                ("K", ctypes.c_double)]


class md_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("atom_steps", ctypes.c_double), ("busy_seconds", ctypes.c_double),
                ("run_seconds", ctypes.c_double), ("admit_seconds", ctypes.c_double),
                ("harvest_seconds", ctypes.c_double), ("chunks", ctypes.c_int64),
                ("resident_atom_steps", ctypes.c_double)]


class md_stats(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("steps_done", ctypes.c_int64), ("n_rebuilds", ctypes.c_int64),
                ("max_neigh_seen", ctypes.c_int), ("kernel_launches_per_step", ctypes.c_int),
                ("kernel_launches_per_rebuild", ctypes.c_int), ("pair_deferred", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("atoms_rebuilt", ctypes.c_int64),
                ("kernels_launched", ctypes.c_int64)]


class md_npt(ctypes.Structure):
    _fields_ = [("T0", ctypes.c_double), ("P0", ctypes.c_double), ("tau_T", ctypes.c_double),
                ("tau_P", ctypes.c_double), ("beta", ctypes.c_double), ("couple", ctypes.c_int * 3)]


MD_TUNE_MAX = 16


class md_tuning(ctypes.Structure):
    _fields_ = [("pair_block", ctypes.c_int), ("pool_blocks_per_sm", ctypes.c_int), ("n_tried", ctypes.c_int),
                ("tried_pair_block", ctypes.c_int * MD_TUNE_MAX),
                ("tried_blocks_per_sm", ctypes.c_int * MD_TUNE_MAX),
                ("tried_ms", ctypes.c_double * MD_TUNE_MAX),
                ("pair_cap", ctypes.c_int), ("tried_pair_cap", ctypes.c_int * MD_TUNE_MAX)]


_lock = threading.Lock()
_lib = None

EXPORTS = ["md_default_options", "md_create", "md_set_positions", "md_set_velocities", "md_compute",
           "md_run", "md_get_state", "md_checkpoint_size", "md_checkpoint_save", "md_checkpoint_load",
           "md_set_npt", "md_get_box", "md_get_stats", "md_set_graph_mode", "md_set_profiling",
           "md_kernel_times", "md_autotune", "md_set_tuning", "md_get_tuning", "md_batch_create", "md_batch_add", "md_batch_remove", "md_batch_status", "md_batch_errors",
           "md_batch_get_state", "md_server_create", "md_server_submit", "md_server_poll", "md_server_wait",
           "md_server_wait_timeout",
           "md_server_drain", "md_server_stats_get", "md_server_clock", "md_server_destroy",
           "md_compute_static", "md_hcacf", "md_fastmath_eval", "md_peak_flops",
           "md_domain_create", "md_domain_set_atoms", "md_domain_message_bound", "md_domain_pack",
           "md_domain_unpack", "md_domain_kick_drift", "md_domain_force", "md_domain_compute", "md_domain_owned",
           "md_domain_last_error", "md_domain_destroy", "md_last_error", "md_destroy"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libmd.so.  Raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(f"libmd.so not built ({_build.LIB}); run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(_build.LIB)
        P = ctypes.c_void_p
        S = ctypes.c_int
        lib.md_default_options.argtypes = [ctypes.POINTER(md_options)]
        lib.md_create.argtypes = [ctypes.POINTER(P), P, P, ctypes.c_int64, P, P,
                                  ctypes.POINTER(md_params), ctypes.POINTER(md_options)]
        lib.md_set_positions.argtypes = [P, P, P, P]
        lib.md_set_velocities.argtypes = [P, P, P, P]
        lib.md_compute.argtypes = [P, P, P, P, P, P]
        lib.md_run.argtypes = [P, ctypes.c_int64, ctypes.c_double, P]
        lib.md_get_state.argtypes = [P, P, P]
        lib.md_checkpoint_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        lib.md_checkpoint_save.argtypes = [P, P, ctypes.c_size_t]
        lib.md_checkpoint_load.argtypes = [P, P, ctypes.c_size_t]
        lib.md_set_npt.argtypes = [P, ctypes.c_int, ctypes.POINTER(md_npt)]
        lib.md_get_box.argtypes = [P, ctypes.c_int, P]
        lib.md_get_stats.argtypes = [P, ctypes.POINTER(md_stats)]
        lib.md_set_graph_mode.argtypes = [P, ctypes.c_int]
        lib.md_set_profiling.argtypes = [P, ctypes.c_int]
        lib.md_kernel_times.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int)]
        lib.md_autotune.argtypes = [P, ctypes.c_int, ctypes.POINTER(md_tuning)]
        lib.md_set_tuning.argtypes = [P, ctypes.POINTER(md_tuning)]
        lib.md_get_tuning.argtypes = [P, ctypes.POINTER(md_tuning)]
        lib.md_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(md_params), ctypes.c_int, P,
                                        ctypes.POINTER(md_batch_options), ctypes.POINTER(md_options)]
        lib.md_batch_add.argtypes = [P, ctypes.POINTER(md_system), ctypes.POINTER(ctypes.c_int)]
        lib.md_batch_remove.argtypes = [P, ctypes.c_int]
        lib.md_batch_status.argtypes = [P, P, P, P, P]
        lib.md_batch_errors.argtypes = [P, P]
        lib.md_batch_get_state.argtypes = [P, ctypes.c_int, P, P]
        lib.md_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(md_server_options),
                                         ctypes.POINTER(md_params), P, ctypes.POINTER(md_params), P]
        lib.md_server_submit.argtypes = [P, ctypes.POINTER(md_job), ctypes.POINTER(ctypes.c_int64)]
        lib.md_server_poll.argtypes = [P, ctypes.c_int64, ctypes.POINTER(md_job_result)]
        lib.md_server_wait.argtypes = [P, ctypes.c_int64, ctypes.POINTER(md_job_result)]
        lib.md_server_wait_timeout.argtypes = [P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(md_job_result)]
        lib.md_server_drain.argtypes = [P]
        lib.md_server_stats_get.argtypes = [P, ctypes.POINTER(md_server_stats)]
        lib.md_server_clock.argtypes = [P]
        lib.md_server_clock.restype = ctypes.c_double
        lib.md_server_destroy.argtypes = [P]
        lib.md_server_destroy.restype = None
        lib.md_compute_static.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, ctypes.c_int64, P, P, P, P, P, P,
                                          ctypes.c_double, P, P, P, P, P, P]
        lib.md_hcacf.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, P, P, ctypes.c_int, P]
        lib.md_fastmath_eval.argtypes = [ctypes.c_int, ctypes.c_int64, P, P]
        lib.md_fastmath_eval.restype = ctypes.c_int
        lib.md_peak_flops.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, P, P]
        lib.md_peak_flops.restype = ctypes.c_int
        lib.md_domain_create.argtypes = [ctypes.POINTER(P), P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int64, ctypes.POINTER(md_params), P, ctypes.POINTER(md_options)]
        lib.md_domain_set_atoms.argtypes = [P, ctypes.c_int64, P, P, P, P, P, P, P, P]
        lib.md_domain_message_bound.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
        lib.md_domain_pack.argtypes = [P, ctypes.c_int, P, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t)]
        lib.md_domain_unpack.argtypes = [P, ctypes.c_int, P, ctypes.c_size_t, P, ctypes.c_size_t]
        lib.md_domain_kick_drift.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
        lib.md_domain_force.argtypes = [P, ctypes.c_double, P]
        lib.md_domain_compute.argtypes = [P, P, P, P, P, P]
        lib.md_domain_owned.argtypes = [P, ctypes.POINTER(ctypes.c_int64), P, P, P]
        lib.md_domain_last_error.argtypes = [P]
        lib.md_domain_last_error.restype = ctypes.c_char_p
        lib.md_domain_destroy.argtypes = [P]
        lib.md_domain_destroy.restype = None
        lib.md_last_error.argtypes = [P]
        lib.md_last_error.restype = ctypes.c_char_p
        lib.md_destroy.argtypes = [P]
        lib.md_destroy.restype = None
        for f in EXPORTS:
            if f not in ("md_last_error", "md_destroy", "md_server_clock", "md_server_destroy",
                         "md_domain_last_error", "md_domain_destroy"):
                getattr(lib, f).restype = S
        _lib = lib
        return lib


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(type(a))


def _check(lib, ctx, status):
    if status != MD_OK:
        msg = lib.md_last_error(ctx).decode() if ctx else ""
        raise MDError(status, msg)


# ----------------------------------------------------------------- C names
def md_default_options() -> md_options:
    lib = load()
    o = md_options()
    _check(lib, None, lib.md_default_options(ctypes.byref(o)))
    return o


def md_create(box, pbc, n_atoms, types, masses_by_type, kind, params, opt: md_options | None = None, n_types=1):
    """params: one element's packed parameters, or (n_types > 1, Tersoff) n_types rows of 11
    followed by the n_types x n_types chi factors."""
    lib = load()
    box = np.ascontiguousarray(box, dtype=np.float64)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32)
    types = np.ascontiguousarray(types, dtype=np.int32)
    masses = np.ascontiguousarray(masses_by_type, dtype=np.float64)
    prm_arr = np.ascontiguousarray(params, dtype=np.float64)
    prm = md_params(int(kind), int(n_types), prm_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    ctx = ctypes.c_void_p()
    st = lib.md_create(ctypes.byref(ctx), _ptr(box), _ptr(pbc), int(n_atoms), _ptr(types), _ptr(masses),
                       ctypes.byref(prm), ctypes.byref(opt) if opt is not None else None)
    if st != MD_OK:
        raise MDError(st, "md_create failed")
    return ctx


def md_set_positions(ctx, x, y, z):
    lib = load()
    _check(lib, ctx, lib.md_set_positions(ctx, _ptr(x), _ptr(y), _ptr(z)))


def md_set_velocities(ctx, vx, vy, vz):
    lib = load()
    _check(lib, ctx, lib.md_set_velocities(ctx, _ptr(vx), _ptr(vy), _ptr(vz)))


def md_compute(ctx, f=None, u=None, w=None, j=None, totals=None):
    lib = load()
    _check(lib, ctx, lib.md_compute(ctx, _ptr(f), _ptr(u), _ptr(w), _ptr(j), _ptr(totals)))


def md_run(ctx, n_steps, dt_fs, series=None):
    lib = load()
    _check(lib, ctx, lib.md_run(ctx, int(n_steps), float(dt_fs), _ptr(series)))


def md_get_state(ctx, x=None, v=None):
    lib = load()
    _check(lib, ctx, lib.md_get_state(ctx, _ptr(x), _ptr(v)))


def md_checkpoint_size(ctx) -> int:
    lib = load()
    n = ctypes.c_size_t()
    _check(lib, ctx, lib.md_checkpoint_size(ctx, ctypes.byref(n)))
    return n.value


def md_checkpoint_save(ctx) -> np.ndarray:
    """The context's full state as a host byte array (md_checkpoint_save)."""
    lib = load()
    buf = np.zeros(md_checkpoint_size(ctx), dtype=np.uint8)
    _check(lib, ctx, lib.md_checkpoint_save(ctx, _ptr(buf), buf.size))
    return buf


def md_checkpoint_load(ctx, buf):
    lib = load()
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib, ctx, lib.md_checkpoint_load(ctx, _ptr(buf), buf.size))


def md_set_npt(ctx, system=0, T0=300.0, P0=0.0, tau_T=100.0, tau_P=1000.0, beta=0.01, couple=(1, 1, 1),
               off=False):
    """Berendsen coupling of one system (off=True: back to NVE)."""
    lib = load()
    if off:
        _check(lib, ctx, lib.md_set_npt(ctx, int(system), None))
        return
    c = md_npt()
    c.T0, c.P0, c.tau_T, c.tau_P, c.beta = float(T0), float(P0), float(tau_T), float(tau_P), float(beta)
    c.couple = (ctypes.c_int * 3)(*[int(a) for a in couple])
    _check(lib, ctx, lib.md_set_npt(ctx, int(system), ctypes.byref(c)))


def md_get_box(ctx, system=0) -> np.ndarray:
    lib = load()
    b = np.zeros(3)
    _check(lib, ctx, lib.md_get_box(ctx, int(system), _ptr(b)))
    return b


def md_fastmath_eval(fn: int, x) -> np.ndarray:
    """The pair passes' fp64 routines evaluated on the GPU: all-fp64 exp (fn 0) and log
    (fn 1), reciprocal (fn 2), reciprocal square root (fn 3), the exp (fn 4) and log (fn 5)
    whose correction polynomial runs as float pairs, the reciprocal (fn 6) and reciprocal
    square root (fn 7) that finish in float pairs, and the all-fp32 float-pair exp (fn 8) and
    log (fn 9) (input split to a float pair, result summed back to a double)."""
    lib = load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    st = lib.md_fastmath_eval(int(fn), x.size, _ptr(x), _ptr(y))
    if st != 0:
        raise MDError(st, "md_fastmath_eval failed")
    return y


def md_peak_flops(precision: int, iters: int, repeats: int = 3):
    """(TFLOP/s, ms) of the FMA-chain peak kernel in fp64 (MD_FP64) or fp32 (MD_MIXED)."""
    lib = load()
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    st = lib.md_peak_flops(int(precision), int(iters), int(repeats), ctypes.byref(tf), ctypes.byref(ms))
    if st != 0:
        raise MDError(st, "md_peak_flops failed")
    return tf.value, ms.value


def md_get_stats(ctx) -> md_stats:
    lib = load()
    s = md_stats()
    _check(lib, ctx, lib.md_get_stats(ctx, ctypes.byref(s)))
    return s


def md_set_graph_mode(ctx, use_graphs: bool):
    lib = load()
    _check(lib, ctx, lib.md_set_graph_mode(ctx, 1 if use_graphs else 0))


def md_set_profiling(ctx, enable: bool):
    lib = load()
    _check(lib, ctx, lib.md_set_profiling(ctx, 1 if enable else 0))


def md_kernel_times(ctx):
    lib = load()
    k = 8
    names = (ctypes.c_char_p * k)()
    n = (ctypes.c_int64 * k)()
    ms = (ctypes.c_double * k)()
    nout = ctypes.c_int()
    _check(lib, ctx, lib.md_kernel_times(ctx, k, names, n, ms, ctypes.byref(nout)))
    return {names[i].decode(): (int(n[i]), float(ms[i])) for i in range(nout.value)}


def md_autotune(ctx, repeats: int = 0) -> md_tuning:
    lib = load()
    t = md_tuning()
    _check(lib, ctx, lib.md_autotune(ctx, int(repeats), ctypes.byref(t)))
    return t


def md_set_tuning(ctx, pair_block: int = 0, pool_blocks_per_sm: int = 16, pair_cap: int = 0):
    lib = load()
    t = md_tuning()
    t.pair_block, t.pool_blocks_per_sm, t.pair_cap = int(pair_block), int(pool_blocks_per_sm), int(pair_cap)
    _check(lib, ctx, lib.md_set_tuning(ctx, ctypes.byref(t)))


def md_get_tuning(ctx) -> md_tuning:
    lib = load()
    t = md_tuning()
    _check(lib, ctx, lib.md_get_tuning(ctx, ctypes.byref(t)))
    return t


def tuning_dict(t: md_tuning) -> dict:
    """The chosen launch parameters and every timed candidate, as plain data."""
    return {"pair_block": t.pair_block, "pool_blocks_per_sm": t.pool_blocks_per_sm, "pair_cap": t.pair_cap,
            "tried": [{"pair_block": t.tried_pair_block[k], "pool_blocks_per_sm": t.tried_blocks_per_sm[k],
                       "pair_cap": t.tried_pair_cap[k], "ms": t.tried_ms[k]} for k in range(t.n_tried)]}


def md_batch_create(atom_capacity, max_systems, kind, param_sets, masses_by_type,
                    opt: md_options | None = None, max_box=0.0, cell_capacity=0):
    lib = load()
    arrs = [np.ascontiguousarray(p, dtype=np.float64) for p in param_sets]
    sets = (md_params * len(arrs))(*[md_params(int(kind), 1, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
                                      for a in arrs])
    masses = np.ascontiguousarray(masses_by_type, dtype=np.float64)
    bo = md_batch_options(float(max_box), int(cell_capacity))
    ctx = ctypes.c_void_p()
    st = lib.md_batch_create(ctypes.byref(ctx), int(atom_capacity), int(max_systems), len(arrs), sets,
                             len(masses), _ptr(masses), ctypes.byref(bo),
                             ctypes.byref(opt) if opt is not None else None)
    if st != MD_OK:
        raise MDError(st, "md_batch_create failed")
    return ctx


def md_batch_add(ctx, system: md_system) -> int:
    lib = load()
    out = ctypes.c_int(-1)
    _check(lib, ctx, lib.md_batch_add(ctx, ctypes.byref(system), ctypes.byref(out)))
    return out.value


def md_batch_remove(ctx, sys_id):
    lib = load()
    _check(lib, ctx, lib.md_batch_remove(ctx, int(sys_id)))


def md_batch_status(ctx, max_systems):
    lib = load()
    active = np.zeros(max_systems, dtype=np.int32)
    left = np.zeros(max_systems, dtype=np.int64)
    tot = np.zeros((max_systems, 13))
    kin = np.zeros(max_systems)
    _check(lib, ctx, lib.md_batch_status(ctx, _ptr(active), _ptr(left), _ptr(tot), _ptr(kin)))
    return active, left, tot, kin


def md_batch_errors(ctx, max_systems) -> np.ndarray:
    """Per-slot md_status of systems that failed on the device (0: none)."""
    lib = load()
    st = np.zeros(max_systems, dtype=np.int32)
    _check(lib, ctx, lib.md_batch_errors(ctx, _ptr(st)))
    return st


def md_batch_get_state(ctx, sys_id, x=None, v=None):
    lib = load()
    _check(lib, ctx, lib.md_batch_get_state(ctx, int(sys_id), _ptr(x), _ptr(v)))


def md_server_create(opt: md_server_options, tersoff_sets=None, tersoff_masses=None, sw_set=None, sw_mass=None):
    lib = load()
    keep = []

    def sets(arrs, kind):
        if arrs is None:
            return None
        a = [np.ascontiguousarray(p, dtype=np.float64) for p in arrs]
        keep.extend(a)
        return (md_params * len(a))(*[md_params(kind, 1, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) for x in a])

    ts = sets(tersoff_sets, MD_TERSOFF)
    ss = sets(sw_set, MD_SW)
    tm = None if tersoff_masses is None else np.ascontiguousarray(tersoff_masses, dtype=np.float64)
    sm = None if sw_mass is None else np.ascontiguousarray(sw_mass, dtype=np.float64)
    srv = ctypes.c_void_p()
    st = lib.md_server_create(ctypes.byref(srv), ctypes.byref(opt), ts, _ptr(tm), ss, _ptr(sm))
    if st != MD_OK:
        raise MDError(st, "md_server_create failed")
    return srv


def md_server_submit(srv, job: md_job) -> int:
    lib = load()
    jid = ctypes.c_int64()
    st = lib.md_server_submit(srv, ctypes.byref(job), ctypes.byref(jid))
    if st != MD_OK:
        raise MDError(st, "md_server_submit failed")
    return jid.value


def md_server_poll(srv, job_id) -> md_job_result:
    r = md_job_result()
    st = load().md_server_poll(srv, int(job_id), ctypes.byref(r))
    if st != MD_OK:
        raise MDError(st, "md_server_poll failed")
    return r


def md_server_wait(srv, job_id) -> md_job_result:
    r = md_job_result()
    st = load().md_server_wait(srv, int(job_id), ctypes.byref(r))
    if st != MD_OK:
        raise MDError(st, "md_server_wait failed")
    return r


def md_server_wait_timeout(srv, job_id, timeout_s):
    """(status, result): status MD_OK when the job finished within timeout_s seconds,
    MD_ERR_TIMEOUT when it had not (the job keeps running)."""
    r = md_job_result()
    st = load().md_server_wait_timeout(srv, int(job_id), float(timeout_s), ctypes.byref(r))
    if st not in (MD_OK, MD_ERR_TIMEOUT):
        raise MDError(st, "md_server_wait_timeout failed")
    return st, r


def md_server_drain(srv):
    st = load().md_server_drain(srv)
    if st != MD_OK:
        raise MDError(st, "md_server_drain failed")


def md_server_stats_get(srv) -> md_server_stats:
    s = md_server_stats()
    load().md_server_stats_get(srv, ctypes.byref(s))
    return s


def md_server_clock(srv) -> float:
    return load().md_server_clock(srv)


def md_server_destroy(srv):
    if srv:
        load().md_server_destroy(srv)


def _check_device_f64(name, t, count):
    """t must be None or a contiguous float64 CUDA tensor of at least `count` elements:
    the library reads and writes it as raw device memory."""
    if t is None:
        return
    if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: a CUDA tensor is required")
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous float64 tensor is required")
    if t.numel() < count:
        raise ValueError(f"{name}: {t.numel()} elements, at least {count} required")


def md_compute_static(kind, params, precision, box, pbc, n_atoms, x, y, z, vx, vy, vz, mass,
                      f=None, u=None, w=None, j=None, totals=None, stream=None):
    """Allocation-free force evaluation (torch CUDA tensors in and out; totals a host
    float64 array of 13, or None)."""
    lib = load()
    if totals is not None and not (isinstance(totals, np.ndarray) and totals.dtype == np.float64
                                   and totals.flags["C_CONTIGUOUS"] and totals.size >= 13):
        raise ValueError("totals: a contiguous host float64 array of at least 13 elements is required")
    n = int(n_atoms)
    for name, t, c in (("x", x, n), ("y", y, n), ("z", z, n), ("vx", vx, n), ("vy", vy, n), ("vz", vz, n),
                       ("f", f, 3 * n), ("u", u, n), ("w", w, 9 * n), ("j", j, 3 * n)):
        if name in ("x", "y", "z") and t is None:
            raise ValueError(f"{name}: positions are required")
        _check_device_f64(name, t, c)
    prm = np.ascontiguousarray(params, dtype=np.float64)
    b = np.ascontiguousarray(box, dtype=np.float64)
    pb = np.ascontiguousarray(pbc, dtype=np.int32)
    st = lib.md_compute_static(int(kind), _ptr(prm), int(precision), _ptr(b), _ptr(pb), int(n_atoms),
                               _ptr(x), _ptr(y), _ptr(z), _ptr(vx), _ptr(vy), _ptr(vz), float(mass),
                               _ptr(f), _ptr(u), _ptr(w), _ptr(j), _ptr(totals), stream)
    if st != MD_OK:
        raise MDError(st, "md_compute_static failed")


def md_hcacf(j, n_rows, row_stride, n_lags, dt_fs=0.0, volume=0.0, temperature=0.0, acf=None, kappa=None,
             io=MD_IO_HOST, stream=None):
    """Raw call: j, acf, kappa are numpy arrays (io=MD_IO_HOST) or torch CUDA tensors
    (io=MD_IO_DEVICE); j points at the first J_x of the layout md_hcacf documents."""
    lib = load()
    st = lib.md_hcacf(_ptr(j), int(n_rows), int(row_stride), int(n_lags), float(dt_fs), float(volume),
                      float(temperature), _ptr(acf), _ptr(kappa), int(io), stream)
    if st != MD_OK:
        raise MDError(st, "md_hcacf")


def green_kubo(series, n_lags, dt_fs=0.0, volume=0.0, temperature=0.0, system=0):
    """HCACF (n_lags, 3) and running kappa (n_lags, 3) of one system from md_run's series:
    a (steps, 5) array (one system) or (steps, n_systems, 5) (a pool)."""
    s = np.ascontiguousarray(series, dtype=np.float64)
    rows = s.shape[0]
    flat = s.reshape(rows, -1)
    stride = flat.shape[1]
    j = flat.reshape(-1)[5 * int(system) + 2:]
    acf = np.zeros((n_lags, 3))
    kappa = np.zeros((n_lags, 3)) if temperature > 0 else None
    md_hcacf(j, rows, stride, n_lags, dt_fs, volume, temperature, acf, kappa)
    return acf, kappa


def md_last_error(ctx) -> str:
    return load().md_last_error(ctx).decode()


def md_destroy(ctx):
    if ctx:
        load().md_destroy(ctx)


# ----------------------------------------------------------------- convenience
class System:
    """One context with host (numpy) I/O, or device (torch CUDA tensor) I/O when
    io=MD_IO_DEVICE.  Arrays are (N,3) row-major on the Python side and SoA in the
    library; the transposes below are the marshalling."""

    def __init__(self, box, pbc, n_atoms, kind, params, mass, precision=MD_FP64, skin=0.0,
                 max_neigh=32, max_active=0, io=MD_IO_HOST, stream=None, hbm_budget=0, types=None, n_types=1):
        self.n = int(n_atoms)
        self.io = io
        opt = md_default_options()
        opt.precision = precision
        opt.skin = skin
        opt.max_neigh = max_neigh
        opt.max_active = max_active
        opt.io = io
        opt.cuda_stream = stream
        opt.hbm_budget = hbm_budget
        t = np.zeros(self.n, np.int32) if types is None else np.asarray(types, dtype=np.int32)
        masses = [float(m) for m in mass] if np.ndim(mass) else [float(mass)]
        self.ctx = md_create(box, pbc, self.n, t, masses, kind, params, opt, n_types=n_types)

    def close(self):
        if self.ctx:
            md_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # host <-> SoA helpers
    @staticmethod
    def _soa(a):
        a = np.asarray(a, dtype=np.float64)
        return np.ascontiguousarray(a.T)

    @staticmethod
    def _device_soa(a):
        # the library runs on its own stream: make torch's producer work visible first
        import torch
        t = a.t().contiguous()
        torch.cuda.current_stream().synchronize()
        return t

    def set_positions(self, pos):
        if self.io == MD_IO_DEVICE:
            t = self._device_soa(pos)
            md_set_positions(self.ctx, t[0], t[1], t[2])
        else:
            s = self._soa(pos)
            md_set_positions(self.ctx, s[0], s[1], s[2])

    def set_velocities(self, vel):
        if self.io == MD_IO_DEVICE:
            t = self._device_soa(vel)
            md_set_velocities(self.ctx, t[0], t[1], t[2])
        else:
            s = self._soa(vel)
            md_set_velocities(self.ctx, s[0], s[1], s[2])

    def compute(self, want=("f", "u", "w", "j")):
        n = self.n
        if self.io == MD_IO_DEVICE:
            import torch
            mk = lambda c: torch.empty(c * max(n, 1), dtype=torch.float64, device="cuda")
        else:
            mk = lambda c: np.empty(c * max(n, 1), dtype=np.float64)
        f = mk(3) if "f" in want else None
        u = mk(1) if "u" in want else None
        w = mk(9) if "w" in want else None
        j = mk(3) if "j" in want else None
        tot = np.zeros(13)
        md_compute(self.ctx, f, u, w, j, tot)
        out = {"totals": tot}
        if f is not None:
            out["F"] = f[:3 * n].reshape(3, n).T
        if u is not None:
            out["U"] = u[:n]
        if w is not None:
            out["W"] = w[:9 * n].reshape(9, n).T
        if j is not None:
            out["J"] = j[:3 * n].reshape(3, n).T
        return out

    def run(self, n_steps, dt, record=True):
        series = np.zeros((max(n_steps, 1), 5)) if record else None
        md_run(self.ctx, n_steps, dt, series)
        return series[:n_steps] if record else None

    def state(self):
        x = np.empty(3 * max(self.n, 1))
        v = np.empty(3 * max(self.n, 1))
        md_get_state(self.ctx, x, v)
        n = self.n
        return x[:3 * n].reshape(3, n).T.copy(), v[:3 * n].reshape(3, n).T.copy()

    def stats(self):
        return md_get_stats(self.ctx)

    def checkpoint(self) -> np.ndarray:
        return md_checkpoint_save(self.ctx)

    def restore(self, image):
        md_checkpoint_load(self.ctx, image)

    def set_npt(self, off=False, **kw):
        md_set_npt(self.ctx, 0, off=off, **kw)

    def box(self):
        return md_get_box(self.ctx, 0)


def multi_params(element_rows, chi):
    """Packed multi-element Tersoff parameters: the element rows, then chi row-major."""
    rows = np.asarray(element_rows, dtype=np.float64).reshape(-1, 11)
    return np.concatenate([rows.reshape(-1), np.asarray(chi, dtype=np.float64).reshape(-1)])


def from_multi(msys, precision=MD_FP64, **kw) -> System:
    """Context for an inputs.MultiSystem (multi-element Tersoff), positions and velocities
    uploaded."""
    nt = len(msys.params)
    s = System(msys.box, msys.pbc, msys.n, MD_TERSOFF, multi_params(msys.params, msys.chi), list(msys.masses),
               precision=precision, types=msys.types, n_types=nt, **kw)
    s.set_positions(msys.pos)
    if msys.vel is not None:
        s.set_velocities(msys.vel)
    return s


def from_inputs(sysm, precision=MD_FP64, **kw) -> System:
    """Context for an inputs.System, with its positions and velocities uploaded."""
    s = System(sysm.box, sysm.pbc, sysm.n, sysm.kind, sysm.params, sysm.mass, precision=precision, **kw)
    s.set_positions(sysm.pos)
    if sysm.vel is not None:
        s.set_velocities(sysm.vel)
    return s


class Pool:
    """A pool context (many systems stepped together) with host I/O."""

    def __init__(self, atom_capacity, max_systems, kind, param_sets, masses_by_type, precision=MD_FP64,
                 skin=0.0, max_neigh=32, max_active=0, stream=None, max_box=0.0, cell_capacity=0):
        opt = md_default_options()
        opt.precision = precision
        opt.skin = skin
        opt.max_neigh = max_neigh
        opt.max_active = max_active
        opt.cuda_stream = stream
        self.max_systems = int(max_systems)
        self.ctx = md_batch_create(atom_capacity, max_systems, kind, param_sets, masses_by_type, opt,
                                   max_box, cell_capacity)
        self.n_atoms = {}

    def add(self, pos, vel, box, pbc, param_set=0, types=None, n_steps=-1, damp=0.0) -> int:
        pos = np.asarray(pos, dtype=np.float64)
        n = pos.shape[0]
        soa = np.ascontiguousarray(pos.T)
        v = np.ascontiguousarray(np.zeros_like(pos).T if vel is None else np.asarray(vel, dtype=np.float64).T)
        t = np.ascontiguousarray(np.zeros(n, np.int32) if types is None else types, dtype=np.int32)
        sd = md_system()
        sd.box = (ctypes.c_double * 3)(*[float(b) for b in box])
        sd.pbc = (ctypes.c_int * 3)(*[int(b) for b in pbc])
        sd.n_atoms = n
        sd.types = t.ctypes.data
        sd.param_set = int(param_set)
        sd.x, sd.y, sd.z = soa[0].ctypes.data, soa[1].ctypes.data, soa[2].ctypes.data
        sd.vx, sd.vy, sd.vz = v[0].ctypes.data, v[1].ctypes.data, v[2].ctypes.data
        sd.n_steps = int(n_steps)
        sd.damp = float(damp)
        sid = md_batch_add(self.ctx, sd)
        self.n_atoms[sid] = n
        return sid

    def remove(self, sid):
        md_batch_remove(self.ctx, sid)
        self.n_atoms.pop(sid, None)

    def set_npt(self, sid, off=False, **kw):
        md_set_npt(self.ctx, sid, off=off, **kw)

    def box(self, sid):
        return md_get_box(self.ctx, sid)

    def run(self, n_steps, dt, record=False):
        series = np.zeros((max(n_steps, 1), self.max_systems, 5)) if record else None
        md_run(self.ctx, n_steps, dt, series)
        return series[:n_steps] if record else None

    def status(self):
        return md_batch_status(self.ctx, self.max_systems)

    def errors(self):
        return md_batch_errors(self.ctx, self.max_systems)

    def state(self, sid):
        n = self.n_atoms[sid]
        x = np.empty(3 * n)
        v = np.empty(3 * n)
        md_batch_get_state(self.ctx, sid, x, v)
        return x.reshape(3, n).T.copy(), v.reshape(3, n).T.copy()

    def close(self):
        if self.ctx:
            md_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (md_server_*) with host I/O."""

    def __init__(self, precision=MD_MIXED, tersoff_atoms=0, sw_atoms=0, max_jobs_per_pool=512,
                 tersoff_dt=0.5, sw_dt=1.0, chunk_steps=8, tersoff_sets=None, tersoff_masses=None,
                 sw_set=None, sw_mass=None):
        opt = md_server_options(int(precision), int(tersoff_atoms), int(sw_atoms), int(max_jobs_per_pool),
                                float(tersoff_dt), float(sw_dt), int(chunk_steps), 0)
        self.srv = md_server_create(opt, tersoff_sets, tersoff_masses, sw_set, sw_mass)
        self._keep = {}

    def submit(self, kind, pos, vel, box, pbc, n_steps, param_set=0, types=None, damp=0.0, want_state=True):
        pos = np.asarray(pos, dtype=np.float64)
        n = pos.shape[0]
        soa = np.ascontiguousarray(pos.T)
        v = np.ascontiguousarray(np.zeros_like(pos).T if vel is None else np.asarray(vel, dtype=np.float64).T)
        t = np.ascontiguousarray(np.zeros(n, np.int32) if types is None else types, dtype=np.int32)
        xo = np.empty(3 * n) if want_state else None
        vo = np.empty(3 * n) if want_state else None
        j = md_job()
        j.kind, j.param_set = int(kind), int(param_set)
        j.box = (ctypes.c_double * 3)(*[float(b) for b in box])
        j.pbc = (ctypes.c_int * 3)(*[int(b) for b in pbc])
        j.n_atoms, j.types = n, t.ctypes.data
        j.x, j.y, j.z = soa[0].ctypes.data, soa[1].ctypes.data, soa[2].ctypes.data
        j.vx, j.vy, j.vz = v[0].ctypes.data, v[1].ctypes.data, v[2].ctypes.data
        j.n_steps, j.damp = int(n_steps), float(damp)
        j.x_out = None if xo is None else xo.ctypes.data
        j.v_out = None if vo is None else vo.ctypes.data
        jid = md_server_submit(self.srv, j)
        self._keep[jid] = (xo, vo, n)
        return jid

    def wait(self, jid):
        r = md_server_wait(self.srv, jid)
        xo, vo, n = self._keep.pop(jid)
        state = None if xo is None else (xo.reshape(3, n).T.copy(), vo.reshape(3, n).T.copy())
        return r, state

    def drain(self):
        md_server_drain(self.srv)

    def stats(self):
        return md_server_stats_get(self.srv)

    def clock(self):
        return md_server_clock(self.srv)

    def close(self):
        if self.srv:
            md_server_destroy(self.srv)
            self.srv = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- spatial decomposition
def _dcheck(lib, dom, status):
    if status != MD_OK:
        raise MDError(status, lib.md_domain_last_error(dom).decode() if dom else "")


def md_domain_create(box, pbc, axis, n_ranks, rank, capacity, kind, params, mass, opt: md_options | None = None):
    lib = load()
    box = np.ascontiguousarray(box, dtype=np.float64)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32)
    prm_arr = np.ascontiguousarray(params, dtype=np.float64)
    prm = md_params(int(kind), 1, prm_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    masses = np.ascontiguousarray([float(mass)], dtype=np.float64)
    dom = ctypes.c_void_p()
    st = lib.md_domain_create(ctypes.byref(dom), _ptr(box), _ptr(pbc), int(axis), int(n_ranks), int(rank),
                              int(capacity), ctypes.byref(prm), _ptr(masses),
                              ctypes.byref(opt) if opt is not None else None)
    if st != MD_OK:
        raise MDError(st, "md_domain_create failed")
    return dom


def md_domain_set_atoms(dom, ids, types, x, y, z, vx=None, vy=None, vz=None):
    lib = load()
    _dcheck(lib, dom, lib.md_domain_set_atoms(dom, len(ids), _ptr(ids), _ptr(types), _ptr(x), _ptr(y), _ptr(z),
                                              _ptr(vx), _ptr(vy), _ptr(vz)))


def md_domain_message_bound(dom, mode) -> int:
    lib = load()
    n = ctypes.c_size_t()
    _dcheck(lib, dom, lib.md_domain_message_bound(dom, int(mode), ctypes.byref(n)))
    return n.value


def md_domain_pack(dom, mode):
    """(to_left, to_right) byte arrays of kind `mode`."""
    lib = load()
    cap = md_domain_message_bound(dom, mode)
    bl = np.empty(cap, dtype=np.uint8)
    br = np.empty(cap, dtype=np.uint8)
    nl, nr = ctypes.c_size_t(), ctypes.c_size_t()
    _dcheck(lib, dom, lib.md_domain_pack(dom, int(mode), _ptr(bl), _ptr(br), cap, ctypes.byref(nl), ctypes.byref(nr)))
    return bl[: nl.value], br[: nr.value]


def md_domain_unpack(dom, mode, from_left, from_right):
    lib = load()
    fl = np.ascontiguousarray(from_left, dtype=np.uint8)
    fr = np.ascontiguousarray(from_right, dtype=np.uint8)
    _dcheck(lib, dom, lib.md_domain_unpack(dom, int(mode), _ptr(fl), fl.size, _ptr(fr), fr.size))


def md_domain_kick_drift(dom, dt) -> bool:
    lib = load()
    r = ctypes.c_int()
    _dcheck(lib, dom, lib.md_domain_kick_drift(dom, float(dt), ctypes.byref(r)))
    return bool(r.value)


def md_domain_force(dom, dt) -> np.ndarray:
    lib = load()
    t = np.zeros(5)
    _dcheck(lib, dom, lib.md_domain_force(dom, float(dt), _ptr(t)))
    return t


def md_domain_owned(dom):
    """(ids, x (n,3), v (n,3)) of the owned atoms."""
    lib = load()
    n = ctypes.c_int64()
    _dcheck(lib, dom, lib.md_domain_owned(dom, ctypes.byref(n), None, None, None))
    k = n.value
    ids = np.empty(max(k, 1), dtype=np.int64)
    x = np.empty(3 * max(k, 1))
    v = np.empty(3 * max(k, 1))
    _dcheck(lib, dom, lib.md_domain_owned(dom, ctypes.byref(n), _ptr(ids), _ptr(x), _ptr(v)))
    return ids[:k].copy(), x[: 3 * k].reshape(3, k).T.copy(), v[: 3 * k].reshape(3, k).T.copy()


def md_domain_compute(dom):
    """Per-atom F, U, W, J of the owned atoms (md_domain_owned's order) and the rank's totals."""
    lib = load()
    n = ctypes.c_int64()
    _dcheck(lib, dom, lib.md_domain_owned(dom, ctypes.byref(n), None, None, None))
    k = n.value
    mk = lambda c: np.empty(c * max(k, 1))
    f, u, w, j, tot = mk(3), mk(1), mk(9), mk(3), np.zeros(13)
    _dcheck(lib, dom, lib.md_domain_compute(dom, _ptr(f), _ptr(u), _ptr(w), _ptr(j), _ptr(tot)))
    return {"F": f[: 3 * k].reshape(3, k).T.copy(), "U": u[:k].copy(), "W": w[: 9 * k].reshape(9, k).T.copy(),
            "J": j[: 3 * k].reshape(3, k).T.copy(), "totals": tot}


def md_domain_last_error(dom) -> str:
    return load().md_domain_last_error(dom).decode()


def md_domain_destroy(dom):
    if dom:
        load().md_domain_destroy(dom)


def domain_route(outboxes):
    """Messages between slab ranks: outboxes[r] = (to_left, to_right) of rank r; returns
    inboxes[r] = (from_left, from_right), where from_left is what rank r - 1 sent right and
    from_right what rank r + 1 sent left (indices mod the rank count)."""
    n = len(outboxes)
    return [(outboxes[(r - 1) % n][1], outboxes[(r + 1) % n][0]) for r in range(n)]


class DomainGroup:
    """Every rank of a slab decomposition held in one process (one GPU), the messages routed
    in memory: each phase runs for all ranks before the next, so no rank waits for another
    inside a kernel.  For tests and single-GPU use of the decomposed path."""

    def __init__(self, box, pbc, axis, n_ranks, capacity, kind, params, mass, precision=MD_FP64, skin=0.0):
        opt = md_default_options()
        opt.precision = precision
        opt.skin = skin
        self.n = int(n_ranks)
        self.doms = [md_domain_create(box, pbc, axis, n_ranks, r, capacity, kind, params, mass, opt)
                     for r in range(self.n)]
        self.rebuilds = 0

    def close(self):
        for d in self.doms:
            md_domain_destroy(d)
        self.doms = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def exchange(self, mode):
        inbox = domain_route([md_domain_pack(d, mode) for d in self.doms])
        for d, (fl, fr) in zip(self.doms, inbox):
            md_domain_unpack(d, mode, fl, fr)

    def start(self, pos, vel, ids=None):
        """All atoms of the system (every rank keeps its slab's), ghosts, first forces."""
        pos = np.asarray(pos, dtype=np.float64)
        n = pos.shape[0]
        ids = np.arange(n, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
        soa = np.ascontiguousarray(pos.T)
        v = np.ascontiguousarray(np.asarray(vel, dtype=np.float64).T)
        ty = np.zeros(n, dtype=np.int32)
        for d in self.doms:
            md_domain_set_atoms(d, ids, ty, soa[0], soa[1], soa[2], v[0], v[1], v[2])
        self.exchange(MD_DOMAIN_GHOSTS)
        return sum(md_domain_force(d, 0.0) for d in self.doms)

    def step(self, dt):
        """One velocity-Verlet step on every rank; the system's U, K, Jx, Jy, Jz."""
        if any([md_domain_kick_drift(d, dt) for d in self.doms]):
            self.exchange(MD_DOMAIN_MIGRATE)
            self.exchange(MD_DOMAIN_GHOSTS)
            self.rebuilds += 1
        else:
            self.exchange(MD_DOMAIN_POSITIONS)
        tot = np.zeros(5)
        for d in self.doms:     # rank order: a fixed summation order
            tot += md_domain_force(d, dt)
        return tot

    def run(self, n_steps, dt):
        return np.array([self.step(dt) for _ in range(n_steps)])

    def state(self, n_atoms):
        """Positions and velocities (n_atoms, 3) by atom id, gathered from the ranks."""
        x = np.full((n_atoms, 3), np.nan)
        v = np.full((n_atoms, 3), np.nan)
        for d in self.doms:
            ids, xo, vo = md_domain_owned(d)
            x[ids] = xo
            v[ids] = vo
        return x, v

    def compute(self, n_atoms):
        out = {k: np.full((n_atoms, c), np.nan) for k, c in (("F", 3), ("U", 1), ("W", 9), ("J", 3))}
        tot = np.zeros(13)
        for d in self.doms:
            ids, _, _ = md_domain_owned(d)
            r = md_domain_compute(d)
            for k in ("F", "W", "J"):
                out[k][ids] = r[k]
            out["U"][ids, 0] = r["U"]
            tot += r["totals"]
        out["U"] = out["U"][:, 0]
        out["totals"] = tot
        return out


class DistTransport:
    """Messages between the ranks of a torch.distributed process group (gloo: host memory;
    the library's messages are host buffers), one rank per process."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.n = dist.get_world_size(group)

    def exchange(self, mode, to_left, to_right):
        """(from_left, from_right): the left neighbour's right-going message and the right
        neighbour's left-going one; sizes first, then the bytes (tags keep the two directions
        apart when both neighbours are the same rank)."""
        import torch
        dist = self.dist
        left, right = (self.rank - 1) % self.n, (self.rank + 1) % self.n
        tl, tr = 100 + 4 * mode, 101 + 4 * mode       # sent left / sent right
        sizes = [torch.tensor([len(to_left)], dtype=torch.int64), torch.tensor([len(to_right)], dtype=torch.int64)]
        got = [torch.zeros(1, dtype=torch.int64), torch.zeros(1, dtype=torch.int64)]
        reqs = [dist.isend(sizes[0], left, group=self.group, tag=tl),
                dist.isend(sizes[1], right, group=self.group, tag=tr),
                dist.irecv(got[0], left, group=self.group, tag=tr),
                dist.irecv(got[1], right, group=self.group, tag=tl)]
        for q in reqs:
            q.wait()
        out = [torch.from_numpy(np.ascontiguousarray(to_left)), torch.from_numpy(np.ascontiguousarray(to_right))]
        inb = [torch.empty(int(got[0].item()), dtype=torch.uint8), torch.empty(int(got[1].item()), dtype=torch.uint8)]
        reqs = [dist.isend(out[0], left, group=self.group, tag=tl + 2),
                dist.isend(out[1], right, group=self.group, tag=tr + 2),
                dist.irecv(inb[0], left, group=self.group, tag=tr + 2),
                dist.irecv(inb[1], right, group=self.group, tag=tl + 2)]
        for q in reqs:
            q.wait()
        return inb[0].numpy(), inb[1].numpy()

    def any(self, flag):
        import torch
        t = torch.tensor([1 if flag else 0], dtype=torch.int64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return bool(t.item())

    def sum(self, values):
        """Sum over the ranks in rank order (gathered, then added on every rank)."""
        import torch
        t = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64))
        parts = [torch.zeros_like(t) for _ in range(self.n)]
        self.dist.all_gather(parts, t, group=self.group)
        acc = np.zeros_like(np.asarray(values, dtype=np.float64))
        for q in parts:
            acc = acc + q.numpy()
        return acc


class Domain:
    """This process's rank of a slab decomposition, its messages carried by `transport`
    (DistTransport, or any object with the same exchange / any / sum methods)."""

    def __init__(self, transport, box, pbc, axis, capacity, kind, params, mass, precision=MD_FP64, skin=0.0):
        opt = md_default_options()
        opt.precision = precision
        opt.skin = skin
        self.t = transport
        self.dom = md_domain_create(box, pbc, axis, transport.n, transport.rank, capacity, kind, params, mass, opt)
        self.rebuilds = 0

    def close(self):
        md_domain_destroy(self.dom)
        self.dom = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def exchange(self, mode):
        to_l, to_r = md_domain_pack(self.dom, mode)
        fl, fr = self.t.exchange(mode, to_l, to_r)
        md_domain_unpack(self.dom, mode, fl, fr)

    def start(self, pos, vel, ids=None):
        pos = np.asarray(pos, dtype=np.float64)
        n = pos.shape[0]
        ids = np.arange(n, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64)
        soa = np.ascontiguousarray(pos.T)
        v = np.ascontiguousarray(np.asarray(vel, dtype=np.float64).T)
        md_domain_set_atoms(self.dom, ids, np.zeros(n, dtype=np.int32), soa[0], soa[1], soa[2], v[0], v[1], v[2])
        self.exchange(MD_DOMAIN_GHOSTS)
        return self.t.sum(md_domain_force(self.dom, 0.0))

    def step(self, dt):
        if self.t.any(md_domain_kick_drift(self.dom, dt)):
            self.exchange(MD_DOMAIN_MIGRATE)
            self.exchange(MD_DOMAIN_GHOSTS)
            self.rebuilds += 1
        else:
            self.exchange(MD_DOMAIN_POSITIONS)
        return self.t.sum(md_domain_force(self.dom, dt))

    def run(self, n_steps, dt):
        return np.array([self.step(dt) for _ in range(n_steps)])

    def owned(self):
        return md_domain_owned(self.dom)
