"""The C-ABI library builds, loads without a GPU, and exports every entry point that
include/md.h declares; argument checks that precede any CUDA call work on the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "md.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_03343_gb300 import _build, md
    _build.build()
    return md.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("md_create", "md_set_positions", "md_set_velocities", "md_compute", "md_run",
                 "md_get_state", "md_last_error", "md_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1610_03343_gb300 import md
    for name in declared_functions():
        assert callable(getattr(md, name)), name


def test_default_options(lib):
    from paper_1610_03343_gb300 import md
    o = md.md_default_options()
    assert o.precision == md.MD_FP64 and o.max_neigh == 32 and o.io == md.MD_IO_HOST


def test_create_rejects_bad_arguments_before_touching_cuda(lib):
    from paper_1610_03343_gb300 import inputs, md
    ctx = ctypes.c_void_p()
    box = np.array([10.0, 10.0, 10.0])
    pbc = np.array([1, 1, 1], dtype=np.int32)
    prm_arr = np.array(inputs.TERSOFF_SI_1989)
    prm = md.md_params(md.MD_TERSOFF, 1, prm_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    masses = np.array([28.0855])
    # NULL box
    assert lib.md_create(ctypes.byref(ctx), None, pbc.ctypes.data, 0, None, masses.ctypes.data,
                         ctypes.byref(prm), None) == -1
    # negative atom count
    assert lib.md_create(ctypes.byref(ctx), box.ctypes.data, pbc.ctypes.data, -5, None, masses.ctypes.data,
                         ctypes.byref(prm), None) == -1
    # unknown potential kind
    bad = md.md_params(7, 1, prm_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert lib.md_create(ctypes.byref(ctx), box.ctypes.data, pbc.ctypes.data, 0, None, masses.ctypes.data,
                         ctypes.byref(bad), None) == -1
    # periodic box shorter than twice the list cutoff (3.0 + 0.45 skin)
    small = np.array([6.0, 10.0, 10.0])
    assert lib.md_create(ctypes.byref(ctx), small.ctypes.data, pbc.ctypes.data, 0, None, masses.ctypes.data,
                         ctypes.byref(prm), None) == -2
    assert not ctx.value


def test_null_context_calls_return_arg_error(lib):
    assert lib.md_run(None, 1, 1.0, None) == -1
    assert lib.md_compute(None, None, None, None, None, None) == -1
    assert lib.md_last_error(None) == b""
    lib.md_destroy(None)


def test_static_binding_rejects_host_arrays_and_short_outputs(lib):
    """md_compute_static writes through raw device pointers: the binding refuses host
    arrays, wrong dtypes and short outputs before calling the library."""
    from paper_1610_03343_gb300 import inputs, md
    s = inputs.si_diamond_tersoff(n=2)
    x = np.ascontiguousarray(s.pos[:, 0])
    with pytest.raises(ValueError, match="CUDA tensor"):
        md.md_compute_static(s.kind, s.params, md.MD_FP64, s.box, s.pbc, s.n, x, x, x, None, None, None,
                             s.mass)
    torch = pytest.importorskip("torch")
    t32 = torch.zeros(s.n, dtype=torch.float32)
    with pytest.raises(ValueError):
        md.md_compute_static(s.kind, s.params, md.MD_FP64, s.box, s.pbc, s.n, t32, t32, t32, None, None, None,
                             s.mass)
    with pytest.raises(ValueError, match="totals"):
        md.md_compute_static(s.kind, s.params, md.MD_FP64, s.box, s.pbc, s.n, None, None, None, None, None,
                             None, s.mass, totals=np.zeros(5))
