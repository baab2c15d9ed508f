"""md_compute_static: the force evaluation for callers that cannot allocate device
memory (it uses one fixed, file-scope scratch array instead).  Checked through the C
ABI against md_compute, the context-based entry point, on two calls in a row (the
second call reuses the array the first one left behind), in both precisions, and with
the force and energy outputs left out (they then live in the scratch array).  This file
is collected last so that a stopping failure here comes after every other test has run."""
import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12        # the fp64 parity bound of the other GPU tests
MIXED_TOL = 1e-5   # the mixed-precision force bound of the other GPU tests


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max())


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03343_gb300 import _build, md as M
    _build.build()
    M.load()
    return M


def static_eval(md, s, precision=0, outputs=("f", "u", "w", "j")):
    import torch
    n = s.n
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, y, z = dev(s.pos[:, 0]), dev(s.pos[:, 1]), dev(s.pos[:, 2])
    vx, vy, vz = dev(s.vel[:, 0]), dev(s.vel[:, 1]), dev(s.vel[:, 2])
    mk = lambda c, k: torch.empty(c * n, dtype=torch.float64, device="cuda") if k in outputs else None
    f, u, w, j = mk(3, "f"), mk(1, "u"), mk(9, "w"), mk(3, "j")
    tot = np.zeros(13)
    torch.cuda.synchronize()
    md.md_compute_static(s.kind, s.params, precision, s.box, s.pbc, n, x, y, z, vx, vy, vz, s.mass,
                         f, u, w, j, tot)
    out = {"totals": tot}
    for key, t, c in (("F", f, 3), ("U", u, 1), ("W", w, 9), ("J", j, 3)):
        if t is not None:
            a = t.cpu().numpy()
            out[key] = a if c == 1 else a.reshape(c, n).T
    return out


CASES = [lambda: I.si_diamond_tersoff(n=6), lambda: I.si_diamond_sw(n=5, jitter_amp=0.08)]
IDS = ["tersoff_si_1728", "sw_si_1000"]


@pytest.mark.parametrize("make", CASES, ids=IDS)
def test_static_entry_point_matches_md_compute_twice(md, make):
    s = make()
    with md.from_inputs(s) as g:
        ref = g.compute()
    for _ in range(2):
        out = static_eval(md, s)
        for k in ("F", "U", "W", "J", "totals"):
            assert rel(out[k], ref[k]) < TOL, k


@pytest.mark.parametrize("make", CASES, ids=IDS)
def test_static_entry_point_mixed_precision(md, make):
    """MD_MIXED: the same fp32 pair arithmetic as md_compute in mixed precision, and the
    forces within the mixed bound of the fp64 oracle; two calls in a row."""
    s = make()
    with md.from_inputs(s, precision=md.MD_MIXED) as g:
        ref = g.compute()
    orc = O.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
    for _ in range(2):
        out = static_eval(md, s, precision=md.MD_MIXED)
        for k in ("F", "U", "W", "J", "totals"):
            assert rel(out[k], ref[k]) < MIXED_TOL, k
        assert rel(out["F"], orc["F"]) < MIXED_TOL


def test_static_entry_point_totals_only(md):
    """f and u NULL: force and energy live in the scratch array; the totals still match."""
    s = I.si_diamond_tersoff(n=5, jitter_amp=0.1, seed_pos=3)
    with md.from_inputs(s) as g:
        ref = g.compute()
    for _ in range(2):
        out = static_eval(md, s, outputs=())
        assert rel(out["totals"], ref["totals"]) < TOL


def test_static_entry_point_rejects_too_many_atoms(md):
    s = I.si_diamond_tersoff(n=12)    # 13,824 atoms > the static maximum
    with pytest.raises(md.MDError) as e:
        static_eval(md, s)
    assert e.value.status == -4
