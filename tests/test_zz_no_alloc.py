"""md_compute_static: the force evaluation for callers that cannot allocate device
memory (it uses one fixed, file-scope scratch array instead).  Checked through the C
ABI against md_compute, the context-based entry point, on two calls in a row (the
second call reuses the array the first one left behind).  This file is collected last
so that a stopping failure here comes after every other test has run."""
import numpy as np
import pytest

from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the fp64 parity bound of the other GPU tests


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


def static_eval(md, s):
    import torch
    n = s.n
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, y, z = dev(s.pos[:, 0]), dev(s.pos[:, 1]), dev(s.pos[:, 2])
    vx, vy, vz = dev(s.vel[:, 0]), dev(s.vel[:, 1]), dev(s.vel[:, 2])
    f = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    w = torch.empty(9 * n, dtype=torch.float64, device="cuda")
    j = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    tot = np.zeros(13)
    torch.cuda.synchronize()
    md.md_compute_static(s.kind, s.params, md.MD_FP64, s.box, s.pbc, n, x, y, z, vx, vy, vz, s.mass,
                         f, u, w, j, tot)
    return dict(F=f.cpu().numpy().reshape(3, n).T, U=u.cpu().numpy(), W=w.cpu().numpy().reshape(9, n).T,
                J=j.cpu().numpy().reshape(3, n).T, totals=tot)


@pytest.mark.parametrize("make", [lambda: I.si_diamond_tersoff(n=6),
                                  lambda: I.si_diamond_sw(n=5, jitter_amp=0.08)],
                         ids=["tersoff_si_1728", "sw_si_1000"])
def test_static_entry_point_matches_md_compute_twice(md, make):
    s = make()
    with md.from_inputs(s) as g:
        ref = g.compute()
    for _ in range(2):
        out = static_eval(md, s)
        for k in ("F", "U", "W", "J", "totals"):
            assert rel(out[k], ref[k]) < TOL, k


def test_static_entry_point_rejects_too_many_atoms(md):
    s = I.si_diamond_tersoff(n=12)    # 13,824 atoms > the static maximum
    with pytest.raises(md.MDError) as e:
        static_eval(md, s)
    assert e.value.status == -4
