"""md_hcacf (CUDA) against the Green-Kubo oracle on the same series: random series,
the heat-current series of real runs (one system and a pool), host and device I/O, the
edge cases of the lag range, and argument errors."""
import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03343_gb300 import _build, md as M
    _build.build()
    M.load()
    return M


def rel(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max())


def series(T, cols=5, seed=1):
    rng = np.random.default_rng(seed)
    s = rng.normal(size=(T, cols))
    s[:, 2:5] += np.sin(np.arange(T) / 7.0)[:, None]
    return s


@pytest.mark.parametrize("T,n_lags", [(1, 1), (7, 7), (1000, 1), (1000, 250), (1000, 1000), (4099, 1531)])
def test_random_series_host(md, T, n_lags):
    s = series(T)
    acf = np.zeros((n_lags, 3))
    kap = np.zeros((n_lags, 3))
    md.md_hcacf(s.reshape(-1)[2:], T, 5, n_lags, 0.5, 2000.0, 300.0, acf, kap)
    ref = O.hcacf(s[:, 2:5], n_lags)
    assert rel(acf, ref) < TOL
    kref = O.running_kappa(ref, 0.5, 2000.0, 300.0)
    assert rel(kap, kref) < TOL if n_lags > 1 else np.all(kap == 0.0)


def test_pool_layout_and_kappa_optional(md):
    T, n_sys = 600, 7
    s = series(T, 5 * n_sys, seed=3).reshape(T, n_sys, 5)
    for sid in (0, 3, 6):
        acf, kap = md.green_kubo(s, 200, system=sid)
        assert kap is None
        assert rel(acf, O.hcacf(s[:, sid, 2:5], 200)) < TOL


def test_device_io(md):
    import torch
    T, n_lags = 2048, 512
    s = series(T, seed=4)
    dj = torch.tensor(s.reshape(-1), dtype=torch.float64, device="cuda")
    acf = torch.zeros(n_lags * 3, dtype=torch.float64, device="cuda")
    kap = torch.zeros(n_lags * 3, dtype=torch.float64, device="cuda")
    md.md_hcacf(dj[2:], T, 5, n_lags, 1.0, 5000.0, 500.0, acf, kap, io=md.MD_IO_DEVICE)
    torch.cuda.synchronize()
    ref = O.hcacf(s[:, 2:5], n_lags)
    assert rel(acf.cpu().numpy().reshape(n_lags, 3), ref) < TOL
    assert rel(kap.cpu().numpy().reshape(n_lags, 3), O.running_kappa(ref, 1.0, 5000.0, 500.0)) < TOL


def test_heat_current_series_of_a_run(md):
    s = I.c_graphene_tersoff(nx=16, ny=28, jitter_amp=0.02)
    with md.from_inputs(s) as g:
        ser = g.run(400, 0.5)
    V = float(np.prod(s.box))
    acf, kap = md.green_kubo(ser, 150, 0.5, V, 300.0)
    ref = O.hcacf(ser[:, 2:5], 150)
    assert rel(acf, ref) < TOL
    assert rel(kap, O.running_kappa(ref, 0.5, V, 300.0)) < TOL


def test_pool_series_of_a_run(md):
    mix = [(I.si_diamond_tersoff(n=3, seed_pos=3, seed_vel=4), 0),
           (I.c_graphene_tersoff(nx=6, ny=10, seed_pos=5, seed_vel=6), 1)]
    pool = md.Pool(4000, 4, I.MD_TERSOFF, [I.TERSOFF_SI_1989, I.TERSOFF_C_1989], [I.MASS_SI, I.MASS_C])
    with pool:
        ids = [pool.add(sy.pos, sy.vel, sy.box, sy.pbc, k, np.full(sy.n, k, np.int32)) for sy, k in mix]
        ser = pool.run(300, 0.5, record=True)
    for sid in ids:
        acf, _ = md.green_kubo(ser, 100, system=sid)
        assert rel(acf, O.hcacf(ser[:, sid, 2:5], 100)) < TOL


@pytest.mark.parametrize("args", [
    dict(n_rows=10, row_stride=5, n_lags=11),
    dict(n_rows=10, row_stride=5, n_lags=0),
    dict(n_rows=0, row_stride=5, n_lags=1),
    dict(n_rows=10, row_stride=2, n_lags=3),
])
def test_argument_errors(md, args):
    s = np.zeros(64)
    acf = np.zeros(64)
    with pytest.raises(md.MDError) as e:
        md.md_hcacf(s, args["n_rows"], args["row_stride"], args["n_lags"], acf=acf)
    assert e.value.status == md.MD_ERR_ARG


def test_kappa_needs_positive_state(md):
    s = np.zeros(50)
    acf = np.zeros(30)
    kap = np.zeros(30)
    with pytest.raises(md.MDError):
        md.md_hcacf(s, 10, 5, 10, 0.5, 100.0, 0.0, acf, kap)
