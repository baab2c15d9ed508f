"""The fp64 routines of the pair passes (fastmath.cuh) against numpy on the host: the
table-driven exp (Tang's method) within 2 ulp over the pair pass's domain and beyond, the
table-driven log within an absolute 2e-16 (1 + |binary exponent|) -- both the all-fp64 form and
the form whose correction polynomial runs as float pairs on the fp32 pipe -- the reciprocal within 1 ulp
(of the correctly rounded 1/x) for 1.2e-38 < |x| < 8.5e37 and the reciprocal square root
within 1 ulp for 1.2e-38 < x < 3.4e38 (each an fp32 seed and one third-order step), including
table and interval boundaries, powers of two, values next to 1 and the range ends; and the
all-fp32 float-pair exp and log of the bond-order chain."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03343_gb300 import _build, md as M
    _build.build()
    M.load()
    return M


def ulp_err(y, ref):
    return np.abs(y - ref) / np.spacing(np.abs(ref))


@pytest.mark.parametrize("fn", [0, 4], ids=["exp_tab", "exp_ff"])
def test_exp_within_two_ulp(md, fn):
    rng = np.random.Generator(np.random.PCG64(1))
    ln2_256 = np.log(2.0) / 256
    x = np.concatenate([
        rng.uniform(-12.0, 0.0, 400000),              # -lambda r, -mu r
        rng.uniform(-80.0, 10.0, 400000),             # n log(beta zeta), -log(1+x)/(2n)
        rng.uniform(-700.0, 700.0, 100000),
        np.arange(-2000, 2000) * ln2_256,              # table boundaries
        np.arange(-2000, 2000) * ln2_256 + ln2_256 / 2,  # reduction interval edges
        np.nextafter(np.arange(-2000, 2000) * ln2_256 + ln2_256 / 2, 0.0),
        [0.0, -0.0, 1e-300, -1e-300, 1e-10, -1e-10, 1.0, -1.0, 700.0, -700.0],
    ])
    y = md.md_fastmath_eval(fn, x)
    e = ulp_err(y, np.exp(x))
    assert e.max() <= 2.0, (x[np.argmax(e)], e.max())
    assert np.median(e) <= 0.5


@pytest.mark.parametrize("fn", [1, 5], ids=["log_tab", "log_ff"])
def test_log_absolute_error(md, fn):
    rng = np.random.Generator(np.random.PCG64(2))
    x = np.concatenate([
        np.exp(rng.uniform(-75.0, 25.0, 400000)),      # zeta, 1 + x of the bond order
        1.0 + rng.uniform(0.0, 300.0, 200000),
        1.0 + np.exp(rng.uniform(-40.0, 0.0, 100000)),
        2.0 ** np.arange(-1000, 1000, dtype=np.float64),
        np.nextafter(2.0 ** np.arange(-1000, 1000, dtype=np.float64), 0.0),
        1.0 + np.arange(257) / 256.0,                  # table interval boundaries
        np.nextafter(1.0 + np.arange(1, 257) / 256.0, 0.0),
        [1.0, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 1e-300, 1e300, 2.2250738585072014e-308],
    ])
    y = md.md_fastmath_eval(fn, x)
    ref = np.log(x)
    expo = np.abs(np.frexp(x)[1] - 1).astype(np.float64)
    bound = 2e-16 * (1.0 + expo)
    err = np.abs(y - ref)
    assert np.all(err <= bound), (x[np.argmax(err / bound)], (err / bound).max())
    assert y[-6] == 0.0 or abs(y[-6]) < 1e-17            # log(1) ~ 0


def round_bits(x, bits=40):
    """x rounded to `bits` significant bits: held exactly by a float pair (split_d keeps 47)."""
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 2.0 ** bits) / 2.0 ** bits, e)


def test_float_pair_exp(md):
    """exp_f2 (fn 8): relative error within 2^-45 for y in [-55, 80] (analysis: about 2^-47,
    plus the low float of the result, up to 2^-24 of it, leaving the normal range -- which the
    conversion back to a double flushes -- an absolute error below 2^-126: relative 2^-45 above
    e^-55 ~ 2^-79)."""
    rng = np.random.Generator(np.random.PCG64(5))
    ln2_256 = np.log(2.0) / 256
    x = round_bits(np.concatenate([
        rng.uniform(-8.0, 2.0, 300000),                 # n log(beta zeta)
        rng.uniform(-55.0, 80.0, 300000),
        rng.uniform(-1e-3, 1e-3, 50000),
        np.arange(-2000, 2000) * ln2_256 + ln2_256 / 2,  # reduction interval edges
        [0.0, 1e-20, -1e-20, 1.0, -1.0, 80.0, -55.0],
    ]))
    y = md.md_fastmath_eval(8, x)
    rel = np.abs(y - np.exp(x)) / np.exp(x)
    assert rel.max() <= 2.0 ** -45, (x[np.argmax(rel)], rel.max())
    lo = round_bits(rng.uniform(-80.0, -55.0, 20000))
    assert np.abs(md.md_fastmath_eval(8, lo) - np.exp(lo)).max() <= 2.0 ** -125


def test_float_pair_log(md):
    """log_f2 (fn 9): absolute error within 2^-46 (1 + |log x|) (analysis: about
    2^-47 (1 + |log x|)) for x from 2^-78 to 2^125 -- the range that the test's conversion of
    a double to a float pair holds to 47 bits, and in which the low float stays normal."""
    rng = np.random.Generator(np.random.PCG64(6))
    x = round_bits(np.concatenate([
        np.exp(rng.uniform(-30.0, 5.0, 300000)),          # beta zeta
        1.0 + np.exp(rng.uniform(-30.0, 1.0, 300000)),    # 1 + (beta zeta)^n
        np.exp(rng.uniform(-54.0, 86.0, 200000)),
        2.0 ** np.arange(-78, 126, dtype=np.float64),
        1.0 + np.arange(257) / 256.0,                     # table interval boundaries
        [1.0, 1.0 + 2.0 ** -40, 1.0 - 2.0 ** -40],
    ]))
    y = md.md_fastmath_eval(9, x)
    ref = np.log(x)
    err = np.abs(y - ref)
    bound = 2.0 ** -46 * (1.0 + np.abs(ref))
    assert np.all(err <= bound), (x[np.argmax(err / bound)], (err / bound).max())


def test_reciprocal_within_one_ulp(md):
    rng = np.random.Generator(np.random.PCG64(3))
    x = np.concatenate([
        rng.uniform(18.0, 300.0, 200000),                  # d^2 + (h - cos)^2
        np.exp(rng.uniform(-70.0, 30.0, 400000)),          # zeta (1 + (beta zeta)^n)
        -np.exp(rng.uniform(-36.0, 1.4, 200000)),          # SW r - a sigma < 0
        2.0 ** np.arange(-125, 127, dtype=np.float64),
        np.nextafter(2.0 ** np.arange(-125, 127, dtype=np.float64), 0.0),
        [1.0, 3.0, 1.2e-38, 8.0e37, -1.0, 7.0],
    ])
    y = md.md_fastmath_eval(2, x)
    e = ulp_err(y, 1.0 / x)
    assert e.max() <= 1.0, (x[np.argmax(e)], e.max())


def test_reciprocal_sqrt_within_one_ulp(md):
    """1/sqrt(x) against the value computed in extended precision (np.longdouble), over the
    bonds' r^2, decades of the fp32-normal range, powers of two and their neighbours."""
    rng = np.random.Generator(np.random.PCG64(4))
    x = np.concatenate([
        rng.uniform(0.5, 16.0, 400000),                     # r^2 of bonds (A^2)
        np.exp(rng.uniform(-85.0, 85.0, 200000)),
        2.0 ** np.arange(-125, 127, dtype=np.float64),
        np.nextafter(2.0 ** np.arange(-125, 127, dtype=np.float64), 0.0),
        np.nextafter(2.0 ** np.arange(-125, 127, dtype=np.float64), np.inf),
        [1.0, 2.0, 3.0, 4.0, 1.2e-38, 3.0e38, 2.25, 5.29],
    ])
    y = md.md_fastmath_eval(3, x)
    ref = (1.0 / np.sqrt(x.astype(np.longdouble)))
    e = np.abs(y.astype(np.longdouble) - ref) / np.spacing(ref.astype(np.float64)).astype(np.longdouble)
    e = e.astype(np.float64)
    assert e.max() <= 1.0, (x[np.argmax(e)], e.max())
    assert np.median(e) <= 0.5


def test_float_pair_reciprocal_and_rsqrt_within_one_ulp(md):
    """The reciprocal (fn 6) and reciprocal square root (fn 7) that finish their correction in
    float pairs, within 1 ulp for normal arguments (a bond order's zeta (1 + x) reaches 1e-30
    near the cutoff switch; the reciprocal square root from 2^-126 up, +inf below), including
    powers of two, their neighbours and both signs."""
    rng = np.random.Generator(np.random.PCG64(5))
    core = np.concatenate([
        rng.uniform(0.5, 16.0, 300000), rng.uniform(18.0, 300.0, 200000),
        np.exp(rng.uniform(-700.0, 700.0, 300000)),
        2.0 ** np.arange(-1021, 1021, dtype=np.float64),
        np.nextafter(2.0 ** np.arange(-1021, 1021, dtype=np.float64), 0.0),
        np.nextafter(2.0 ** np.arange(-1021, 1021, dtype=np.float64), np.inf),
        [1.0, 2.0, 3.0, 4.0, 2.25, 5.29, 7.0, 1e-30, 1e-300],
    ])
    x = np.concatenate([core, -core])
    y = md.md_fastmath_eval(6, x)
    e = ulp_err(y, 1.0 / x)
    assert e.max() <= 1.0, (x[np.argmax(e)], e.max())
    pos = core[core >= 2.0 ** -126]          # below, +inf by design (a zero-length bond)
    y = md.md_fastmath_eval(7, pos)
    ref = 1.0 / np.sqrt(pos.astype(np.longdouble))
    e = (np.abs(y.astype(np.longdouble) - ref) / np.spacing(ref.astype(np.float64)).astype(np.longdouble)).astype(np.float64)
    assert e.max() <= 1.0, (pos[np.argmax(e)], e.max())
    assert np.median(e) <= 0.5
    assert np.isinf(md.md_fastmath_eval(7, np.array([0.0, 1e-300, 2.0 ** -127]))).all()
