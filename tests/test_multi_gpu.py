"""GPU parity of multi-element Tersoff (Tersoff 1989 multicomponent form, Si-C) through the
C ABI against the oracle's multi-element routines, element by element on the same seeded
inputs.  Bounds as for one element: fp64 1e-12 on F, U_i, W_i, J_i and totals, 1e-10 on
trajectories, mixed precision 1e-5 on forces."""
import numpy as np
import pytest

import oracle as O
from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
TRAJ_TOL = 1e-10
MIXED_TOL = 1e-5


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
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a).max())


CASES = [
    ("sic_zincblende_512", lambda: I.sic_zincblende(n=4, jitter_amp=0.05)),
    ("sic_zincblende_hot_1728", lambda: I.sic_zincblende(n=6, jitter_amp=0.12, temperature=1200.0, seed_pos=3)),
    ("si_c_substituted_512", lambda: I.sic_substituted_diamond(n=4)),
    ("si_c_substituted_1000_c60", lambda: I.sic_substituted_diamond(n=5, c_fraction=0.6, seed_types=8)),
    ("sic_zincblende_13824", lambda: I.sic_zincblende(n=12, jitter_amp=0.05, seed_pos=4)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_compute_fp64_matches_oracle(md, name, make):
    s = make()
    ref = O.compute_multi(s.pos, s.box, s.pbc, s.types, s.params, s.chi, s.vel)
    with md.from_multi(s) as g:
        out = g.compute()
    for k in ("F", "U", "W", "J"):
        assert rel(out[k], ref[k]) < FP64_TOL, (name, k, rel(out[k], ref[k]))
    assert rel(out["totals"], ref["totals"]) < FP64_TOL


@pytest.mark.parametrize("name,make", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_compute_mixed_force_error(md, name, make):
    s = make()
    ref = O.compute_multi(s.pos, s.box, s.pbc, s.types, s.params, s.chi, s.vel)
    with md.from_multi(s, precision=md.MD_MIXED) as g:
        out = g.compute()
    assert rel(out["F"], ref["F"]) < MIXED_TOL


@pytest.mark.parametrize("make,steps,dt", [
    (lambda: I.sic_zincblende(n=4, jitter_amp=0.05, temperature=600.0), 40, 0.5),
    (lambda: I.sic_substituted_diamond(n=4, temperature=600.0), 40, 0.5),
], ids=["sic_zincblende_512", "si_c_substituted_512"])
def test_trajectory_matches_oracle(md, make, steps, dt):
    s = make()
    with md.from_multi(s, skin=0.2) as g:
        ser = g.run(steps, dt)
        pos, vel = g.state()
    p2, v2, ser2 = O.run_multi(s.pos, s.vel, s.atom_masses, s.box, s.pbc, s.types, s.params, s.chi, steps, dt)
    d = pos - p2
    d -= np.round(d / s.box) * s.box * s.pbc
    assert np.abs(d).max() < TRAJ_TOL
    assert rel(vel, v2) < TRAJ_TOL
    for c in range(5):
        assert rel(ser[:, c], ser2[:, c]) < TRAJ_TOL, c


def test_two_labels_of_one_element_equal_the_single_element_path_bitwise(md):
    """Both elements Si with chi = 1: every mixed constant equals the element's own, so the
    multi-element kernel must reproduce the single-element kernel bit for bit."""
    s = I.si_diamond_tersoff(n=4, jitter_amp=0.08)
    rng = np.random.Generator(np.random.PCG64(12))
    types = rng.integers(0, 2, size=s.n).astype(np.int32)
    m = I.MultiSystem("si_two_labels", s.pos, s.box, s.pbc, types, (I.TERSOFF_SI_1989, I.TERSOFF_SI_1989),
                      ((1.0, 1.0), (1.0, 1.0)), (I.MASS_SI, I.MASS_SI), s.vel)
    for prec in (0, 1):
        with md.from_inputs(s, precision=prec) as g1:
            a = g1.compute()
            sa = g1.run(12, 1.0)
        with md.from_multi(m, precision=prec) as g2:
            b = g2.compute()
            sb = g2.run(12, 1.0)
        for k in ("F", "U", "W", "J", "totals"):
            assert np.array_equal(a[k], b[k]), (prec, k)
        assert np.array_equal(sa, sb), prec


def test_bad_multi_element_arguments_are_rejected(md):
    s = I.sic_zincblende(n=2)
    prm = md.multi_params(s.params, s.chi)
    with pytest.raises(md.MDError) as e:       # an element index out of range
        md.md_create(s.box, s.pbc, s.n, np.full(s.n, 2, np.int32), list(s.masses), I.MD_TERSOFF, prm, n_types=2)
    assert e.value.status == md.MD_ERR_ARG
    with pytest.raises(md.MDError):            # several elements are Tersoff only
        md.md_create(s.box, s.pbc, s.n, s.types, list(s.masses), I.MD_SW, prm, n_types=2)
    bad = prm.copy(); bad[22] = -1.0           # a non-positive chi
    with pytest.raises(md.MDError):
        md.md_create(s.box, s.pbc, s.n, s.types, list(s.masses), I.MD_TERSOFF, bad, n_types=2)
