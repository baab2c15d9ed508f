"""Launch tuning: the pair pass's block size, the pools' blocks per SM and the bond slots of
the fp64 Tersoff common-case pass change only the speed.  Every candidate must give bitwise
the same forces, per-atom fields and trajectories (with 3 slots every 4-bonded Si atom goes
to the full-capacity pass), the autotuner must pick one of its candidates, and a run after
tuning must equal a run without it."""
import numpy as np
import pytest

from paper_1610_03343_gb300 import inputs as I

pytestmark = pytest.mark.gpu

BLOCKS = (32, 64, 128, 256)


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1610_03343_gb300 import _build, md as M
    _build.build()
    M.load()
    return M


def single_cases():
    return [
        (I.si_diamond_tersoff(n=5, jitter_amp=0.05), 1.0),
        (I.c_graphene_tersoff(nx=12, ny=20, jitter_amp=0.02), 0.5),
        (I.si_diamond_sw(n=5, jitter_amp=0.1), 1.0),
    ]


def pool_mix():
    return [
        (I.si_diamond_tersoff(n=3, jitter_amp=0.05, seed_pos=3, seed_vel=4), 0),
        (I.c_graphene_tersoff(nx=6, ny=10, jitter_amp=0.02, seed_pos=5, seed_vel=6), 1),
        (I.si_diamond_tersoff(n=4, jitter_amp=0.05, seed_pos=7, seed_vel=8), 0),
        (I.c_diamond_tersoff(n=3, jitter_amp=0.02, seed_pos=9, seed_vel=10), 1),
        (I.si_diamond_tersoff(n=2, jitter_amp=0.05, seed_pos=11, seed_vel=12), 0),
    ]


def make_pool(md, precision):
    pool = md.Pool(20000, 8, I.MD_TERSOFF, [I.TERSOFF_SI_1989, I.TERSOFF_C_1989], [I.MASS_SI, I.MASS_C],
                   precision=precision)
    ids = [pool.add(s.pos, s.vel, s.box, s.pbc, pset, np.full(s.n, pset, np.int32)) for s, pset in pool_mix()]
    return pool, ids


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", range(3))
def test_pair_block_does_not_change_results(md, precision, case):
    s, dt = single_cases()[case]
    ref = None
    for cap in (0, 3):
        for b in BLOCKS:
            with md.from_inputs(s, precision=precision) as g:
                md.md_set_tuning(g.ctx, pair_block=b, pair_cap=cap)
                t = md.md_get_tuning(g.ctx)
                assert t.pair_block == b
                # the 3-bond staging exists for the single-system fp64 Tersoff pass only
                assert t.pair_cap == (3 if (cap == 3 and precision == 0 and s.kind == I.MD_TERSOFF) else 4)
                out = g.compute(want=("f", "u", "w", "j"))
                ser = g.run(16, dt)
                x, v = g.state()
                got = (out["F"], out["U"], out["W"], out["J"], out["totals"], ser, x, v)
            if ref is None:
                ref = got
            else:
                for a, r in zip(got, ref):
                    assert np.array_equal(a, r), (s.name, b, cap)


@pytest.mark.parametrize("precision", [0, 1])
def test_pool_launch_shape_does_not_change_results(md, precision):
    ref = None
    for b, g in ((64, 16), (32, 1), (256, 4), (128, 64)):
        pool, ids = make_pool(md, precision)
        with pool:
            md.md_set_tuning(pool.ctx, pair_block=b, pool_blocks_per_sm=g)
            ser = pool.run(20, 0.5, record=True)
            got = [ser] + [np.concatenate(pool.state(sid)) for sid in ids]
        if ref is None:
            ref = got
        else:
            for a, r in zip(got, ref):
                assert np.array_equal(a, r), (b, g)


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_single_system(md, precision):
    s, dt = single_cases()[0]
    with md.from_inputs(s, precision=precision) as g0, md.from_inputs(s, precision=precision) as g1:
        g0.run(5, dt)
        g1.run(5, dt)
        t = md.md_autotune(g1.ctx, 3)
        caps = (4, 3) if precision == 0 else (4,)   # Tersoff Si: both stagings for fp64
        assert t.pair_block in BLOCKS and t.pair_cap in caps
        assert t.n_tried == len(BLOCKS) * len(caps)
        tried = sorted((t.tried_pair_cap[k], t.tried_pair_block[k]) for k in range(t.n_tried))
        assert tried == sorted((c, b) for c in caps for b in BLOCKS)
        assert all(t.tried_ms[k] > 0 for k in range(t.n_tried))
        k_best = [(t.tried_pair_cap[k], t.tried_pair_block[k]) for k in range(t.n_tried)].index((t.pair_cap, t.pair_block))
        assert t.tried_ms[k_best] == min(t.tried_ms[k] for k in range(t.n_tried))
        got = md.md_get_tuning(g1.ctx)
        assert (got.pair_block, got.pair_cap) == (t.pair_block, t.pair_cap)
        s0, s1 = g0.run(12, dt), g1.run(12, dt)
        assert np.array_equal(s0, s1)
        for a, b in zip(g0.state(), g1.state()):
            assert np.array_equal(a, b)


def test_autotune_pool(md):
    p0, ids0 = make_pool(md, 1)
    p1, ids1 = make_pool(md, 1)
    with p0, p1:
        p0.run(3, 0.5)
        p1.run(3, 0.5)
        t = md.md_autotune(p1.ctx, 3)
        assert t.n_tried == 4 + 5
        assert t.pair_block in BLOCKS and t.pool_blocks_per_sm in (4, 8, 16, 32, 64)
        tuned = md.tuning_dict(t)
        assert len(tuned["tried"]) == 9
        s0, s1 = p0.run(10, 0.5, record=True), p1.run(10, 0.5, record=True)
        assert np.array_equal(s0, s1)
        for a, b in zip(ids0, ids1):
            assert np.array_equal(np.concatenate(p0.state(a)), np.concatenate(p1.state(b)))


def test_set_tuning_rejects_bad_values(md):
    s, _ = single_cases()[0]
    with md.from_inputs(s) as g:
        for b, gp in ((48, 16), (512, 16), (64, 0), (64, 65)):
            with pytest.raises(md.MDError) as e:
                md.md_set_tuning(g.ctx, pair_block=b, pool_blocks_per_sm=gp)
            assert e.value.status == md.MD_ERR_ARG
        for cap in (1, 2, 5, 8):
            with pytest.raises(md.MDError) as e:
                md.md_set_tuning(g.ctx, pair_block=64, pair_cap=cap)
            assert e.value.status == md.MD_ERR_ARG
        md.md_set_tuning(g.ctx, pair_block=0)
        assert md.md_get_tuning(g.ctx).pair_block == 64
        assert md.md_get_tuning(g.ctx).pair_cap == 4


def test_autotune_before_positions_is_a_state_error(md):
    s, _ = single_cases()[0]
    with md.System(s.box, s.pbc, s.n, s.kind, s.params, s.mass) as g:
        with pytest.raises(md.MDError) as e:
            md.md_autotune(g.ctx)
        assert e.value.status == md.MD_ERR_STATE


def test_three_bond_staging_defers_bonds_in_the_switching_region(md):
    """The fp64 3-bond staging holds no f_C values: an atom with a bond in R <= r < S goes to
    the full-capacity pass.  A sheet stretched so that bonds straddle R = 1.8 A (bond 1.78 A,
    second neighbours at 3.1 A, outside S) defers some atoms and not others; its forces,
    per-atom fields and trajectory equal the 4-bond staging's bit for bit and the oracle's
    to 1e-12."""
    import oracle as O
    s = I.c_graphene_tersoff(nx=8, ny=12, a_cc=1.78, jitter_amp=0.06, seed_pos=21, seed_vel=22)
    ref = O.compute(s.pos, s.box, s.pbc, s.kind, s.params, s.vel)
    got = {}
    for cap in (3, 4):
        with md.from_inputs(s, precision=0) as g:
            md.md_set_tuning(g.ctx, pair_block=64, pair_cap=cap)
            assert md.md_get_tuning(g.ctx).pair_cap == cap
            out = g.compute(want=("f", "u", "w", "j"))
            deferred = g.stats().pair_deferred
            ser = g.run(16, 0.5)
            x, v = g.state()
        got[cap] = (out["F"], out["U"], out["W"], out["J"], out["totals"], ser, x, v)
        if cap == 3:
            assert 0 < deferred < s.n, deferred
            for k in ("F", "U", "W", "J"):
                den = np.abs(ref[k]).max()
                assert np.abs(out[k] - ref[k]).max() / den < 1e-12, k
    for a, b in zip(got[3], got[4]):
        assert np.array_equal(a, b)


def test_many_switching_bonds_switch_to_the_staging_with_fc(md):
    """Where most atoms have a bond in the switching region (the stretched sheet: 300 of 384),
    the stagings without f_C defer them all; after the first md_run call the context stages
    4 bonds with f_C, defers none, and the trajectory goes on exactly as the oracle's."""
    import oracle as O
    s = I.c_graphene_tersoff(nx=8, ny=12, a_cc=1.78, jitter_amp=0.06, seed_pos=21, seed_vel=22)
    with md.from_inputs(s, precision=0) as g:
        md.md_set_tuning(g.ctx, pair_block=64, pair_cap=3)
        ser1 = g.run(4, 0.5)
        assert md.md_get_tuning(g.ctx).pair_cap == 4
        ser2 = g.run(4, 0.5)
        assert g.stats().pair_deferred == 0
        x, v = g.state()
    p2, v2, ser_ref = O.run(s.pos, s.vel, s.mass, s.box, s.pbc, s.kind, s.params, 8, 0.5)
    d = x - p2
    d -= np.round(d / s.box) * s.box
    assert np.abs(d).max() < 1e-10
    assert np.abs(v - v2).max() / np.abs(v2).max() < 1e-10
    ser = np.concatenate([ser1, ser2])
    for c in range(5):
        assert np.abs(ser[:, c] - ser_ref[:, c]).max() / np.abs(ser_ref[:, c]).max() < 1e-10, c
