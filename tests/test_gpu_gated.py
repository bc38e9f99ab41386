"""GPU parity of the gated steps of the full method against the oracle, each fed the same
inputs: the selective median (Eq. 10) bit for bit, alpha refinement (Eq. 5-7) and the
beta-gated level (Eq. 8-9) within the usual tolerances (gate decisions taken within 1e-5 of
the threshold and near-ties counted, not failed), then the whole gated pass end to end."""
import numpy as np
import pytest

import oracle
from paper_1901_09593_gb300 import scenes
from tests.gpu_util import COST_TOL, TIE_TOL, compare_level, dev, host

pytestmark = pytest.mark.gpu

ALPHA = float(np.float32(0.9))   # the kernels compare float costs with the float threshold
BETA = float(np.float32(0.9))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09593_gb300 import build
    build.build()
    oracle.build()


def ctx_for(w, h, D, K, win, r, flags):
    from paper_1901_09593_gb300 import Context
    return Context(w, h, D, K, win, r, flags, alpha=ALPHA, beta=BETA)


@pytest.mark.parametrize("h,w,dmax", [(37, 83, 60), (1001, 1403, 640)])
def test_selective_median_bit_exact(h, w, dmax):
    # a small map (32 x 8 tiles) and a ragged benchmark-sized one (32 x 32 tiles, two sorted
    # pixels a thread, odd job counts), disparities up to the large pair's range
    from paper_1901_09593_gb300 import _lib
    rng = np.random.default_rng(0)
    d = rng.integers(0, dmax, (h, w)).astype(np.int16)
    c = (rng.random((h, w)) * 1.3 - 0.2).astype(np.float32)
    ctx = ctx_for(w, h, dmax + 1, 1, 5, 2, _lib.MSBM_FLAG_SELECTIVE_MEDIAN)
    out = host(ctx.selective_median(0, dev(d), dev(c)))
    ref = oracle.selective_median(d, c.astype(np.float64), ALPHA)
    np.testing.assert_array_equal(out, ref)


def test_alpha_refinement_matches_oracle():
    from paper_1901_09593_gb300 import _lib
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 2)
    a, b = sc.left[:80, :128].copy(), sc.right[:80, :128].copy()
    ctx = ctx_for(128, 80, 24, 1, 5, 2, _lib.MSBM_FLAG_ALPHA_REFINE)
    ctx.pyramid(dev(a), dev(b))
    d, c = ctx.match_level(0)
    d0, c0 = host(d).copy(), host(c).copy()
    ctx.alpha_refine(0, d, c)
    dg, cg = host(d), host(c)
    do, co, c2o, ref = oracle.alpha_refine(a, b, 2, 24, ALPHA, d0, c0.astype(np.float64))
    assert ref.any() and not ref.all()
    np.testing.assert_array_equal(dg[~ref], d0[~ref])
    np.testing.assert_array_equal(cg[~ref], c0[~ref])
    assert np.abs(cg[ref] - co[ref]).max() <= COST_TOL
    near = (co - c2o) < TIE_TOL
    assert np.all((dg == do) | near)


def test_beta_level_matches_oracle_with_oracle_priors():
    from paper_1901_09593_gb300 import _lib
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 3)
    s = sc.spec
    K = 3
    ref = oracle.disparity(sc.left, sc.right, s.max_disp, K, s.window, s.radius)
    ctx = ctx_for(s.width, s.height, s.max_disp, K, s.window, s.radius, _lib.MSBM_FLAG_BETA_FALLBACK)
    ctx.pyramid(dev(sc.left), dev(sc.right))
    pa, pb = oracle.pyramid(sc.left, K), oracle.pyramid(sc.right, K)
    for k in (1, 0):
        prior, cprior = ref["d"][k + 1], ref["C"][k + 1].astype(np.float32)
        d, c, fb = ctx.match_level_beta(k, dev(prior), dev(cprior))
        dk = oracle.level_disp(s.max_disp, k)
        do, co, c2o, ev, fbo, ch = oracle.match_level_beta(pa[k], pb[k], s.window // 2, dk, s.radius, prior,
                                                           cprior.astype(np.float64), BETA)
        fbg = host(fb).astype(bool)
        near_gate = np.abs(ch - BETA) < 1e-5
        assert np.all((fbg == fbo) | near_gate)
        same = fbg == fbo
        assert fbo.any() and not fbo.all()
        compare_level(host(d)[same], host(c)[same], do[same], co[same], c2o[same], f"beta level {k}")


@pytest.mark.parametrize("win", [3, 7, 13])
def test_beta_level_window_classes_ragged(win):
    # the fallback's full-range cell search at a small, the benchmark's and the widest
    # window, on a level with an odd width and height (cells cut by both edges) and a
    # disparity range of many candidate groups; where the gate is decided alike everywhere,
    # the evaluation count is the oracle's too
    from paper_1901_09593_gb300 import _lib
    spec = scenes.SceneSpec(317, 239, 4, 96, 2, win, 2, 2.0, False)
    sc = scenes.make_pair(spec, 11)
    K, D, r = 2, spec.max_disp, spec.radius
    ref = oracle.disparity(sc.left, sc.right, D, K, win, r)
    ctx = ctx_for(spec.width, spec.height, D, K, win, r, _lib.MSBM_FLAG_BETA_FALLBACK)
    ctx.pyramid(dev(sc.left), dev(sc.right))
    pa, pb = oracle.pyramid(sc.left, K), oracle.pyramid(sc.right, K)
    prior, cprior = ref["d"][1], ref["C"][1].astype(np.float32)
    ctx.eval_count(reset=True)
    d, c, fb = ctx.match_level_beta(0, dev(prior), dev(cprior))
    ev_g = ctx.eval_count(reset=True)
    do, co, c2o, ev, fbo, ch = oracle.match_level_beta(pa[0], pb[0], win // 2, oracle.level_disp(D, 0), r, prior,
                                                       cprior.astype(np.float64), BETA)
    fbg = host(fb).astype(bool)
    assert np.all((fbg == fbo) | (np.abs(ch - BETA) < 1e-5))
    assert fbo.any() and not fbo.all()
    if np.array_equal(fbg, fbo):
        assert ev_g == ev, (ev_g, ev)
    same = fbg == fbo
    compare_level(host(d)[same], host(c)[same], do[same], co[same], c2o[same], f"beta level 0, window {win}")


def test_beta_level_full_size_element_wise():
    # level 0 of the 1400x1000 benchmark pair (D = 256, 7x7): the gate, the restricted search
    # of the other pixels and the fallback's full-range search of about a quarter of the level
    # (one list of some 90 000 cells walked by the persistent grid), every pixel against the
    # oracle fed the same priors; the evaluation count is the oracle's where the gate agrees
    from paper_1901_09593_gb300 import _lib
    sc = scenes.make_pair(scenes.SPECS["bench_1400x1000"], 0)
    s = sc.spec
    ref = oracle.disparity(sc.left, sc.right, s.max_disp, s.levels, s.window, s.radius)
    ctx = ctx_for(s.width, s.height, s.max_disp, s.levels, s.window, s.radius, _lib.MSBM_FLAG_BETA_FALLBACK)
    ctx.pyramid(dev(sc.left), dev(sc.right))
    prior, cprior = ref["d"][1], ref["C"][1].astype(np.float32)
    ctx.eval_count(reset=True)
    d, c, fb = ctx.match_level_beta(0, dev(prior), dev(cprior))
    ev_g = ctx.eval_count(reset=True)
    pa, pb = oracle.pyramid(sc.left, 1), oracle.pyramid(sc.right, 1)
    do, co, c2o, ev, fbo, ch = oracle.match_level_beta(pa[0], pb[0], s.window // 2, s.max_disp, s.radius, prior,
                                                       cprior.astype(np.float64), BETA)
    fbg = host(fb).astype(bool)
    assert np.all((fbg == fbo) | (np.abs(ch - BETA) < 1e-5))
    assert 0.1 < fbo.mean() < 0.5
    if np.array_equal(fbg, fbo):
        assert ev_g == ev, (ev_g, ev)
    same = fbg == fbo
    compare_level(host(d)[same], host(c)[same], do[same], co[same], c2o[same], "beta level 0, 1400x1000")


def test_full_method_full_size_matches_oracle():
    # the whole full method (alpha refinement, beta fallback at every finer level, selective
    # median) on the benchmark pair against the oracle's: a near-tie at a coarse level may
    # move a few pixels below it, so the maps are compared by agreement and bad-pixel rate
    from paper_1901_09593_gb300 import _lib
    sc = scenes.make_pair(scenes.SPECS["bench_1400x1000"], 0)
    s = sc.spec
    ctx = ctx_for(s.width, s.height, s.max_disp, s.levels, s.window, s.radius, _lib.MSBM_FLAGS_FULL_METHOD)
    ctx.eval_count(reset=True)
    d, c = ctx.disparity(dev(sc.left), dev(sc.right))
    ctx.sync()
    ev_g = ctx.eval_count(reset=True)
    ref = oracle.disparity_full(sc.left, sc.right, s.max_disp, s.levels, s.window, s.radius, ALPHA, BETA,
                                oracle.FULL_METHOD)
    dg = host(d)
    assert (dg == ref["d"][0]).mean() > 0.995
    assert abs(scenes.bad_rate(dg, sc.gt, sc.mask) - scenes.bad_rate(ref["d"][0], sc.gt, sc.mask)) < 0.002
    assert abs(ev_g - ref["evals"]) <= 0.01 * ref["evals"], (ev_g, ref["evals"])


def test_gated_pass_end_to_end_small():
    from paper_1901_09593_gb300 import _lib
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 4)
    s = sc.spec
    ctx = ctx_for(s.width, s.height, s.max_disp, s.levels, s.window, s.radius, _lib.MSBM_FLAGS_FULL_METHOD)
    d, c = ctx.disparity(dev(sc.left), dev(sc.right))
    ctx.sync()
    ref = oracle.disparity_full(sc.left, sc.right, s.max_disp, s.levels, s.window, s.radius, ALPHA, BETA,
                                oracle.FULL_METHOD)
    dg = host(d)
    assert (dg == ref["d"][0]).mean() > 0.99
    bg = scenes.bad_rate(dg, sc.gt, sc.mask)
    bo = scenes.bad_rate(ref["d"][0], sc.gt, sc.mask)
    assert abs(bg - bo) < 0.005
    assert ctx.eval_count() > 0


@pytest.mark.parametrize("flags_name", ["MSBM_FLAG_SELECTIVE_MEDIAN", "MSBM_FLAGS_FULL_METHOD"])
def test_gated_pass_beats_flat_bad_rate_on_benchmark_pair(flags_name):
    from paper_1901_09593_gb300 import _lib
    sc = scenes.make_pair(scenes.SPECS["bench_1400x1000"], 0)
    s = sc.spec
    ctx = ctx_for(s.width, s.height, s.max_disp, s.levels, s.window, s.radius, getattr(_lib, flags_name))
    d, c = ctx.disparity(dev(sc.left), dev(sc.right))
    flat = ctx_for(s.width, s.height, s.max_disp, 1, s.window, s.radius, 0)
    df, cf = flat.disparity(dev(sc.left), dev(sc.right))
    ctx.sync()
    flat.sync()
    bad_h = scenes.bad_rate(host(d), sc.gt, sc.mask)
    bad_f = scenes.bad_rate(host(df), sc.gt, sc.mask)
    assert bad_h <= bad_f, (bad_h, bad_f)


def test_window_halving_levels_match_oracle():
    # per-level block size halving (Sec. III): level k matches with half-width max(1, n >> k)
    from paper_1901_09593_gb300 import Context, _lib
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 8)
    s = sc.spec
    K, win = 3, 11
    flags = _lib.MSBM_FLAG_WINDOW_HALVING
    ctx = Context(s.width, s.height, s.max_disp, K, win, s.radius, flags)
    ctx.pyramid(dev(sc.left), dev(sc.right))
    ref = oracle.disparity_full(sc.left, sc.right, s.max_disp, K, win, s.radius, ALPHA, BETA,
                                oracle.WINDOW_HALVING)
    pa, pb = oracle.pyramid(sc.left, K), oracle.pyramid(sc.right, K)
    for k in range(K - 1, -1, -1):
        n = oracle.level_half_width(win // 2, k)
        dk = oracle.level_disp(s.max_disp, k)
        if k == K - 1:
            d, c = ctx.match_level(k)
            do, co, c2o, _ = oracle.match_level(pa[k], pb[k], n, dk)
        else:
            prior = ref["d"][k + 1]
            d, c = ctx.match_level(k, dev(prior))
            do, co, c2o, _ = oracle.match_level(pa[k], pb[k], n, dk, s.radius, prior)
        compare_level(host(d), host(c), do, co, c2o, f"halving level {k} (n={n})")
    d, c = ctx.disparity(dev(sc.left), dev(sc.right))
    ctx.sync()
    assert (host(d) == ref["d"][0]).mean() > 0.99
    assert ctx.eval_count() > 0
