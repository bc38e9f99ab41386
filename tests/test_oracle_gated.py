"""Pins for the oracle's gated steps of the full method: the bicubic cost prior (Sec.
III-C), the beta-gated fallback (Eq. 8-9 second branch), alpha refinement (Sec. III-B,
Eq. 5-7) and the selective median (Sec. III-D, Eq. 10).  Independent computations here:
half-pixel Catmull-Rom weights written out by hand, brute-force ZNCC averages, a numpy
median, and the limits of each gate that reduce it to an already-pinned step."""
import numpy as np
import pytest

from paper_1901_09593_gb300 import scenes
from tests.test_oracle_zncc import zncc_twopass

# Catmull-Rom (Keys, a = -1/2) at offset 1/2: weights of the samples at -1, 0, 1, 2
HALF = np.array([-1.0, 9.0, 9.0, -1.0]) / 16.0


def upsample_by_hand(c, h, w):
    hc, wc = c.shape
    out = np.zeros((h, w))
    for y in range(h):
        for x in range(w):
            ys = [y // 2] if y % 2 == 0 else [y // 2 + k for k in (-1, 0, 1, 2)]
            wy = [1.0] if y % 2 == 0 else HALF
            xs = [x // 2] if x % 2 == 0 else [x // 2 + k for k in (-1, 0, 1, 2)]
            wx = [1.0] if x % 2 == 0 else HALF
            s = 0.0
            for a, yy in zip(wy, ys):
                for b, xx in zip(wx, xs):
                    s += a * b * c[min(max(yy, 0), hc - 1), min(max(xx, 0), wc - 1)]
            out[y, x] = s
    return out


def test_bicubic_prior_matches_hand_weights(oracle_mod):
    rng = np.random.default_rng(0)
    c = rng.random((6, 9))
    up = oracle_mod.upsample_cost(c, 17, 11)
    np.testing.assert_allclose(up, upsample_by_hand(c, 11, 17), atol=1e-14)
    # at even coordinates the prior is the coarse value itself
    np.testing.assert_array_equal(up[0::2, 0::2][:6, :9], c[:, :9][:6])


def test_bicubic_reproduces_linear_ramps_in_the_interior(oracle_mod):
    yy, xx = np.mgrid[0:8, 0:10].astype(float)
    c = 0.25 + 0.03 * yy - 0.02 * xx
    up = oracle_mod.upsample_cost(c, 20, 16)
    Y, X = np.mgrid[0:16, 0:20] / 2.0
    inner = (Y >= 1) & (Y <= 6) & (X >= 1) & (X <= 8)
    np.testing.assert_allclose(up[inner], (0.25 + 0.03 * Y - 0.02 * X)[inner], atol=1e-14)
    np.testing.assert_allclose(oracle_mod.upsample_cost(np.full((4, 5), 0.7), 9, 7), 0.7, atol=1e-15)


def test_beta_gate_limits_reduce_to_pinned_branches(oracle_mod):
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 3)
    a, b = sc.left[40:88, 60:180].copy(), sc.right[40:88, 60:180].copy()
    pa, pb = oracle_mod.pyramid(a, 2), oracle_mod.pyramid(b, 2)
    dc, cc, _, _ = oracle_mod.match_level(pa[1], pb[1], 2, 16)
    # beta below every cost: the restricted branch everywhere
    d, c, c2, ev, fb, ch = oracle_mod.match_level_beta(pa[0], pb[0], 2, 32, 2, dc, cc, -2.0)
    dr, cr, c2r, evr = oracle_mod.match_level(pa[0], pb[0], 2, 32, 2, dc)
    assert not fb.any() and ev == evr
    np.testing.assert_array_equal(d, dr)
    np.testing.assert_array_equal(c, cr)
    # beta above every cost: the full search everywhere
    d, c, c2, ev, fb, ch = oracle_mod.match_level_beta(pa[0], pb[0], 2, 32, 2, dc, cc, 2.0)
    df, cf, c2f, evf = oracle_mod.match_level(pa[0], pb[0], 2, 32)
    assert fb.all() and ev == evf
    np.testing.assert_array_equal(d, df)
    # in between: each pixel takes the branch its upsampled cost selects
    d, c, c2, ev, fb, ch = oracle_mod.match_level_beta(pa[0], pb[0], 2, 32, 2, dc, cc, 0.9)
    np.testing.assert_allclose(ch, oracle_mod.upsample_cost(cc, pa[0].shape[1], pa[0].shape[0]), atol=1e-15)
    np.testing.assert_array_equal(fb, ~(ch > 0.9))
    np.testing.assert_array_equal(d[fb], df[fb])
    np.testing.assert_array_equal(d[~fb], dr[~fb])
    assert 0 < fb.mean() < 1


def test_alpha_refinement_matches_bruteforce(oracle_mod):
    rng = np.random.default_rng(4)
    a = rng.integers(0, 256, (7, 11)).astype(np.uint8)
    b = rng.integers(0, 256, (7, 11)).astype(np.uint8)
    n, dk = 1, 6
    d0, c0, c20, _ = oracle_mod.match_level(a, b, n, dk)
    # alpha above every cost: every pixel refined
    d, c, c2, ref = oracle_mod.alpha_refine(a, b, n, dk, 2.0, d0, c0, c20)
    assert ref.all()
    h, w = a.shape
    for y in range(h):
        for x in range(w):
            vals = []
            for z in range(min(dk - 1, x) + 1):
                nb = [zncc_twopass(a, b, n, m, q, z) for m in range(y - 1, y + 2) for q in range(x - 1, x + 2)
                      if 0 <= m < h and 0 <= q < w]
                vals.append(np.mean(nb))
            i = int(np.argmax(vals))
            s = sorted(vals, reverse=True)
            assert abs(c[y, x] - vals[i]) < 1e-12
            if len(s) == 1 or s[0] - s[1] > 1e-9:
                assert d[y, x] == i
    # alpha below every cost: nothing changes
    d, c, c2, ref = oracle_mod.alpha_refine(a, b, n, dk, -2.0, d0, c0, c20)
    assert not ref.any()
    np.testing.assert_array_equal(d, d0)
    np.testing.assert_array_equal(c, c0)


def test_selective_median_matches_numpy(oracle_mod):
    rng = np.random.default_rng(5)
    d = rng.integers(0, 40, (13, 17)).astype(np.int16)
    c = rng.random((13, 17)) * 1.2 - 0.1
    alpha = 0.6
    out = oracle_mod.selective_median(d, c, alpha)
    h, w = d.shape
    for y in range(h):
        for x in range(w):
            if c[y, x] > alpha:
                assert out[y, x] == d[y, x]
                continue
            nb = np.array([d[m, q] for m in range(y - 2, y + 3) for q in range(x - 2, x + 3)
                           if 0 <= m < h and 0 <= q < w and c[m, q] > alpha])
            expect = d[y, x] if nb.size == 0 else np.sort(nb)[(nb.size - 1) // 2]
            assert out[y, x] == expect, (y, x)
    np.testing.assert_array_equal(oracle_mod.selective_median(d, c, -2.0), d)   # nothing filtered
    np.testing.assert_array_equal(oracle_mod.selective_median(d, c, 2.0), d)    # nothing qualifies


def test_full_method_driver_composes_the_steps(oracle_mod):
    # alpha and beta differ here so that a gate fed the other threshold shows
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 6)
    a, b = sc.left[:96, :160].copy(), sc.right[:96, :160].copy()
    D, K, w, r, al, be = 32, 3, 5, 2, 0.8, 0.9
    plain = oracle_mod.disparity(a, b, D, K, w, r)
    f0 = oracle_mod.disparity_full(a, b, D, K, w, r, al, be, 0)
    for k in range(K):
        np.testing.assert_array_equal(f0["d"][k], plain["d"][k])
    assert f0["evals"] == plain["evals"]
    full = oracle_mod.disparity_full(a, b, D, K, w, r, al, be, oracle_mod.FULL_METHOD)
    pa, pb = oracle_mod.pyramid(a, K), oracle_mod.pyramid(b, K)
    dkc = oracle_mod.level_disp(D, K - 1)
    d, c, c2, evals = oracle_mod.match_level(pa[K - 1], pb[K - 1], w // 2, dkc)
    d, c, c2, refined = oracle_mod.alpha_refine(pa[K - 1], pb[K - 1], w // 2, dkc, al, d, c, c2)
    assert 0 < refined.sum() < refined.size
    # alpha refinement evaluates every candidate of the pixel at each neighbour inside the image
    hk, wk = refined.shape
    for y, x in zip(*np.nonzero(refined)):
        nb = sum(1 for m in range(y - 1, y + 2) for q in range(x - 1, x + 2) if 0 <= m < hk and 0 <= q < wk)
        evals += nb * (min(dkc - 1, x) + 1)
    np.testing.assert_array_equal(full["d"][K - 1], d)
    between = 0
    for k in range(K - 2, -1, -1):
        dk, ck, c2k, ev, _, chat = oracle_mod.match_level_beta(pa[k], pb[k], w // 2, oracle_mod.level_disp(D, k), r,
                                                               d, c, be)
        evals += ev
        between += int(np.sum((ck > al) & (ck <= be))) + int(np.sum((chat > al) & (chat <= be)))
        d = oracle_mod.selective_median(dk, ck, al)
        c = ck
        np.testing.assert_array_equal(full["d"][k], d)
        np.testing.assert_array_equal(full["C"][k], c)
    assert between > 0                     # the two thresholds select different pixels
    assert full["evals"] == evals


def test_selective_median_improves_the_planted_scene(oracle_mod):
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 1)
    s = sc.spec
    plain = oracle_mod.disparity(sc.left, sc.right, s.max_disp, s.levels, s.window, s.radius)
    med = oracle_mod.disparity_full(sc.left, sc.right, s.max_disp, s.levels, s.window, s.radius, 0.9, 0.9,
                                    oracle_mod.SELECTIVE_MEDIAN)
    assert scenes.bad_rate(med["d"][0], sc.gt, sc.mask) <= scenes.bad_rate(plain["d"][0], sc.gt, sc.mask)


def test_window_halving_rule_by_hand(oracle_mod):
    # Sec. III: the block size halves at every level; Sec. IV: 11x11 at full resolution.
    # Half-widths n_k = max(1, n_0 >> k): windows 11, 5, 3, 3, ...
    table = {5: [5, 2, 1, 1, 1], 3: [3, 1, 1, 1], 1: [1, 1, 1], 6: [6, 3, 1, 1], 4: [4, 2, 1, 1]}
    for n0, expect in table.items():
        assert [oracle_mod.level_half_width(n0, k) for k in range(len(expect))] == expect
    assert [2 * oracle_mod.level_half_width(5, k) + 1 for k in range(4)] == [11, 5, 3, 3]


def test_window_halving_composes_per_level_windows(oracle_mod):
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 7)
    a, b = sc.left[:72, :150].copy(), sc.right[:72, :150].copy()
    D, K, w, r = 40, 3, 11, 2
    full = oracle_mod.disparity_full(a, b, D, K, w, r, 0.9, 0.9, oracle_mod.WINDOW_HALVING)
    pa, pb = oracle_mod.pyramid(a, K), oracle_mod.pyramid(b, K)
    prior = None
    evals = 0
    for k in range(K - 1, -1, -1):
        n = max(1, (w // 2) >> k)
        dk = oracle_mod.level_disp(D, k)
        if prior is None:
            d, c, c2, ev = oracle_mod.match_level(pa[k], pb[k], n, dk)
        else:
            d, c, c2, ev = oracle_mod.match_level(pa[k], pb[k], n, dk, r, prior)
        np.testing.assert_array_equal(full["d"][k], d)
        np.testing.assert_array_equal(full["C"][k], c)
        prior, evals = d, evals + ev
    assert full["evals"] == evals
    # one level: halving changes nothing; without the flag every level uses w
    one = oracle_mod.disparity_full(a, b, D, 1, w, r, 0.9, 0.9, oracle_mod.WINDOW_HALVING)
    np.testing.assert_array_equal(one["d"][0], oracle_mod.disparity(a, b, D, 1, w, r)["d"][0])
    plain = oracle_mod.disparity_full(a, b, D, K, w, r, 0.9, 0.9, 0)
    np.testing.assert_array_equal(plain["d"][0], oracle_mod.disparity(a, b, D, K, w, r)["d"][0])
    assert not np.array_equal(plain["d"][K - 1], full["d"][K - 1])
