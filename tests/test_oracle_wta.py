"""Pins for the oracle's winner-take-all levels (Eq. 3-4, Eq. 8-9 first branch) and the
hierarchical driver (Sec. III, Fig. 1): brute force on tiny inputs, planted-disparity
recovery on noise-free scenes (which fixes the disparity sign convention), K = 1 equals
flat matching, a radius covering every candidate equals the full search, candidate
counting, and admissibility of every upsampled prior."""
import numpy as np
import pytest

from paper_1901_09593_gb300 import scenes
from tests.test_oracle_zncc import zncc_twopass


def brute_level(a, b, n, dk, r=0, prior=None):
    h, w = a.shape
    d = np.zeros((h, w), np.int16)
    c = np.zeros((h, w))
    gap = np.zeros((h, w))
    evals = 0
    for y in range(h):
        for x in range(w):
            zmax = min(dk - 1, x)
            cands = list(range(0, zmax + 1))
            if prior is not None:
                dh = min(max(2 * int(prior[y // 2, x // 2]), 0), zmax)
                cands = [z for z in cands if dh - r <= z <= dh + r]
            vals = [zncc_twopass(a, b, n, y, x, z) for z in cands]
            i = int(np.argmax(vals))           # first maximum = smallest z
            d[y, x] = cands[i]
            c[y, x] = vals[i]
            s = sorted(vals, reverse=True)
            gap[y, x] = s[0] - s[1] if len(s) > 1 else np.inf
            evals += len(cands)
    return d, c, gap, evals


@pytest.mark.parametrize("n,dk", [(1, 5), (2, 8), (3, 4)])
def test_full_level_matches_bruteforce(oracle_mod, n, dk):
    rng = np.random.default_rng(100 + n)
    a = rng.integers(0, 256, (9, 14)).astype(np.uint8)
    b = rng.integers(0, 256, (9, 14)).astype(np.uint8)
    d, c, c2, ev = oracle_mod.match_level(a, b, n, dk)
    bd, bc, gap, bev = brute_level(a, b, n, dk)
    assert ev == bev
    np.testing.assert_allclose(c, bc, atol=1e-12, rtol=0)
    clear = gap > 1e-9
    np.testing.assert_array_equal(d[clear], bd[clear])
    # second-best: C - C2 agrees with the brute-force gap
    fin = np.isfinite(gap)
    np.testing.assert_allclose((c - c2)[fin], gap[fin], atol=1e-12)
    assert np.all(np.isneginf(c2[~fin]))


@pytest.mark.parametrize("r", [0, 1, 2])
def test_restricted_level_matches_bruteforce(oracle_mod, r):
    rng = np.random.default_rng(200 + r)
    a = rng.integers(0, 256, (10, 13)).astype(np.uint8)
    b = rng.integers(0, 256, (10, 13)).astype(np.uint8)
    dk = 9
    prior = rng.integers(0, 5, (5, 7)).astype(np.int16)
    d, c, c2, ev = oracle_mod.match_level(a, b, 1, dk, r, prior)
    bd, bc, gap, bev = brute_level(a, b, 1, dk, r, prior)
    assert ev == bev
    np.testing.assert_allclose(c, bc, atol=1e-12, rtol=0)
    clear = gap > 1e-9
    np.testing.assert_array_equal(d[clear], bd[clear])


def test_radius_covering_all_candidates_equals_full_search(oracle_mod):
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 7)
    a, b = sc.left[:40, :96].copy(), sc.right[:40, :96].copy()
    prior = np.random.default_rng(0).integers(0, 16, (20, 48)).astype(np.int16)
    full = oracle_mod.match_level(a, b, 2, 32)
    restr = oracle_mod.match_level(a, b, 2, 32, 64, prior)
    for u, v in zip(full, restr):
        np.testing.assert_array_equal(u, v)


def test_candidate_count_identity(oracle_mod):
    rng = np.random.default_rng(9)
    a = rng.integers(0, 256, (21, 33)).astype(np.uint8)
    b = rng.integers(0, 256, (21, 33)).astype(np.uint8)
    dk, r = 12, 2
    prior = rng.integers(0, 6, (11, 17)).astype(np.int16)
    _, _, _, ev = oracle_mod.match_level(a, b, 2, dk, r, prior)
    expect = 0
    for y in range(21):
        for x in range(33):
            zmax = min(dk - 1, x)
            dh = min(2 * int(prior[y // 2, x // 2]), zmax)
            expect += min(zmax, dh + r) - max(0, dh - r) + 1
    assert ev == expect
    _, _, _, evf = oracle_mod.match_level(a, b, 2, dk)
    assert evf == sum(min(dk - 1, x) + 1 for x in range(33)) * 21


def test_exact_ties_go_to_the_smallest_candidate(oracle_mod):
    # Tie-break reading: among candidates with equal rho the smallest z wins.  Exact ties
    # built two ways: (1) a flat left window has rho = 0 for every candidate; (2) a right
    # image periodic along rows with period 4 and a left image equal to it shifted by 1
    # column give byte-identical right windows at z = 1, 5, 9, ..., so rho = 1 exactly at
    # each of them.
    rng = np.random.default_rng(31)
    h, w, n, dk = 12, 40, 1, 16
    tile = rng.integers(0, 256, (h, 4)).astype(np.uint8)
    b = np.tile(tile, (1, w // 4))
    a = np.roll(b, 1, axis=1)
    a[:, :8] = 77                                            # flat left windows for x <= 6
    d, c, c2, _ = oracle_mod.match_level(a, b, n, dk)
    flat = np.zeros((h, w), bool)
    flat[:, :7] = True
    assert np.all(d[flat] == 0) and np.all(c[flat] == 0.0)
    assert np.all(c2[:, 1:7] == 0.0)                         # every candidate ties at 0
    per = np.zeros((h, w), bool)
    per[:, 8 + n:w - n] = True                               # left window periodic and inside the image
    assert np.all(d[per] == 1) and np.all(c[per] == 1.0) and np.all(c2[per] == 1.0)
    # restricted branch (dhat = 2 * prior): the span decides which of the tied candidates remain
    prior = np.zeros(((h + 1) // 2, (w + 1) // 2), np.int16)
    prior[:] = 2                                             # dhat = 4, r = 2: span 2 .. 6 holds z = 5 only
    d, c, _, _ = oracle_mod.match_level(a, b, n, dk, 2, prior)
    assert np.all(d[per] == 5) and np.all(c[per] == 1.0)
    prior[:] = 1                                             # dhat = 2, r = 4: span 0 .. 6 holds z = 1 and 5
    d, c, c2, _ = oracle_mod.match_level(a, b, n, dk, 4, prior)
    assert np.all(d[per] == 1) and np.all(c2[per] == 1.0)
    prior[:] = 3                                             # dhat = 6, r = 1: span 5 .. 7, flat pixels clip it
    d, _, _, _ = oracle_mod.match_level(a, b, n, dk, 1, prior)
    assert np.all(d[per] == 5)
    assert np.all(d[:, 6] == 5) and np.all(d[:, 1:5] == np.arange(1, 5) - 1)


def _interior_one_region(sc, n):
    """Left pixels whose whole window lies in one region with one disparity, is visible,
    and whose matched right window lies inside the image: there the warped right window is
    an exact copy of the left window."""
    h, w = sc.left.shape
    lab, gt = sc.labels, sc.gt.astype(np.int64)
    ok = np.zeros((h, w), bool)
    for y in range(n, h - n):
        for x in range(n, w - n):
            d = gt[y, x]
            if x - d - n < 0:
                continue
            win = (slice(y - n, y + n + 1), slice(x - n, x + n + 1))
            if np.all(lab[win] == lab[y, x]) and np.all(sc.mask[win]) and np.all(gt[win] == d):
                ok[y, x] = True
    return ok


def test_flat_bm_recovers_planted_disparities_exactly(oracle_mod):
    spec = scenes.SceneSpec(160, 96, 4, 32, 1, 5, 0, 0.0, False)
    sc = scenes.make_pair(spec, 11)
    out = oracle_mod.disparity(sc.left, sc.right, 32, 1, 5, 0)
    ok = _interior_one_region(sc, 2)
    assert ok.sum() > 0.4 * ok.size
    np.testing.assert_array_equal(out["d"][0][ok], sc.gt[ok].astype(np.int16))
    assert np.all(out["C"][0][ok] == 1.0)


def test_flat_bm_recovery_rate_with_noise(oracle_mod):
    spec = scenes.SPECS["small_320x240"]
    sc = scenes.make_pair(spec, 3)
    out = oracle_mod.disparity(sc.left, sc.right, 32, 1, 5, 2)
    ok = _interior_one_region(sc, 2)
    rate = np.mean(out["d"][0][ok] == sc.gt[ok])
    assert rate >= 0.97, rate


def test_k1_is_flat_matching(oracle_mod):
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 2)
    a, b = sc.left[:48, :120].copy(), sc.right[:48, :120].copy()
    out = oracle_mod.disparity(a, b, 32, 1, 5, 2)
    d, c, c2, ev = oracle_mod.match_level(a, b, 2, 32)
    np.testing.assert_array_equal(out["d"][0], d)
    np.testing.assert_array_equal(out["C"][0], c)
    assert out["evals"] == ev


@pytest.mark.parametrize("D", [32, 27])
def test_hierarchy_composes_levels_and_priors_are_admissible(oracle_mod, D):
    # D = 27 is not a multiple of 2^(K-1): the levels search D_k = ceil(D / 2^k) = 27, 14, 7
    # candidates (Sec. III), written out here rather than taken from the oracle
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 4)
    a, b = sc.left[:100, :200].copy(), sc.right[:100, :200].copy()
    K, w, r = 3, 5, 2
    dks = [D, (D + 1) // 2, (D + 3) // 4]
    out = oracle_mod.disparity(a, b, D, K, w, r)
    pa, pb = oracle_mod.pyramid(a, K), oracle_mod.pyramid(b, K)
    d, c, c2, ev = oracle_mod.match_level(pa[K - 1], pb[K - 1], w // 2, dks[K - 1])
    np.testing.assert_array_equal(out["d"][K - 1], d)
    total = ev
    for k in range(K - 2, -1, -1):
        prior = out["d"][k + 1]
        dk = dks[k]
        hk, wk = pa[k].shape
        yy, xx = np.mgrid[0:hk, 0:wk]
        dh = 2 * prior[yy // 2, xx // 2].astype(np.int64)
        assert np.all(dh <= np.minimum(dk - 1, xx)), "upsampled prior must be admissible"
        d, c, c2, ev = oracle_mod.match_level(pa[k], pb[k], w // 2, dk, r, prior)
        np.testing.assert_array_equal(out["d"][k], d)
        np.testing.assert_array_equal(out["C"][k], c)
        total += ev
    assert out["evals"] == total


def test_hierarchical_recovers_noise_free_scene(oracle_mod):
    spec = scenes.SceneSpec(320, 240, 4, 32, 3, 5, 2, 0.0, False)
    sc = scenes.make_pair(spec, 5)
    out = oracle_mod.disparity(sc.left, sc.right, 32, 3, 5, 2)
    ok = _interior_one_region(sc, 2)
    rate = np.mean(out["d"][0][ok] == sc.gt[ok])
    assert rate >= 0.95, rate


def test_driver_rejects_invalid_arguments(oracle_mod):
    a = np.zeros((8, 8), np.uint8)
    for D, K, w, r in ((0, 1, 3, 0), (8, 0, 3, 0), (8, 1, 4, 0), (8, 1, 3, -1)):
        with pytest.raises(ValueError):
            oracle_mod.disparity(a, a, D, K, w, r)
