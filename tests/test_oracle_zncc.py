"""Pins for the oracle's ZNCC (Eq. 1-2, read as standard zero-mean normalised
cross-correlation in [-1, 1], left reference, right column x - z, clamp-to-edge windows).

The oracle evaluates from exact integer sums (c = N*Sab - Sa*Sb ...).  The brute force
below is the textbook two-pass form over explicitly gathered windows; they must agree to
1e-12.  Invariants fix what neither could get wrong in the same way."""
import numpy as np
import pytest


def window(img, y, x, n):
    h, w = img.shape
    ys = np.clip(np.arange(y - n, y + n + 1), 0, h - 1)
    xs = np.clip(np.arange(x - n, x + n + 1), 0, w - 1)
    return img[np.ix_(ys, xs)].astype(np.float64)


def zncc_twopass(a_img, b_img, n, y, x, z):
    a = window(a_img, y, x, n)
    b = window(b_img, y, x - z, n)
    ac, bc = a - a.mean(), b - b.mean()
    saa, sbb = (ac * ac).sum(), (bc * bc).sum()
    if saa == 0 or sbb == 0:
        return 0.0
    return float((ac * bc).sum() / np.sqrt(saa * sbb))


@pytest.mark.parametrize("w", [3, 5, 7, 9])
def test_zncc_matches_twopass_bruteforce(oracle_mod, w):
    rng = np.random.default_rng(w)
    n = w // 2
    for trial in range(4):
        h, wd = rng.integers(3, 13), rng.integers(4, 17)
        a = rng.integers(0, 256, (h, wd)).astype(np.uint8)
        b = rng.integers(0, 256, (h, wd)).astype(np.uint8)
        for y in range(h):
            for x in range(wd):
                for z in range(0, x + 1):
                    got = oracle_mod.zncc(a, b, n, y, x, z)
                    ref = zncc_twopass(a, b, n, y, x, z)
                    assert abs(got - ref) <= 1e-12, (trial, y, x, z, got, ref)


def test_zncc_bounds_and_flat_windows(oracle_mod):
    rng = np.random.default_rng(1)
    a = rng.integers(0, 256, (16, 24)).astype(np.uint8)
    b = rng.integers(0, 256, (16, 24)).astype(np.uint8)
    vals = [oracle_mod.zncc(a, b, 2, y, x, z) for y in range(16) for x in range(24) for z in range(x + 1)]
    assert max(vals) <= 1.0 and min(vals) >= -1.0
    flat = np.full((10, 10), 93, np.uint8)
    assert oracle_mod.zncc(flat, b[:10, :10].copy(), 1, 4, 4, 0) == 0.0
    assert oracle_mod.zncc(b[:10, :10].copy(), flat, 1, 4, 4, 2) == 0.0


@pytest.mark.parametrize("w", [3, 5, 7])
def test_zncc_self_is_exactly_one(oracle_mod, w):
    # For windows up to 7x7, Va*Va < 2^53, so c / sqrt(Va*Va) is exactly 1 in FP64.
    rng = np.random.default_rng(10 + w)
    a = rng.integers(0, 256, (14, 18)).astype(np.uint8)
    for y in range(14):
        for x in range(18):
            assert oracle_mod.zncc(a, a, w // 2, y, x, 0) == 1.0


def test_zncc_gain_offset_invariance_and_sign_flip(oracle_mod):
    rng = np.random.default_rng(3)
    a = rng.integers(0, 128, (12, 20)).astype(np.uint8)
    b = rng.integers(0, 128, (12, 20)).astype(np.uint8)
    b_aff = (2 * b.astype(np.int64) + 1).astype(np.uint8)          # exact gain 2, offset 1
    a_aff = (a.astype(np.int64) + 100).astype(np.uint8)             # exact offset
    b_neg = (255 - b.astype(np.int64)).astype(np.uint8)             # gain -1
    for y in range(12):
        for x in range(20):
            for z in range(x + 1):
                r = oracle_mod.zncc(a, b, 2, y, x, z)
                assert abs(oracle_mod.zncc(a_aff, b_aff, 2, y, x, z) - r) <= 1e-12
                assert abs(oracle_mod.zncc(a, b_neg, 2, y, x, z) + r) <= 1e-12


def test_zncc_symmetric_under_swapping_images(oracle_mod):
    # rho(left window at x, right window at x - z) == rho with the images swapped, the
    # window at x - z as the reference and "disparity" -z.
    rng = np.random.default_rng(4)
    a = rng.integers(0, 256, (10, 15)).astype(np.uint8)
    b = rng.integers(0, 256, (10, 15)).astype(np.uint8)
    for y in range(10):
        for x in range(15):
            for z in range(x + 1):
                assert oracle_mod.zncc(a, b, 1, y, x, z) == oracle_mod.zncc(b, a, 1, y, x - z, -z)
