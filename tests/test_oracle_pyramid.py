"""Pins for the oracle's Gaussian pyramid (Sec. III, Fig. 1; reading: 5-tap binomial,
clamp-to-edge, ceil halving, integer rounding).  The oracle sums the 2-D kernel directly;
the brute force here filters separably with numpy edge padding, a different computation
that must agree bit for bit because every step is exact integer arithmetic."""
import numpy as np
import pytest

C5 = np.array([1, 4, 6, 4, 1], dtype=np.int64)


def separable_reduce(img: np.ndarray) -> np.ndarray:
    h, w = img.shape
    p = np.pad(img.astype(np.int64), 2, mode="edge")
    v = sum(C5[a] * p[a:a + h, :] for a in range(5))          # vertical taps, (h, w+4)
    s = sum(C5[b] * v[:, b:b + w] for b in range(5))          # horizontal taps, (h, w)
    return ((s[0::2, 0::2] + 128) >> 8).astype(np.uint8)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (5, 1), (2, 3), (9, 17), (24, 31), (60, 80)])
def test_reduce_matches_separable_bruteforce(oracle_mod, shape):
    rng = np.random.default_rng(shape[0] * 1000 + shape[1])
    img = rng.integers(0, 256, shape).astype(np.uint8)
    out = oracle_mod.reduce(img)
    assert out.shape == ((shape[0] + 1) // 2, (shape[1] + 1) // 2)
    np.testing.assert_array_equal(out, separable_reduce(img))


@pytest.mark.parametrize("v", [0, 1, 77, 128, 254, 255])
def test_constant_image_is_fixed_point(oracle_mod, v):
    img = np.full((13, 22), v, np.uint8)
    np.testing.assert_array_equal(oracle_mod.reduce(img), np.full((7, 11), v, np.uint8))


def test_impulse_response_is_binomial_outer_product(oracle_mod):
    # An interior impulse of height 255 at (8, 10) (even coordinates, so the decimated
    # grid passes through it): output (4 + i, 5 + j) sees weight c[2-2i]*c[2-2j] for
    # |2i|, |2j| <= 2, i.e. the centre tap 36, edge taps 6*1, corner 1*1.
    img = np.zeros((20, 24), np.uint8)
    img[8, 10] = 255
    out = oracle_mod.reduce(img).astype(np.int64)
    expect = np.zeros_like(out)
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            wgt = C5[2 - 2 * i] * C5[2 - 2 * j]
            expect[4 + i, 5 + j] = (255 * wgt + 128) >> 8
    np.testing.assert_array_equal(out, expect)
    # row sum of the 1-D taps at even offsets is 1+6+1 = 8 of 16: total mass 64/256 of the
    # impulse lands on the decimated grid
    assert expect.sum() == (255 * 36 + 128) // 256 + 4 * ((255 * 6 + 128) // 256) + 4 * ((255 + 128) // 256)


def test_pyramid_levels_and_sizes(oracle_mod):
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (37, 53)).astype(np.uint8)
    levels = oracle_mod.pyramid(img, 4)
    assert [lv.shape for lv in levels] == [(37, 53), (19, 27), (10, 14), (5, 7)]
    np.testing.assert_array_equal(levels[0], img)
    for k in range(1, 4):
        np.testing.assert_array_equal(levels[k], separable_reduce(levels[k - 1]))


def test_level_disp_is_ceiling(oracle_mod):
    assert [oracle_mod.level_disp(256, k) for k in range(5)] == [256, 128, 64, 32, 16]
    assert [oracle_mod.level_disp(33, k) for k in range(4)] == [33, 17, 9, 5]
    # nested ceilings: D_{k+1} == ceil(D_k / 2) for every D, k
    for d in range(1, 300):
        for k in range(6):
            assert oracle_mod.level_disp(d, k + 1) == -(-oracle_mod.level_disp(d, k) // 2)
