"""Pins for the oracle's differentiable level: epsilon-regularised float ZNCC (Eq. 2 with
two-pass means), soft-argmax readout over the admissible candidates, and its analytic
backward with respect to both images.  Pinned by FP64 central finite differences, by the
offset/gain invariances the gradient must have when epsilon = 0, and by the T -> 0 limit
reducing to the hard WTA of the integer path."""
import numpy as np
import pytest

from paper_1901_09593_gb300 import scenes

T = 0.05
N7 = 49


def _crop(seed=0, h=24, w=40):
    sc = scenes.make_float_pair(scenes.SPECS["diff_640x480"], seed)
    y0, x0 = 200, 300
    return sc.left[y0:y0 + h, x0:x0 + w].copy(), sc.right[y0:y0 + h, x0:x0 + w].copy()


def _loss(oracle_mod, L, R, wts, n, nd, eps):
    return float((oracle_mod.softargmax_fwd(L, R, n, nd, T, eps) * wts).sum())


def test_rho_matches_twopass_definition(oracle_mod):
    L, R = _crop(1, 8, 12)
    ds, rho = oracle_mod.softargmax_fwd(L, R, 2, 6, T, 1e-6 * 25, want_rho=True)
    h, w = L.shape
    for y in range(h):
        for x in range(w):
            for z in range(6):
                if z > x:
                    assert np.isneginf(rho[0, y, x, z])
                    continue
                ys = np.clip(np.arange(y - 2, y + 3), 0, h - 1)
                a = L[np.ix_(ys, np.clip(np.arange(x - 2, x + 3), 0, w - 1))]
                b = R[np.ix_(ys, np.clip(np.arange(x - z - 2, x - z + 3), 0, w - 1))]
                ac, bc = a - a.mean(), b - b.mean()
                ref = (ac * bc).sum() / np.sqrt(((ac * ac).sum() + 25e-6) * ((bc * bc).sum() + 25e-6))
                assert abs(rho[0, y, x, z] - ref) < 1e-13
            zs = np.arange(min(5, x) + 1)
            r = rho[0, y, x, zs] / T
            p = np.exp(r - r.max())
            p /= p.sum()
            assert abs(ds[0, y, x] - (zs * p).sum()) < 1e-12


def test_gradient_matches_central_differences_directional(oracle_mod):
    L, R = _crop(2, 20, 36)
    n, nd, eps = 3, 16, 1e-6 * N7
    rng = np.random.default_rng(0)
    wts = rng.standard_normal(L.shape)
    gL, gR = oracle_mod.softargmax_bwd(L, R, n, nd, T, eps, wts)
    # central differences converge as h^2 here (1.6e-5 relative at h=1e-4, 1.6e-9 at 1e-6)
    h = 1e-6
    for trial in range(3):
        vL = rng.standard_normal(L.shape)
        vR = rng.standard_normal(R.shape)
        fd = (_loss(oracle_mod, L + h * vL, R + h * vR, wts, n, nd, eps)
              - _loss(oracle_mod, L - h * vL, R - h * vR, wts, n, nd, eps)) / (2 * h)
        an = (gL[0] * vL).sum() + (gR[0] * vR).sum()
        assert abs(fd - an) <= 2e-8 * max(1.0, abs(an)), (fd, an)


def test_gradient_matches_central_differences_per_pixel(oracle_mod):
    L, R = _crop(3, 16, 28)
    n, nd, eps = 3, 12, 1e-6 * N7
    rng = np.random.default_rng(1)
    wts = rng.standard_normal(L.shape)
    gL, gR = oracle_mod.softargmax_bwd(L, R, n, nd, T, eps, wts)
    h = 1e-6
    # includes border pixels, where clamped window reads accumulate
    pts = [(0, 0), (0, 27), (15, 0), (15, 27), (7, 13), (3, 20), (10, 5), (8, 1)]
    for (y, x) in pts:
        for img, g in ((0, gL), (1, gR)):
            P, M = L.copy(), L.copy()
            Q, S = R.copy(), R.copy()
            if img == 0:
                P[y, x] += h
                M[y, x] -= h
            else:
                Q[y, x] += h
                S[y, x] -= h
            fd = (_loss(oracle_mod, P, Q, wts, n, nd, eps) - _loss(oracle_mod, M, S, wts, n, nd, eps)) / (2 * h)
            assert abs(fd - g[0, y, x]) <= 1e-6 * max(1.0, abs(fd)), (img, y, x, fd, g[0, y, x])


def test_gradient_invariances_without_epsilon(oracle_mod):
    # With eps = 0, rho is unchanged by a global offset or gain of either image, so the
    # gradient is orthogonal to the all-ones image and to the image itself.
    L, R = _crop(4, 18, 30)
    wts = np.random.default_rng(2).standard_normal(L.shape)
    gL, gR = oracle_mod.softargmax_bwd(L, R, 2, 10, T, 0.0, wts)
    scale = np.abs(gL).sum() + np.abs(gR).sum()
    assert abs(gL.sum()) <= 1e-10 * scale
    assert abs(gR.sum()) <= 1e-10 * scale
    assert abs((gL[0] * L).sum()) <= 1e-10 * scale
    assert abs((gR[0] * R).sum()) <= 1e-10 * scale


def test_small_temperature_reduces_to_hard_wta(oracle_mod):
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 8)
    a, b = sc.left[60:84, 100:150].copy(), sc.right[60:84, 100:150].copy()
    d, c, c2, _ = oracle_mod.match_level(a, b, 2, 16)
    ds, rho = oracle_mod.softargmax_fwd(a / 255.0, b / 255.0, 2, 16, 1e-4, 0.0, want_rho=True)
    clear = (c - c2) > 1e-2
    assert clear.mean() > 0.5
    np.testing.assert_allclose(ds[0][clear], d[clear], atol=1e-6)
    # and the float rho equals the integer-sum rho
    h, w = a.shape
    for y in range(0, h, 5):
        for x in range(0, w, 7):
            for z in range(min(15, x) + 1):
                assert abs(rho[0, y, x, z] - oracle_mod.zncc(a, b, 2, y, x, z)) < 1e-12
