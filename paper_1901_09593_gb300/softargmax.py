"""Differentiable ZNCC level: soft-argmax disparity with a hand-written backward.

``ZnccSoftArgmax.apply(left, right, window, ndisp, temperature, eps)`` maps float32 image
batches (B, H, W) on the GPU to d_soft (B, H, W).  Forward and backward run in libmsbm's
kernels.  When a gradient is wanted the forward keeps the cost volume and the window
statistics (msbm_zncc_softargmax_fwd_saved, B x ndisp x H x W floats) for the backward
(msbm_zncc_softargmax_bwd_saved); ``ZnccSoftArgmax.apply(..., keep=False)`` keeps nothing
and the backward recomputes them (msbm_zncc_softargmax_fwd / _bwd).
"""
from __future__ import annotations

import ctypes

from . import _lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _torch():
    import torch
    return torch


def default_eps(window: int) -> float:
    return 1e-6 * window * window


def _check(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a CUDA float32 tensor")
    if t.dim() != 3 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (B, H, W) tensor")


def forward_raw(left, right, window: int, ndisp: int, temperature: float, eps: float, keep: bool = False):
    """Returns (d_soft, m, l, saved): saved is the kept cost volume and statistics (a uint8
    device tensor) when keep, else None."""
    torch = _torch()
    _check(left, "left")
    _check(right, "right")
    if left.shape != right.shape:
        raise ValueError("left and right must have the same shape")
    lib = _lib.load()
    b, h, w = left.shape
    d = torch.empty_like(left)
    m = torch.empty_like(left)
    l = torch.empty_like(left)
    st = torch.cuda.current_stream(left.device).cuda_stream
    if not keep:
        _lib.check(lib.msbm_zncc_softargmax_fwd(_p(left), _p(right), b, h, w, window, ndisp,
                                                float(temperature), float(eps), _p(d), _p(m), _p(l),
                                                ctypes.c_void_p(st)), "msbm_zncc_softargmax_fwd")
        return d, m, l, None
    nbytes = lib.msbm_zncc_softargmax_saved_bytes(b, h, w, window, ndisp)
    saved = torch.empty(nbytes, dtype=torch.uint8, device=left.device)
    _lib.check(lib.msbm_zncc_softargmax_fwd_saved(_p(left), _p(right), b, h, w, window, ndisp,
                                                  float(temperature), float(eps), _p(d), _p(m), _p(l),
                                                  _p(saved), nbytes, ctypes.c_void_p(st)),
               "msbm_zncc_softargmax_fwd_saved")
    return d, m, l, saved


def backward_raw(left, right, window, ndisp, temperature, eps, d, m, l, g, saved=None):
    torch = _torch()
    lib = _lib.load()
    b, h, w = left.shape
    nbytes = lib.msbm_zncc_softargmax_workspace_bytes(b, h, w, window, ndisp)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=left.device)
    gl = torch.empty_like(left)
    gr = torch.empty_like(left)
    g = g.contiguous()
    st = torch.cuda.current_stream(left.device).cuda_stream
    if saved is None:
        _lib.check(lib.msbm_zncc_softargmax_bwd(_p(left), _p(right), b, h, w, window, ndisp,
                                                float(temperature), float(eps), _p(d), _p(m), _p(l), _p(g),
                                                _p(gl), _p(gr), _p(ws), nbytes, ctypes.c_void_p(st)),
                   "msbm_zncc_softargmax_bwd")
    else:
        _lib.check(lib.msbm_zncc_softargmax_bwd_saved(_p(left), _p(right), b, h, w, window, ndisp,
                                                      float(temperature), float(eps), _p(d), _p(m), _p(l), _p(g),
                                                      _p(saved), saved.numel(), _p(gl), _p(gr), _p(ws), nbytes,
                                                      ctypes.c_void_p(st)),
                   "msbm_zncc_softargmax_bwd_saved")
    return gl, gr


def _make_function():
    torch = _torch()

    class ZnccSoftArgmax(torch.autograd.Function):
        """d_soft = sum_z z softmax_z(ZNCC_eps(left, right, z) / T) over 0 <= z <= min(ndisp-1, x)."""

        @staticmethod
        def forward(ctx, left, right, window=7, ndisp=64, temperature=0.05, eps=None, keep=True):
            eps = default_eps(window) if eps is None else eps
            left = left.contiguous()
            right = right.contiguous()
            # keep the cost volume only when a gradient will be asked for
            keep = bool(keep) and any(ctx.needs_input_grad[:2])
            d, m, l, saved = forward_raw(left, right, window, ndisp, temperature, eps, keep)
            ctx.save_for_backward(left, right, d, m, l)
            ctx.kept = saved
            ctx.cfg = (window, ndisp, temperature, eps)
            return d

        @staticmethod
        def backward(ctx, g):
            left, right, d, m, l = ctx.saved_tensors
            window, ndisp, temperature, eps = ctx.cfg
            gl, gr = backward_raw(left, right, window, ndisp, temperature, eps, d, m, l, g, ctx.kept)
            ctx.kept = None
            return gl, gr, None, None, None, None, None

    return ZnccSoftArgmax


_FN = None


def __getattr__(name):
    global _FN
    if name == "ZnccSoftArgmax":
        if _FN is None:
            _FN = _make_function()
        return _FN
    raise AttributeError(name)
