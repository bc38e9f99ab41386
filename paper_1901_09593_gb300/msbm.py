"""PyTorch-facing wrapper of the C ABI: argument marshalling only.

Every step of the computation runs in libmsbm's CUDA kernels; this module checks tensor
types and shapes, allocates outputs with PyTorch, passes raw device pointers and the
current CUDA stream, and maps status codes to exceptions.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


def _torch():
    import torch
    return torch


def _stream_ptr(device) -> int:
    torch = _torch()
    return int(torch.cuda.current_stream(device).cuda_stream)


def _check_map(t, w: int, h: int, dtype, name: str) -> None:
    """A dense (h, w) CUDA tensor of `dtype`: the C ABI takes such maps as bare pointers and
    cannot check their size."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{name} must be a CUDA {dtype} tensor")
    if t.shape != (h, w) or not t.is_contiguous():
        raise ValueError(f"{name} must be a dense ({h}, {w}) tensor")


def _check_image(t, w: int, h: int, name: str) -> int:
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8:
        raise TypeError(f"{name} must be a CUDA uint8 tensor")
    if t.dim() != 2 or t.shape[0] != h or t.shape[1] != w or t.stride(1) != 1:
        raise ValueError(f"{name} must be ({h}, {w}) with unit column stride")
    return int(t.stride(0))


class Context:
    """A hierarchical ZNCC block matcher for one image size and parameter set."""

    def __init__(self, width: int, height: int, max_disp: int, levels: int, window: int,
                 radius: int, flags: int = 0, device=None, alpha: float = 0.9, beta: float = 0.9):
        torch = _torch()
        self._lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index)
        self.params = _lib.msbm_params(width, height, max_disp, levels, window, radius, flags, alpha, beta)
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.msbm_create(ctypes.byref(self.params),
                                             ctypes.c_void_p(_stream_ptr(self.device)),
                                             ctypes.byref(self._ctx)), "msbm_create")
        self.width, self.height, self.levels = width, height, levels
        self._outs_ok = (None, None)     # the caller's output tensors last checked

    # -- lifetime ---------------------------------------------------------------------
    def close(self) -> None:
        if self._ctx:
            self._lib.msbm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check_outs(self, d_out, cost_out) -> None:
        """Level-0 output maps given by the caller; the tensors of the previous call are not
        checked again (repeated calls with the same outputs stay cheap)."""
        if d_out is self._outs_ok[0] and cost_out is self._outs_ok[1]:
            return
        torch = _torch()
        if d_out is not None:
            _check_map(d_out, self.width, self.height, torch.int16, "d_out")
        if cost_out is not None:
            _check_map(cost_out, self.width, self.height, torch.float32, "cost_out")
        self._outs_ok = (d_out, cost_out)

    def _bind_stream(self) -> None:
        _lib.check(self._lib.msbm_set_stream(self._ctx, ctypes.c_void_p(_stream_ptr(self.device))))

    # -- queries ----------------------------------------------------------------------
    def level_shape(self, level: int):
        w, h, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _lib.check(self._lib.msbm_level_shape(self._ctx, level, ctypes.byref(w), ctypes.byref(h),
                                              ctypes.byref(d)), "msbm_level_shape")
        return w.value, h.value, d.value

    def set_level_tuning(self, level: int, sx: int, zblock: int = 0) -> None:
        """Full-range tile width 32*sx and z-block at `level` (speed only)."""
        _lib.check(self._lib.msbm_set_level_tuning(self._ctx, level, sx, zblock), "msbm_set_level_tuning")

    def sync(self) -> None:
        _lib.check(self._lib.msbm_sync(self._ctx), "msbm_sync")

    def eval_count(self, reset: bool = True) -> int:
        v = ctypes.c_int64()
        _lib.check(self._lib.msbm_eval_count(self._ctx, ctypes.byref(v), int(reset)), "msbm_eval_count")
        return int(v.value)

    def pass_kernel_count(self) -> int:
        """Kernel launches of one disparity() call (the captured pass graph's kernel nodes)."""
        v = ctypes.c_int32()
        _lib.check(self._lib.msbm_pass_kernel_count(self._ctx, ctypes.byref(v)), "msbm_pass_kernel_count")
        return int(v.value)

    # -- steps ------------------------------------------------------------------------
    def pyramid(self, left, right) -> None:
        self._bind_stream()
        pitch = _check_image(left, self.width, self.height, "left")
        if _check_image(right, self.width, self.height, "right") != pitch:
            raise ValueError("left and right must share a row pitch")
        _lib.check(self._lib.msbm_pyramid(self._ctx, ctypes.c_void_p(left.data_ptr()),
                                          ctypes.c_void_p(right.data_ptr()), pitch), "msbm_pyramid")

    def level_image(self, level: int, which: int):
        torch = _torch()
        self._bind_stream()
        w, h, _ = self.level_shape(level)
        out = torch.empty((h, w), dtype=torch.uint8, device=self.device)
        _lib.check(self._lib.msbm_level_image(self._ctx, level, which, ctypes.c_void_p(out.data_ptr())),
                   "msbm_level_image")
        return out

    def match_level(self, level: int, prior=None, with_cost: bool = True):
        torch = _torch()
        self._bind_stream()
        w, h, _ = self.level_shape(level)
        pp = None
        if prior is not None:
            wp, hp = (w + 1) // 2, (h + 1) // 2
            if (not prior.is_cuda or prior.dtype != torch.int16 or tuple(prior.shape) != (hp, wp)
                    or not prior.is_contiguous()):
                raise ValueError(f"prior must be a contiguous CUDA int16 tensor of shape ({hp}, {wp})")
            pp = ctypes.c_void_p(prior.data_ptr())
        d = torch.empty((h, w), dtype=torch.int16, device=self.device)
        c = torch.empty((h, w), dtype=torch.float32, device=self.device) if with_cost else None
        _lib.check(self._lib.msbm_match_level(self._ctx, level, pp, ctypes.c_void_p(d.data_ptr()),
                                              ctypes.c_void_p(c.data_ptr()) if c is not None else None),
                   "msbm_match_level")
        return d, c

    def alpha_refine(self, level: int, d, cost) -> None:
        """Eq. 5-7 in place on (d, cost) of `level` (pyramid from pyramid())."""
        torch = _torch()
        w, h, _ = self.level_shape(level)
        _check_map(d, w, h, torch.int16, "d")
        _check_map(cost, w, h, torch.float32, "cost")
        self._bind_stream()
        _lib.check(self._lib.msbm_alpha_refine(self._ctx, level, ctypes.c_void_p(d.data_ptr()),
                                               ctypes.c_void_p(cost.data_ptr())), "msbm_alpha_refine")

    def selective_median(self, level: int, d, cost):
        """Eq. 10: returns the filtered map."""
        torch = _torch()
        w, h, _ = self.level_shape(level)
        _check_map(d, w, h, torch.int16, "d")
        _check_map(cost, w, h, torch.float32, "cost")
        self._bind_stream()
        out = torch.empty_like(d)
        _lib.check(self._lib.msbm_selective_median(self._ctx, level, ctypes.c_void_p(d.data_ptr()),
                                                   ctypes.c_void_p(cost.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr())), "msbm_selective_median")
        return out

    def match_level_beta(self, level: int, prior, cost_prior):
        """Eq. 8-9 (both branches): returns (d, cost, fallback mask)."""
        torch = _torch()
        self._bind_stream()
        w, h, _ = self.level_shape(level)
        _check_map(prior, (w + 1) // 2, (h + 1) // 2, torch.int16, "prior")
        _check_map(cost_prior, (w + 1) // 2, (h + 1) // 2, torch.float32, "cost_prior")
        d = torch.empty((h, w), dtype=torch.int16, device=self.device)
        c = torch.empty((h, w), dtype=torch.float32, device=self.device)
        fb = torch.empty((h, w), dtype=torch.uint8, device=self.device)
        _lib.check(self._lib.msbm_match_level_beta(
            self._ctx, level, ctypes.c_void_p(prior.data_ptr()), ctypes.c_void_p(cost_prior.data_ptr()),
            ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(fb.data_ptr())),
            "msbm_match_level_beta")
        return d, c, fb

    def disparity(self, left, right, d_out=None, cost_out=None, with_cost: bool = True):
        """Whole hierarchical pass on device tensors; returns level-0 (d, cost)."""
        torch = _torch()
        self._bind_stream()
        pitch = _check_image(left, self.width, self.height, "left")
        if _check_image(right, self.width, self.height, "right") != pitch:
            raise ValueError("left and right must share a row pitch")
        self._check_outs(d_out, cost_out)
        if d_out is None:
            d_out = torch.empty((self.height, self.width), dtype=torch.int16, device=self.device)
        if cost_out is None and with_cost:
            cost_out = torch.empty((self.height, self.width), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.msbm_disparity(self._ctx, ctypes.c_void_p(left.data_ptr()),
                                            ctypes.c_void_p(right.data_ptr()), pitch,
                                            ctypes.c_void_p(d_out.data_ptr()),
                                            ctypes.c_void_p(cost_out.data_ptr()) if cost_out is not None else None),
                   "msbm_disparity")
        return d_out, cost_out

    def disparity_host(self, left: np.ndarray, right: np.ndarray, d_out: np.ndarray | None = None,
                       cost_out: np.ndarray | None = None):
        """Whole pass on host arrays, waiting for the result: the images are copied into device
        staging buffers and the maps copied back (asynchronous DMA for page-locked arrays)."""
        self._bind_stream()
        for a, nm in ((left, "left"), (right, "right")):
            if a.dtype != np.uint8 or a.shape != (self.height, self.width) or a.strides[1] != 1:
                raise ValueError(f"{nm} must be uint8 ({self.height}, {self.width})")
        if left.strides[0] != right.strides[0]:
            raise ValueError("left and right must share a row pitch")
        if d_out is None:
            d_out = np.empty((self.height, self.width), np.int16)
        if d_out.dtype != np.int16 or d_out.shape != (self.height, self.width) or not d_out.flags.c_contiguous:
            raise ValueError(f"d_out must be a dense int16 ({self.height}, {self.width}) array")
        if cost_out is not None and (cost_out.dtype != np.float32 or cost_out.shape != (self.height, self.width)
                                     or not cost_out.flags.c_contiguous):
            raise ValueError(f"cost_out must be a dense float32 ({self.height}, {self.width}) array")
        _lib.check(self._lib.msbm_disparity_host(
            self._ctx, left.ctypes.data, right.ctypes.data, left.strides[0], d_out.ctypes.data,
            cost_out.ctypes.data if cost_out is not None else None), "msbm_disparity_host")
        return d_out, cost_out

    def disparity_host_frames(self, lefts, rights, d_outs, cost_outs=None):
        """A sequence of pairs in host arrays, pipelined (msbm_disparity_host_frames): frame
        i+1's upload and frame i-1's download overlap frame i's pass when the arrays are
        page-locked.  Waits for the last frame; returns (d_outs, cost_outs)."""
        self._bind_stream()
        n = len(lefts)
        if n < 1 or len(rights) != n or len(d_outs) != n or (cost_outs is not None and len(cost_outs) != n):
            raise ValueError("lefts, rights, d_outs (and cost_outs) must be equally long and non-empty")
        pitch = lefts[0].strides[0]
        for i in range(n):
            for a, nm in ((lefts[i], "left"), (rights[i], "right")):
                if a.dtype != np.uint8 or a.shape != (self.height, self.width) or a.strides[1] != 1 \
                        or a.strides[0] != pitch:
                    raise ValueError(f"{nm}[{i}] must be uint8 ({self.height}, {self.width}) at one row pitch")
            if d_outs[i].dtype != np.int16 or d_outs[i].shape != (self.height, self.width) \
                    or not d_outs[i].flags.c_contiguous:
                raise ValueError(f"d_outs[{i}] must be a dense int16 ({self.height}, {self.width}) array")
            c = None if cost_outs is None else cost_outs[i]
            if c is not None and (c.dtype != np.float32 or c.shape != (self.height, self.width)
                                  or not c.flags.c_contiguous):
                raise ValueError(f"cost_outs[{i}] must be a dense float32 ({self.height}, {self.width}) array")
        P = ctypes.c_void_p
        L = (P * n)(*[a.ctypes.data for a in lefts])
        R = (P * n)(*[a.ctypes.data for a in rights])
        D = (P * n)(*[a.ctypes.data for a in d_outs])
        C = None if cost_outs is None else (P * n)(*[None if c is None else c.ctypes.data for c in cost_outs])
        _lib.check(self._lib.msbm_disparity_host_frames(self._ctx, n, L, R, pitch, D, C),
                   "msbm_disparity_host_frames")
        return d_outs, cost_outs

    def profile_disparity(self, left, right, d_out, cost_out):
        """One pass with per-stage CUDA-event timing; returns the list of milliseconds in
        launch order (pyramid, statistics planes, coarsest full search, restricted levels
        K-2..0)."""
        torch = _torch()
        self._bind_stream()
        pitch = _check_image(left, self.width, self.height, "left")
        if _check_image(right, self.width, self.height, "right") != pitch:
            raise ValueError("left and right must share a row pitch")
        _check_map(d_out, self.width, self.height, torch.int16, "d_out")
        if cost_out is not None:
            _check_map(cost_out, self.width, self.height, torch.float32, "cost_out")
        n = self.levels + 2
        ms = (ctypes.c_float * n)()
        _lib.check(self._lib.msbm_profile_disparity(
            self._ctx, ctypes.c_void_p(left.data_ptr()), ctypes.c_void_p(right.data_ptr()), pitch,
            ctypes.c_void_p(d_out.data_ptr()),
            ctypes.c_void_p(cost_out.data_ptr()) if cost_out is not None else None, ms, n),
            "msbm_profile_disparity")
        return [float(v) for v in ms]

    def stage_names(self):
        k, f = self.levels, self.params.flags
        top = f"full_level{k - 1}" + ("+alpha" if f & _lib.MSBM_FLAG_ALPHA_REFINE else "")
        fin = (("+beta" if f & _lib.MSBM_FLAG_BETA_FALLBACK else "")
               + ("+median" if f & _lib.MSBM_FLAG_SELECTIVE_MEDIAN else ""))
        return (["pyramid", "statistics"] + [top] + [f"restricted_level{i}{fin}" for i in range(k - 2, -1, -1)])

    def level_result(self, level: int):
        """Copies of an intermediate level's (d, cost) from the last disparity()."""
        torch = _torch()
        self._bind_stream()
        w, h, _ = self.level_shape(level)
        d = torch.empty((h, w), dtype=torch.int16, device=self.device)
        c = torch.empty((h, w), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.msbm_level_result(self._ctx, level, ctypes.c_void_p(d.data_ptr()),
                                               ctypes.c_void_p(c.data_ptr())), "msbm_level_result")
        return d, c
