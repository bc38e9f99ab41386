"""Batched hierarchical matching: many pairs of mixed sizes in one persistent launch.

Argument marshalling over msbm_batch_create / msbm_batch_run (see include/msbm.h); every
step runs in libmsbm's persistent kernel.  The coarsest-level tiling of each pair can be
taken from the autotuner (``paper_1901_09593_gb300.autotune``).
"""
from __future__ import annotations

import ctypes

from . import _lib


def _torch():
    import torch
    return torch


def _same(a, b) -> bool:
    """Same list of the same tensor objects (or both None)."""
    if a is None or b is None:
        return a is b
    return len(a) == len(b) and all(x is y for x, y in zip(a, b))


class Batch:
    """specs: iterable of (width, height, max_disp, levels, window, radius)."""

    def __init__(self, specs, full_sx=None, full_zblock=None, flags: int = 0):
        torch = _torch()
        self._lib = _lib.load()
        self.specs = [tuple(int(v) for v in s) for s in specs]
        n = len(self.specs)
        arr = (_lib.msbm_params * n)()
        for i, (w, h, d, k, win, r) in enumerate(self.specs):
            arr[i] = _lib.msbm_params(w, h, d, k, win, r, flags, 0.9, 0.9)
        sx = (ctypes.c_int32 * n)(*full_sx) if full_sx is not None else None
        zb = (ctypes.c_int32 * n)(*full_zblock) if full_zblock is not None else None
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._b = ctypes.c_void_p()
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _lib.check(self._lib.msbm_batch_create(arr, n, sx, zb, st, ctypes.byref(self._b)),
                   "msbm_batch_create")
        self._keep = None

    def close(self):
        if self._b:
            self._lib.msbm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n, g, s = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _lib.check(self._lib.msbm_batch_info(self._b, ctypes.byref(n), ctypes.byref(g), ctypes.byref(s)))
        return {"items": n.value, "grid": g.value, "segments": s.value}

    def alloc_outputs(self, with_cost=True):
        torch = _torch()
        d = [torch.empty((h, w), dtype=torch.int16, device=self.device) for (w, h, *_r) in self.specs]
        c = ([torch.empty((h, w), dtype=torch.float32, device=self.device) for (w, h, *_r) in self.specs]
             if with_cost else None)
        return d, c

    def run(self, lefts, rights, d_outs=None, cost_outs=None):
        """lefts/rights: lists of CUDA uint8 (H, W) tensors.  Returns (d_outs, cost_outs)."""
        torch = _torch()
        n = len(self.specs)
        if len(lefts) != n or len(rights) != n:
            raise ValueError(f"expected {n} pairs")
        if d_outs is None:
            d_outs, cost_outs = self.alloc_outputs(with_cost=True)
        else:
            self._check_outs(d_outs, cost_outs)
        for i, (w, h, *_r) in enumerate(self.specs):
            for t, nm in ((lefts[i], "left"), (rights[i], "right")):
                if not t.is_cuda or t.dtype != torch.uint8 or tuple(t.shape) != (h, w) or t.stride(1) != 1:
                    raise ValueError(f"{nm}[{i}] must be a CUDA uint8 ({h}, {w}) tensor")
            if lefts[i].stride(0) != rights[i].stride(0):
                raise ValueError("left and right of a pair must share a pitch")
        P = ctypes.c_void_p
        L = (P * n)(*[t.data_ptr() for t in lefts])
        R = (P * n)(*[t.data_ptr() for t in rights])
        pitch = (ctypes.c_size_t * n)(*[t.stride(0) for t in lefts])
        D = (P * n)(*[t.data_ptr() for t in d_outs])
        C = (P * n)(*[t.data_ptr() for t in cost_outs]) if cost_outs is not None else None
        _lib.check(self._lib.msbm_batch_run(self._b, L, R, pitch, D, C), "msbm_batch_run")
        self._keep = (lefts, rights, d_outs, cost_outs)
        return d_outs, cost_outs

    def _check_outs(self, d_outs, cost_outs):
        """The caller's output maps: dense CUDA tensors of each pair's level-0 size (the C ABI
        takes bare pointers).  The tensors of the previous call are not checked again."""
        torch = _torch()
        last = getattr(self, "_outs_ok", None)
        if last is not None and _same(last[0], d_outs) and _same(last[1], cost_outs):
            return
        n = len(self.specs)
        if len(d_outs) != n or (cost_outs is not None and len(cost_outs) != n):
            raise ValueError(f"expected {n} output maps")
        for i, (w, h, *_r) in enumerate(self.specs):
            outs = [(d_outs[i], torch.int16, "d_outs")]
            if cost_outs is not None and cost_outs[i] is not None:
                outs.append((cost_outs[i], torch.float32, "cost_outs"))
            for t, dt, nm in outs:
                if (not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dt or t.shape != (h, w)
                        or not t.is_contiguous()):
                    raise ValueError(f"{nm}[{i}] must be a dense CUDA {dt} ({h}, {w}) tensor")
        self._outs_ok = (list(d_outs), None if cost_outs is None else list(cost_outs))

    def level_result(self, pair: int, level: int):
        """(d, cost) of `pair` at `level` >= 1 from the last run (device tensors)."""
        torch = _torch()
        w, h = self.specs[pair][0], self.specs[pair][1]
        for _ in range(level):
            w, h = (w + 1) // 2, (h + 1) // 2
        d = torch.empty((h, w), dtype=torch.int16, device=self.device)
        c = torch.empty((h, w), dtype=torch.float32, device=self.device)
        _lib.check(self._lib.msbm_batch_level_result(self._b, int(pair), int(level), ctypes.c_void_p(d.data_ptr()),
                                                     ctypes.c_void_p(c.data_ptr())), "msbm_batch_level_result")
        return d, c

    def sync(self):
        _lib.check(self._lib.msbm_batch_sync(self._b), "msbm_batch_sync")

    def eval_count(self, reset=True):
        v = ctypes.c_int64()
        _lib.check(self._lib.msbm_batch_eval_count(self._b, ctypes.byref(v), int(reset)))
        return int(v.value)
