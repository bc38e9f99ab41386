"""Autotuner for the full-range ZNCC search: picks the tile width (32*sx columns) and the
z-block (candidates staged per pass) per (level size, D_k, window) by timing each candidate
on the GPU with CUDA events, and caches the choice in a JSON file.

Results never depend on the choice; only speed does.  Used by ``Context`` callers (flat
matching, the coarsest level) and to build batch plans (sx in {1, 2} there).
"""
from __future__ import annotations

import json
import os
import threading

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune_cache.json")
_lock = threading.Lock()


def _zblock_options(sx: int, dk: int):
    tx = 32 * sx
    zmax = ((256 - tx - 32) // 32) * 32
    opts = [z for z in range(32, zmax + 1, 32) if z < dk + 32]
    return opts or [32]


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_full_level(width: int, height: int, dk: int, window: int, sx_options=(1, 2, 4), reps: int = 10,
                    cache_path: str | None = _CACHE, force: bool = False):
    """Returns {"sx": .., "zblock": .., "ms": .., "table": [...]} for the fastest setting."""
    import numpy as np
    import torch

    from .msbm import Context
    name = torch.cuda.get_device_name()
    key = f"{name}|{width}x{height}|D{dk}|w{window}|sx{','.join(map(str, sx_options))}"
    if cache_path and not force:
        with _lock:
            hit = _load_cache(cache_path).get(key)
        if hit:
            return hit
    rng = np.random.default_rng(0)
    left = torch.from_numpy(rng.integers(0, 256, (height, width), dtype=np.uint8)).cuda()
    right = torch.from_numpy(rng.integers(0, 256, (height, width), dtype=np.uint8)).cuda()
    ctx = Context(width, height, dk, 1, window, 0)
    ctx.pyramid(left, right)
    table = []
    stream = torch.cuda.current_stream()
    for sx in sx_options:
        for zb in _zblock_options(sx, dk):
            ctx.set_level_tuning(0, sx, zb)
            for _ in range(3):
                ctx.match_level(0)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for e0, e1 in ev:
                e0.record(stream)
                ctx.match_level(0, with_cost=True)
                e1.record(stream)
            torch.cuda.synchronize()
            ms = sorted(e0.elapsed_time(e1) for e0, e1 in ev)[reps // 2]
            table.append({"sx": sx, "zblock": zb, "ms": ms})
    ctx.close()
    best = min(table, key=lambda t: t["ms"])
    out = {"sx": best["sx"], "zblock": best["zblock"], "ms": best["ms"], "table": table}
    if cache_path:
        with _lock:
            cache = _load_cache(cache_path)
            cache[key] = out
            _save_cache(cache_path, cache)
    return out


def level_shape(width, height, max_disp, k):
    for _ in range(k):
        width, height = (width + 1) // 2, (height + 1) // 2
    return width, height, -(-max_disp // (1 << k))


def tune_batch(specs, cache_path: str | None = _CACHE):
    """Coarsest-level (sx, zblock) for each (width, height, max_disp, levels, window, radius)."""
    sx, zb = [], []
    memo = {}
    for (w, h, d, k, win, _r) in specs:
        shape = level_shape(w, h, d, k - 1)
        key = (*shape, win)
        if key not in memo:
            memo[key] = tune_full_level(shape[0], shape[1], shape[2], win, sx_options=(1, 2), cache_path=cache_path)
        sx.append(memo[key]["sx"])
        zb.append(memo[key]["zblock"])
    return sx, zb


def tune_batch_mode(specs, lefts, rights, full_sx=None, full_zblock=None, reps: int = 10,
                    cache_path: str | None = _CACHE, force: bool = False):
    """Batch execution mode for a workload: times the persistent launch and the grouped
    launches (MSBM_FLAG_BATCH_GROUPED) on the caller's pairs with CUDA events and returns
    {"grouped": bool, "persistent_ms": .., "grouped_ms": ..}, cached by the pairs' shapes.
    Results never depend on the choice."""
    import hashlib

    import torch

    from . import _lib
    from .batch import Batch
    name = torch.cuda.get_device_name()
    shape = json.dumps([list(s) for s in specs] + [list(full_sx or []), list(full_zblock or [])])
    key = f"{name}|batchmode|{hashlib.sha256(shape.encode()).hexdigest()[:16]}"
    if cache_path and not force:
        with _lock:
            hit = _load_cache(cache_path).get(key)
        if hit:
            return hit
    stream = torch.cuda.current_stream()
    out = {}
    for nm, flags in (("persistent", 0), ("grouped", _lib.MSBM_FLAG_BATCH_GROUPED)):
        b = Batch(specs, full_sx, full_zblock, flags=flags)
        d, c = b.alloc_outputs()
        for _ in range(3):
            b.run(lefts, rights, d, c)
        b.sync()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in ev:
            e0.record(stream)
            b.run(lefts, rights, d, c)
            e1.record(stream)
        b.sync()
        out[nm + "_ms"] = sorted(e0.elapsed_time(e1) for e0, e1 in ev)[reps // 2]
        b.close()
    out["grouped"] = out["grouped_ms"] < out["persistent_ms"]
    if cache_path:
        with _lock:
            cache = _load_cache(cache_path)
            cache[key] = out
            _save_cache(cache_path, cache)
    return out
