#!/usr/bin/env python
"""Throughput of multi-scale hierarchical ZNCC block matching on one GB300 per rank.

Workload: the 1400x1000 benchmark-shaped pair (seeded synthetic slanted-plane scene, 12
regions, noise sigma 3), D = 256, K = 4 pyramid levels, 7x7 window, refinement radius 2.
A step is one whole hierarchical pass (pyramid, coarsest full search, three restricted
levels) on one pair already resident in HBM; the L2 is flushed between steps (the pair
is smaller than L2).  Flat full-range 7x7 block matching (K = 1) is timed on the same
pair for comparison, and both maps are scored against the ground truth.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun each rank matches its own pair (seed =
rank): weak scaling, no data-path collective; only the timings are reduced (max).
`--impl reference` times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "bench_1400x1000"
METRIC = "Gpix·disp/s and frames/s, hierarchical vs flat ZNCC BM, same bad-pixel rate"
L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------------------------------
# distributed plumbing (host side only: rank discovery, barrier, max-reduction)
# ---------------------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(value: float, dist, device=None) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def pair_seed(rank: int) -> int:
    """Each rank matches its own independent pair (weak scaling)."""
    return rank


# ---------------------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [ln.split(",") for ln in open(self.path).read().strip().splitlines() if ln.strip()]
            os.unlink(self.path)
        except OSError:
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            busy = [s for s in sm if s > 0.5 * max(sm)] or sm
            out = {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ---------------------------------------------------------------------------------------
# roofline accounting
# ---------------------------------------------------------------------------------------
def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# One "op" is one 32-bit lane instruction.  Nominal issue peak: SMs x 128 lanes x max SM
# clock (one warp instruction per clock per SM sub-partition), an upper bound for every pipe.
def alu_peak_tops(sms: int, mhz: float) -> float:
    return sms * 128 * mhz * 1e6 / 1e12


def dp4a_per_eval(window: int) -> int:
    # the direct window: one 4-way byte dot product per 4 window bytes per row (the method's
    # sum of products; the remaining per-evaluation terms are a handful of scalar operations)
    return window * ((window + 3) // 4)


def ops_per_eval_restricted(window: int) -> int:
    # dp4a for the window plus the exact int32 combine, int-to-float, two scalings, compare
    return dp4a_per_eval(window) + 5


OPS_PER_EVAL_FULL = 8   # sliding sums: 2 vertical + 2 horizontal, c (2), scale (1), compare (1)

PROBE_KINDS = {"dp4a": 0, "funnel_shift": 1, "ffma": 2, "int_add_logic": 3, "lds32": 4}


def measure_pipe_peaks(sms: int, stream, target_ms: float = 25.0) -> dict:
    """Issue rates of the instruction classes the matching kernels use, measured on this GPU
    with msbm_pipe_probe (8 CTAs of 256 threads per SM), best of three runs each."""
    import ctypes

    from paper_1901_09593_gb300 import _lib
    lib = _lib.load()
    out = {}
    for name, kind in PROBE_KINDS.items():
        ms, ops = ctypes.c_float(), ctypes.c_double()

        def run(iters):
            _lib.check(lib.msbm_pipe_probe(kind, sms * 8, iters, ctypes.c_void_p(stream.cuda_stream),
                                           ctypes.byref(ms), ctypes.byref(ops)), "msbm_pipe_probe")
            return ms.value, ops.value
        t, _ = run(64)
        iters = max(64, int(64 * target_ms / max(t, 1e-3)))
        best = max(o / (t_ * 1e-3) for t_, o in (run(iters) for _ in range(3)))
        out[name] = {"lane_ops_per_s": best, "iters": iters, "ctas": sms * 8}
    return out


def stage_work(name, spec, levels_wh, evals_by_level):
    """(bound, algorithmic amount, unit) of one stage of the pass: HBM bytes for the pyramid,
    dp4a lane operations (the window's sum of products) for the matching levels."""
    if name == "pyramid":
        # read both input images once, write every level's apron buffer of both images
        w0, h0 = levels_wh[0]
        return "hbm", 2 * w0 * h0 + sum(2 * (w + 32) * (h + 16) for w, h in levels_wh), "B"
    if name == "statistics":
        # read the right image of levels 0..K-2 and write their 8-byte statistics planes
        return "hbm", sum(9 * w * h for w, h in levels_wh[:-1]), "B"
    k = int(name[len("full_level"):]) if name.startswith("full_level") else int(name[len("restricted_level"):])
    return "dp4a", evals_by_level[k] * dp4a_per_eval(spec.window), "dp4a"


# DRAM bytes (read + write) per launch from one committed ncu capture of a kernel, valid
# while the sources it was taken on are unchanged: the key is a SHA-256 prefix of those
# files.  A constant, not a measurement of this run; null once the sources change.
# frames per end-to-end run: a stream long enough that the pipeline's fill and drain (about
# two frames) do not set the rate
E2E_MIN_FRAMES = 128

MEASURED_TRAFFIC = {
    "restricted_level0": {"files": ["zncc_restricted.cu", "zncc_cell_tile.cuh", "msbm_device.cuh",
                                    "msbm_internal.h"],
                          "sha256_16": "8cc262a182bf6f7f", "bytes": 13223936},
}


def measured_traffic(kernel):
    import hashlib
    rec = MEASURED_TRAFFIC.get(kernel)
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in rec["files"]:
        with open(os.path.join(ROOT, "paper_1901_09593_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sha256_16"] else None


def equal_or_better(methods, flat_fps, flat_bad1):
    """The fastest measured hierarchical method whose bad-1 rate is at most flat matching's."""
    ok = [(v["frames_per_s"], k, v) for k, v in methods.items()
          if "frames_per_s" in v and v.get("bad1", 1.0) <= flat_bad1]
    if not ok:
        return None
    f, k, v = max(ok)
    return {"method": k, "frames_per_s": f, "bad1": v["bad1"], "flat_frames_per_s": flat_fps,
            "flat_bad1": flat_bad1, "speedup": f / flat_fps}


def full_evals(w, h, dk):
    return sum(min(dk - 1, x) + 1 for x in range(w)) * h


def restricted_evals(prior, w, h, dk, r):
    import numpy as np
    yy, xx = np.mgrid[0:h, 0:w]
    zmax = np.minimum(dk - 1, xx)
    dh = np.clip(2 * prior[yy // 2, xx // 2].astype(np.int64), 0, zmax)
    lo = np.maximum(0, dh - r)
    hi = np.minimum(zmax, dh + r)
    return int((hi - lo + 1).sum())


# ---------------------------------------------------------------------------------------
# oracle (CPU baseline)
# ---------------------------------------------------------------------------------------
def time_oracle(sc, budget_s: float, min_runs: int = 1):
    import oracle
    s = sc.spec
    oracle.build()
    runs, t0 = 0, time.perf_counter()
    while True:
        oracle.disparity(sc.left, sc.right, s.max_disp, s.levels, s.window, s.radius)
        runs += 1
        el = time.perf_counter() - t0
        if runs >= min_runs and el >= budget_s:
            break
    return runs, el, oracle.max_threads()


def oracle_side_samples(sc, cores: int) -> dict:
    """One flat (K = 1) oracle frame on all host cores and one hierarchical frame on one
    core, for context beside the baseline (a few seconds in all)."""
    import oracle
    s = sc.spec
    t0 = time.perf_counter()
    oracle.disparity(sc.left, sc.right, s.max_disp, 1, s.window, s.radius)
    flat_s = time.perf_counter() - t0
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.disparity(sc.left, sc.right, s.max_disp, s.levels, s.window, s.radius)
        one_s = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return {"flat_frames_per_s": 1.0 / flat_s, "hier_one_core_frames_per_s": 1.0 / one_s,
            "side_samples": "one flat K = 1 frame on all cores; one hierarchical frame on one core"}


def reference_rows(height: int, levels: int, t_frame: float, n_runs: int, budget_s: float) -> int:
    """Rows of the frame each reference step processes: the whole frame when n_runs frames fit
    the time budget, else the largest band from the top that does, in multiples of
    2^(levels-1) rows (every row costs about the same: the candidate sets depend on x and on
    the coarser maps only)."""
    if n_runs * t_frame <= budget_s:
        return height
    unit = 1 << (levels - 1)
    rows = int(height * budget_s / (n_runs * t_frame)) // unit * unit
    return min(height, max(unit, rows))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1901_09593_gb300 import scenes
    spec = scenes.SPECS[WORKLOAD]
    sc = scenes.make_pair(spec, pair_seed(0))
    oracle.build()
    t0 = time.perf_counter()
    oracle.disparity(sc.left, sc.right, spec.max_disp, spec.levels, spec.window, spec.radius)
    t_frame = time.perf_counter() - t0
    rows = reference_rows(spec.height, spec.levels, t_frame, args.warmup + args.steps, args.ref_budget)
    left, right = sc.left[:rows].copy(), sc.right[:rows].copy()
    for _ in range(args.warmup - 1):
        oracle.disparity(left, right, spec.max_disp, spec.levels, spec.window, spec.radius)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.disparity(left, right, spec.max_disp, spec.levels, spec.window, spec.radius)
    el = time.perf_counter() - t0
    fps = args.steps * rows / spec.height / el
    cores = oracle.max_threads()
    what = "full-frame hierarchical passes" if rows == spec.height else \
        f"hierarchical passes over rows 0..{rows - 1} (a {rows}/{spec.height} band of the frame; frames/s scaled by it)"
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(spec),
        "cpu_baseline": {"kind": "oracle", "value": fps, "unit": "frames/s", "cores": cores,
                         "sample": f"{args.steps} {what} of the "
                                   f"{spec.width}x{spec.height} pair, FP64 C oracle, OpenMP"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_pair(args, dev, flush, stream, name, what):
    """One seeded pair of a named workload: hierarchical (plain and with the selective
    median) and flat full-range matching, each timed with CUDA events (median step)."""
    import torch

    from paper_1901_09593_gb300 import Context, _lib, scenes
    spec = scenes.SPECS[name]
    sc = scenes.make_pair(spec, 0)
    L = torch.from_numpy(sc.left).to(dev)
    R = torch.from_numpy(sc.right).to(dev)
    res = {"workload": f"{name}: {what}"}
    for name, levels, flags in (("hierarchical", spec.levels, 0),
                                ("selective_median", spec.levels, _lib.MSBM_FLAG_SELECTIVE_MEDIAN),
                                ("flat", 1, 0)):
        ctx = Context(spec.width, spec.height, spec.max_disp, levels, spec.window, spec.radius, flags)
        d = torch.empty((spec.height, spec.width), dtype=torch.int16, device=dev)
        c = torch.empty((spec.height, spec.width), dtype=torch.float32, device=dev)
        for _ in range(3):
            ctx.disparity(L, R, d, c)
        ctx.sync()
        steps = (5 if spec.width * spec.height > 4e6 else 20) if levels == 1 else max(5, min(args.steps, 30))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            ctx.disparity(L, R, d, c)
            e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)
        dh = d.cpu().numpy()
        res[name] = {"frames_per_s": 1e3 / ms, "ms_per_frame": ms,
                     "bad1": scenes.bad_rate(dh, sc.gt, sc.mask, 1.0), "bad2": scenes.bad_rate(dh, sc.gt, sc.mask, 2.0)}
        ctx.close()
    res["hier_over_flat_speedup"] = res["hierarchical"]["frames_per_s"] / res["flat"]["frames_per_s"]
    return res


def bench_batch(args, dev, flush, stream):
    """48 seeded pairs of mixed sizes (each its own scene) through one batch pass: the
    persistent launch and the grouped launches, the mode the autotuner picks being the
    batch's number; against the same pairs through 48 single-pair graphs in sequence."""
    import torch

    from paper_1901_09593_gb300 import Batch, Context, _lib, autotune, scenes

    def timed_ms(fn, steps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        for _ in range(4):
            flush.zero_()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        return statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)

    def run_set(specs_s, seed0):
        specs = [(s.width, s.height, s.max_disp, s.levels, s.window, s.radius) for s in specs_s]
        scs = [scenes.make_pair(s, seed0 + i) for i, s in enumerate(specs_s)]
        Ls = [torch.from_numpy(sc.left).to(dev) for sc in scs]
        Rs = [torch.from_numpy(sc.right).to(dev) for sc in scs]
        sx, zb = autotune.tune_batch(specs)
        mode = autotune.tune_batch_mode(specs, Ls, Rs, sx, zb)
        steps = max(5, min(args.steps, 30))
        res = {}
        for nm, fl in (("persistent", 0), ("grouped", _lib.MSBM_FLAG_BATCH_GROUPED)):
            b = Batch(specs, sx, zb, flags=fl)
            d, c = b.alloc_outputs()
            res[nm + "_ms"] = timed_ms(lambda: b.run(Ls, Rs, d, c), steps)
            if nm == "persistent":
                info = b.info()
            b.sync()
            b.eval_count(reset=True)
            b.run(Ls, Rs, d, c)
            b.sync()
            res["evals_per_batch"] = b.eval_count(reset=True)
            b.close()
        ctxs = [Context(*sp) for sp in specs]
        d1 = [torch.empty((sp[1], sp[0]), dtype=torch.int16, device=dev) for sp in specs]
        c1 = [torch.empty((sp[1], sp[0]), dtype=torch.float32, device=dev) for sp in specs]

        def seq():
            for i, cx in enumerate(ctxs):
                cx.disparity(Ls[i], Rs[i], d1[i], c1[i])
        res["sequential_contexts_ms"] = timed_ms(seq, steps)
        for cx in ctxs:
            cx.close()
        chosen = "grouped" if mode["grouped"] else "persistent"
        res.update({"mode": chosen, "autotune": mode, "ms_per_batch": res[chosen + "_ms"],
                    "pairs_per_s": len(specs) / (res[chosen + "_ms"] * 1e-3),
                    "speedup_vs_sequential": res["sequential_contexts_ms"] / res[chosen + "_ms"],
                    "steps": steps})
        return res, info

    specs_s = scenes.make_batch_specs(48, 0)
    res, info = run_set(specs_s, 2000)
    res["gpix_disp_per_s"] = res["evals_per_batch"] / (res["ms_per_batch"] * 1e-3) / 1e9
    res.update({"workload": "48 seeded mixed-size pairs (320x240 .. 1920x1080, each its own scene, D = W/5, "
                            "K to width >= 160, window 5/7, r = 2)",
                "queue_items": info["items"], "grid_ctas": info["grid"]})
    small = [s for s in specs_s if s.width == 320]
    if small:
        small = (small * (48 // len(small) + 1))[:48]
        sres, _ = run_set(small, 3000)
        sres["workload"] = "48 pairs 320x240, each its own scene (D = 64, K = 2, window 5/7 as drawn, r = 2)"
        res["small_pairs"] = sres
    return res


def bench_diff(args, dev, flush, stream, pipes=None):
    """Soft-argmax ZNCC level forward + backward, 8 x 640 x 480, 64 candidates, 7x7, T=0.05:
    through the autograd.Function (forward_ms, forward_backward_ms), and each launch of the
    C ABI alone with its roofline (forward against the measured FFMA rate, backward against
    HBM)."""
    import numpy as np
    import torch

    from paper_1901_09593_gb300 import scenes
    from paper_1901_09593_gb300.softargmax import ZnccSoftArgmax, default_eps
    spec = scenes.SPECS["diff_640x480"]
    pairs = [scenes.make_float_pair(spec, s) for s in range(8)]
    L = torch.tensor(np.stack([p.left for p in pairs]), dtype=torch.float32, device=dev)
    R = torch.tensor(np.stack([p.right for p in pairs]), dtype=torch.float32, device=dev)
    g = torch.ones_like(L)

    def step():
        lt = L.detach().requires_grad_(True)
        rt = R.detach().requires_grad_(True)
        out = ZnccSoftArgmax.apply(lt, rt, 7, 64, 0.05, default_eps(7))
        out.backward(g)
        return out

    def fwd():
        with torch.no_grad():
            return ZnccSoftArgmax.apply(L, R, 7, 64, 0.05, default_eps(7))

    res = {}
    for name, fn in (("forward", fwd), ("forward_backward", step)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        steps = max(3, min(args.steps, 10))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name + "_ms"] = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)
    evals = 8 * 480 * sum(min(63, x) + 1 for x in range(640))
    res.update({"workload": "8 x 640 x 480 float32 pairs, 7x7 ZNCC over 64 candidates, soft-argmax T=0.05",
                "evals": evals, "forward_gpix_disp_per_s": evals / (res["forward_ms"] * 1e-3) / 1e9})
    # the two C-ABI calls of a training step, each timed alone (the forward keeping the cost
    # volume and window statistics, the backward reading them)
    from paper_1901_09593_gb300.softargmax import backward_raw, forward_raw
    eps = default_eps(7)
    kept = {}

    def fwd_keep():
        kept["v"] = forward_raw(L, R, 7, 64, 0.05, eps, True)

    def bwd_kept():
        d, m, l, sv = kept["v"]
        backward_raw(L, R, 7, 64, 0.05, eps, d, m, l, g, sv)

    for name, fn in (("forward_kept", fwd_keep), ("backward_kept", bwd_kept)):
        fn()
        torch.cuda.synchronize(dev)
        steps = max(3, min(args.steps, 10))
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        res[name + "_ms"] = statistics.median(ts)
    # roofline: the forward's 49 FFMA per evaluation (the window product; the score and the
    # online softmax add a few more) against the measured FFMA rate; the backward's bytes
    # per evaluation against HBM: the kept rho read and alpha written by the coefficient
    # kernel (8 B), alpha read by the gradient kernel with its tile halo ((32+6)^2/32^2 x 4 B)
    ffma = (pipes or {}).get("ffma", {}).get("lane_ops_per_s")
    peaks = load_peaks() or {}
    hbm = peaks.get("hbm_gbs") or 6800.0
    fwd_rate = evals * 49 / (res["forward_kept_ms"] * 1e-3)
    bwd_bytes = evals * (8 + 4 * 38 * 38 / (32 * 32))
    res["roofline"] = {
        "forward": {"bound": "ffma", "achieved": fwd_rate / 1e12, "unit": "T FFMA/s",
                    "peak": ffma / 1e12 if ffma else None, "frac": fwd_rate / ffma if ffma else None},
        "backward": {"bound": "hbm", "achieved": bwd_bytes / (res["backward_kept_ms"] * 1e-3) / 1e9,
                     "unit": "GB/s", "peak": hbm,
                     "frac": bwd_bytes / (res["backward_kept_ms"] * 1e-3) / 1e9 / hbm,
                     "algorithmic_bytes": bwd_bytes}}
    return res


def _flat_and_methods(args, sc, L, R, d, c, timed, methods):
    """Flat K = 1 matching and the gated methods on the benchmark pair (rows of the line
    beside the timed hierarchical pass)."""
    import torch

    from paper_1901_09593_gb300 import Context, _lib, scenes
    spec = sc.spec
    W, H = spec.width, spec.height
    flat = Context(W, H, spec.max_disp, 1, spec.window, spec.radius)
    # the flat baseline at its autotuned tiling (tile width 32*sx, z-block)
    from paper_1901_09593_gb300 import autotune
    tune = autotune.tune_full_level(W, H, spec.max_disp, spec.window)
    flat.set_level_tuning(0, tune["sx"], tune["zblock"])
    df = torch.empty_like(d)
    cf = torch.empty_like(c)
    fsteps = max(3, min(args.steps, 20))
    fms = timed(lambda: flat.disparity(L, R, df, cf), fsteps, max(3, args.warmup // 2))
    flat.sync()
    flat_fps = fsteps / (sum(fms) / 1e3)
    flat_evals = full_evals(W, H, spec.max_disp)
    df_h = df.cpu().numpy()
    bad1_f = scenes.bad_rate(df_h, sc.gt, sc.mask, 1.0)
    bad2_f = scenes.bad_rate(df_h, sc.gt, sc.mask, 2.0)

    # -- the gated steps of the full method on the same pair (Sec. III-B/C/D)
    for name, fl in (("selective_median", _lib.MSBM_FLAG_SELECTIVE_MEDIAN),
                     ("full_method", _lib.MSBM_FLAGS_FULL_METHOD),
                     ("window_halving", _lib.MSBM_FLAG_WINDOW_HALVING),
                     ("full_method_window_halving", _lib.MSBM_FLAGS_FULL_METHOD | _lib.MSBM_FLAG_WINDOW_HALVING)):
        cx = Context(W, H, spec.max_disp, spec.levels, spec.window, spec.radius, fl, alpha=0.9, beta=0.9)
        dm = torch.empty_like(d)
        cm = torch.empty_like(c)
        msteps = max(3, min(args.steps, 50))
        mms = timed(lambda: cx.disparity(L, R, dm, cm), msteps, max(3, args.warmup // 2))
        cx.sync()
        cx.eval_count(reset=True)
        cx.disparity(L, R, dm, cm)
        ev_m = cx.eval_count(reset=True)
        dmh = dm.cpu().numpy()
        prof = [cx.profile_disparity(L, R, dm, cm) for _ in range(5)]
        methods[name] = {"frames_per_s": msteps / (sum(mms) / 1e3), "ms_per_frame": sum(mms) / msteps,
                         "evals_per_frame": ev_m, "bad1": scenes.bad_rate(dmh, sc.gt, sc.mask, 1.0),
                         "bad2": scenes.bad_rate(dmh, sc.gt, sc.mask, 2.0), "alpha": 0.9, "beta": 0.9,
                         "stages_ms": {nm: round(statistics.mean(v), 5)
                                       for nm, v in zip(cx.stage_names(), zip(*prof))}}
        cx.close()
    flat.close()
    methods["_flat_tuning"] = {"sx": tune["sx"], "zblock": tune["zblock"]}
    return flat_fps, bad1_f, bad2_f, fsteps


def config_dict(spec):
    return {"workload": f"{WORKLOAD}: hierarchical ZNCC BM, {spec.width}x{spec.height} uint8 pair, "
                        f"D={spec.max_disp}, K={spec.levels}, {spec.window}x{spec.window} window, "
                        f"r={spec.radius}",
            "width": spec.width, "height": spec.height, "max_disp": spec.max_disp,
            "levels": spec.levels, "window": spec.window, "radius": spec.radius,
            "l2": "flushed between timed steps (256 MB write; inputs are smaller than L2)",
            "parallelism": "independent pairs per rank (weak scaling)"}


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    from paper_1901_09593_gb300 import Context, _lib, build, scenes

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    build.build()
    spec = scenes.SPECS[WORKLOAD]
    sc = scenes.make_pair(spec, pair_seed(rank))
    W, H = spec.width, spec.height
    L = torch.from_numpy(sc.left).to(dev)
    R = torch.from_numpy(sc.right).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    ctx = Context(W, H, spec.max_disp, spec.levels, spec.window, spec.radius)
    d = torch.empty((H, W), dtype=torch.int16, device=dev)
    c = torch.empty((H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        # a head start of untimed L2 flushes so that the host's launches run ahead of the GPU
        # from the first timed step on (else the first step's event pair also spans the host
        # latency of its launch call)
        for _ in range(4):
            flush.zero_()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize(dev)
        return [e0.elapsed_time(e1) for e0, e1 in ev]

    # -- flat full-range block matching on the same GPU and pair (also warms the GPU up
    # before the timed region)
    methods = {}
    flat_fps, flat_evals, bad1_f, bad2_f, fsteps = None, full_evals(W, H, spec.max_disp), None, None, 0
    if not args.no_flat:
        flat_fps, bad1_f, bad2_f, fsteps = _flat_and_methods(args, sc, L, R, d, c, timed, methods)
    # -- hierarchical, graph replay: the timed region
    for _ in range(args.warmup):
        ctx.disparity(L, R, d, c)
    ctx.sync()
    ctx.eval_count(reset=True)
    barrier(dist)
    torch.cuda.synchronize(dev)
    clk = ClockSampler(local)
    clk.start()
    wall0 = time.perf_counter()
    ms = timed(lambda: ctx.disparity(L, R, d, c), args.steps, 0)
    wall = time.perf_counter() - wall0
    barrier(dist)
    clocks = clk.stop()
    ctx.sync()
    evals_total = ctx.eval_count(reset=True)
    t_dev = sum(ms) / 1e3
    t_max = reduce_max(t_dev, dist, dev)
    frames = world * args.steps
    fps = frames / t_max
    evals_per_frame = evals_total / args.steps
    d_h = d.cpu().numpy()
    bad1_h = scenes.bad_rate(d_h, sc.gt, sc.mask, 1.0)
    bad2_h = scenes.bad_rate(d_h, sc.gt, sc.mask, 2.0)

    methods["plain"] = {"frames_per_s": fps / world, "ms_per_frame": 1e3 * t_max / args.steps,
                        "evals_per_frame": evals_per_frame, "bad1": bad1_h, "bad2": bad2_h}

    # -- per-kernel timing (CUDA events around each launch, same stream) -> roofline
    nprof = max(5, min(args.steps, 30))
    stage_names = ctx.stage_names()
    acc = [[] for _ in stage_names]
    for _ in range(nprof):
        flush.zero_()
        for i, v in enumerate(ctx.profile_disparity(L, R, d, c)):
            acc[i].append(v)
    stage_ms = [statistics.mean(a) for a in acc]
    levels_wh = [ctx.level_shape(k)[:2] for k in range(spec.levels)]
    evals_by_level = {}
    K = spec.levels
    wk, hk, dkk = ctx.level_shape(K - 1)
    evals_by_level[K - 1] = full_evals(wk, hk, dkk)
    for k in range(K - 2, -1, -1):
        wk, hk, dkk = ctx.level_shape(k)
        prior = ctx.level_result(k + 1)[0].cpu().numpy()
        evals_by_level[k] = restricted_evals(prior, wk, hk, dkk, spec.radius)
    peaks = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = (clocks.get("sm_max_mhz") or (peaks or {}).get("sm_max_mhz") or 2070.0)
    # measured pipe rates (the denominators of the matching stages), clocks sampled meanwhile
    pclk = ClockSampler(local)
    pclk.start()
    pipes = measure_pipe_peaks(sms, stream)
    pclocks = pclk.stop()
    pmhz = pclocks.get("sm_mhz") or sm_max
    for v in pipes.values():
        v["per_sm_per_clock"] = round(v["lane_ops_per_s"] / (sms * pmhz * 1e6), 2)
    dp4a_peak = pipes["dp4a"]["lane_ops_per_s"] / 1e12
    stages = []
    for nm, t in zip(stage_names, stage_ms):
        bound, amount, unit = stage_work(nm, spec, levels_wh, evals_by_level)
        stages.append({"kernel": nm, "ms": round(t, 5), "share": None, "bound": bound,
                       "work": amount, "work_unit": unit})
    tot = sum(stage_ms)
    hbm_peak = (peaks or {}).get("hbm_gbs") or 6800.0
    for s_ in stages:
        s_["share"] = round(s_["ms"] / tot, 4) if tot > 0 else None
        # achieved fraction of the stage's roofline (algorithmic work / event-timed duration)
        if s_["ms"] > 0:
            if s_["bound"] == "hbm":
                s_["roofline_frac"] = round(s_["work"] / (s_["ms"] * 1e-3) / 1e9 / hbm_peak, 4)
            else:
                s_["roofline_frac"] = round(s_["work"] / (s_["ms"] * 1e-3) / 1e12 / dp4a_peak, 4)
    dom = max(stages, key=lambda s_: s_["ms"])
    if dom["bound"] == "hbm":
        peak = hbm_peak
        ach = dom["work"] / (dom["ms"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s"}
    else:
        ach = dom["work"] / (dom["ms"] * 1e-3) / 1e12
        roof = {"bound": "alu", "pipe": "dp4a", "achieved": ach, "peak": dp4a_peak, "unit": "T dp4a/s",
                "frac": ach / dp4a_peak,
                "peak_source": f"measured in this run by msbm_pipe_probe (dp4a, {sms * 8} CTAs x 256 threads) "
                               f"at {pmhz:.0f} MHz median SM clock",
                # the same time against the nominal issue rate, with all of an evaluation's
                # algorithmic operations (dp4a + the scalar combine)
                "issue_frac_nominal": (dom["work"] / dp4a_per_eval(spec.window)
                                       * ops_per_eval_restricted(spec.window) / (dom["ms"] * 1e-3) / 1e12
                                       / alu_peak_tops(sms, sm_max))}
    roof["kernel"] = dom["kernel"]
    roof["traffic"] = measured_traffic(dom["kernel"])
    roof["pipes"] = pipes
    roof["pipe_clock_mhz"] = pmhz

    # -- end to end through the C ABI with pinned host buffers: a stream of frames (at least
    # E2E_MIN_FRAMES, so that the pipeline's fill and drain do not dominate) through the
    # pipelined host call (each frame's images uploaded, its pass, its disparity map
    # downloaded -- the result of record; frame i+1's upload, frame i-1's download and the
    # alternate pass pipeline's work overlap frame i's pass).  The same with the cost map
    # downloaded as well is reported beside it.
    pin_l = torch.from_numpy(sc.left).pin_memory()
    pin_r = torch.from_numpy(sc.right).pin_memory()
    pin_d = [torch.empty((H, W), dtype=torch.int16).pin_memory() for _ in range(2)]
    pin_c = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
    hl, hr = pin_l.numpy(), pin_r.numpy()
    K = max(args.steps, E2E_MIN_FRAMES)
    lefts, rights = [hl] * K, [hr] * K
    ds = [pin_d[i % 2].numpy() for i in range(K)]
    cs = [pin_c[i % 2].numpy() for i in range(K)]
    nw = max(3, args.warmup)

    def e2e_run(costs):
        ctx.disparity_host_frames(lefts[:nw], rights[:nw], ds[:nw], None if costs is None else costs[:nw])
        barrier(dist)
        t0 = time.perf_counter()
        ctx.disparity_host_frames(lefts, rights, ds, costs)
        return world * K / reduce_max(time.perf_counter() - t0, dist, dev)
    e2e_fps = e2e_run(None)
    assert np.array_equal(pin_d[(K - 1) % 2].numpy(), d_h), "pipelined host path differs from the device pass"
    e2e_cost_fps = e2e_run(cs)
    # one frame at a time (no overlap across frames), for comparison
    t0 = time.perf_counter()
    for i in range(min(K, 50)):
        ctx.disparity_host(hl, hr, ds[i], cs[i])
    e2e_single_fps = min(K, 50) / (time.perf_counter() - t0)

    # -- CPU baseline: the oracle on this host (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        runs, el, cores = time_oracle(sc, args.cpu_budget)
        cpu = {"kind": "oracle", "value": runs / el, "unit": "frames/s", "cores": cores,
               "sample": f"{runs} full-frame hierarchical passes of the {W}x{H} pair "
                         f"(FP64 C oracle, OpenMP over rows), {el:.1f} s"}
        cpu.update(oracle_side_samples(sc, cores))

    additions = {}
    if rank == 0 and not args.no_additions:
        additions["batching"] = bench_batch(args, dev, flush, stream)
        additions["differentiable"] = bench_diff(args, dev, flush, stream, pipes)
        additions["large_pair"] = bench_pair(args, dev, flush, stream, "large_2880x1984",
                                             "2880x1984 uint8 pair, D=640, K=5, 9x9 window, r=3")
        additions["small_pair"] = bench_pair(args, dev, flush, stream, "small_320x240",
                                             "320x240 uint8 pair, D=32, K=3, 5x5 window, r=2")

    launches_per_step = ctx.pass_kernel_count()
    hvf = None if flat_fps is None else equal_or_better(methods, flat_fps, bad1_f)
    # Key order: the contract's keys, then the bulky detail, then the headline comparison
    # last (a reader that keeps only the end of the line still sees it).
    line = {
        "metric": METRIC,
        "value": fps,
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": config_dict(spec),
        "gpu_launches": launches_per_step * args.steps,
        "step_ms": {"median": statistics.median(ms), "min": min(ms), "max": max(ms)},
        "wall_s_timed_region": wall,
        "additions": additions,
        "methods": methods,
        "stages": stages,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": 2 * W * H,
                "d2h_bytes_per_step": 2 * W * H, "api": "msbm_disparity_host_frames (pipelined)",
                "result": "int16 disparity map",
                "frames": K,
                "with_cost_map": {"frames_per_s": e2e_cost_fps, "d2h_bytes_per_step": W * H * (2 + 4)},
                "one_frame_per_call_with_cost_frames_per_s": e2e_single_fps},
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "gpix_disp_per_s": evals_per_frame * fps / 1e9,
        "gpix_disp_per_s_flat_equivalent": W * H * spec.max_disp * fps / 1e9,
        "evals_per_frame": evals_per_frame,
        "flat": None if flat_fps is None else {
            "frames_per_s": flat_fps, "ms_per_frame": 1e3 / flat_fps,
            "gpix_disp_per_s": flat_evals * flat_fps / 1e9, "evals_per_frame": flat_evals,
            "bad1": bad1_f, "bad2": bad2_f, "steps": fsteps},
        "hier_over_flat_speedup": None if flat_fps is None else fps / world / flat_fps,
        "bad1": bad1_h, "bad2": bad2_h,
        # the hierarchical method at a bad-pixel rate equal to or better than flat matching's
        "hier_vs_flat_equal_or_better_bad_rate": hvf,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle CPU time")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds of oracle work for --impl reference (warm-up + timed steps)")
    ap.add_argument("--no-additions", action="store_true", help="skip the batching and differentiable lines")
    ap.add_argument("--no-flat", action="store_true", help="skip flat matching and the gated methods (profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
