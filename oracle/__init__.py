"""FP64 CPU oracle for hierarchical ZNCC block matching -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use
this package.  It wraps ``msbm_oracle.c`` (plain C, FP64, OpenMP over rows) through
ctypes and shares no code with the CUDA library.  ``build()`` compiles it with gcc into
``oracle/_build/``; the first call of any function builds it if needed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no -ffast-math: IEEE FP64 throughout)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            lib.oracle_reduce.argtypes = [P, i, i, P]
            lib.oracle_pyramid.argtypes = [P, i, i, i, P]
            lib.oracle_zncc.argtypes = [P, P, i, i, i, i, i, i]
            lib.oracle_zncc.restype = d
            lib.oracle_match_level.argtypes = [P, P, i, i, i, i, i, P, i, i, P, P, P]
            lib.oracle_match_level.restype = ll
            lib.oracle_disparity.argtypes = [P, P, i, i, i, i, i, i, P, P, P]
            lib.oracle_disparity.restype = ll
            lib.oracle_softargmax_fwd.argtypes = [P, P, i, i, i, i, i, d, d, P, P]
            lib.oracle_softargmax_bwd.argtypes = [P, P, i, i, i, i, i, d, d, P, P, P]
            lib.oracle_bicubic_at.argtypes = [P, i, i, d, d]
            lib.oracle_bicubic_at.restype = d
            lib.oracle_upsample_cost.argtypes = [P, i, i, i, i, P]
            lib.oracle_match_level_beta.argtypes = [P, P, i, i, i, i, i, P, P, i, i, d, P, P, P, P, P]
            lib.oracle_match_level_beta.restype = ll
            lib.oracle_alpha_refine.argtypes = [P, P, i, i, i, i, d, P, P, P, P]
            lib.oracle_selective_median.argtypes = [P, P, i, i, d, P]
            lib.oracle_disparity_full.argtypes = [P, P, i, i, i, i, i, i, d, d, i, P, P, P]
            lib.oracle_disparity_full.restype = ll
            lib.oracle_level_half_width.argtypes = [i, i]
            lib.oracle_level_half_width.restype = i
            lib.oracle_max_threads.restype = i
            lib.oracle_set_threads.argtypes = [i]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u8(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint8:
        raise TypeError("expected uint8 image")
    return a


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def level_size(w: int, h: int, k: int) -> tuple[int, int]:
    for _ in range(k):
        w, h = (w + 1) // 2, (h + 1) // 2
    return w, h


def level_disp(d: int, k: int) -> int:
    return -(-d // (1 << k))


def reduce(img) -> np.ndarray:
    """One pyramid step (5-tap binomial, clamp-to-edge, 2x decimation)."""
    img = _u8(img)
    h, w = img.shape
    out = np.empty(((h + 1) // 2, (w + 1) // 2), np.uint8)
    _load().oracle_reduce(_ptr(img), w, h, _ptr(out))
    return out


def pyramid(img, levels: int) -> list[np.ndarray]:
    img = _u8(img)
    h, w = img.shape
    sizes = [level_size(w, h, k) for k in range(levels)]
    buf = np.empty(sum(a * b for a, b in sizes), np.uint8)
    _load().oracle_pyramid(_ptr(img), w, h, levels, _ptr(buf))
    out, o = [], 0
    for a, b in sizes:
        out.append(buf[o:o + a * b].reshape(b, a).copy())
        o += a * b
    return out


def zncc(a_img, b_img, n: int, y: int, x: int, z: int) -> float:
    """ZNCC (Eq. 2) of the left window at (y, x) and the right window at (y, x - z)."""
    a_img, b_img = _u8(a_img), _u8(b_img)
    h, w = a_img.shape
    return float(_load().oracle_zncc(_ptr(a_img), _ptr(b_img), w, h, n, y, x, z))


def match_level(a_img, b_img, n: int, dk: int, r: int = 0, prior=None):
    """One level of WTA: full range if ``prior`` is None, else the restricted search
    around 2 * prior(y/2, x/2).  Returns (d int16, C f64, C2 f64, evaluations)."""
    a_img, b_img = _u8(a_img), _u8(b_img)
    h, w = a_img.shape
    d = np.empty((h, w), np.int16)
    c = np.empty((h, w), np.float64)
    c2 = np.empty((h, w), np.float64)
    if prior is None:
        pp, hp, wp = None, 0, 0
    else:
        prior = np.ascontiguousarray(prior, dtype=np.int16)
        hp, wp = prior.shape
        pp = _ptr(prior)
    ev = _load().oracle_match_level(_ptr(a_img), _ptr(b_img), w, h, n, dk, r, pp, wp, hp,
                                    _ptr(d), _ptr(c), _ptr(c2))
    return d, c, c2, int(ev)


def disparity(left, right, max_disp: int, levels: int, window: int, radius: int):
    """Hierarchical pass.  Returns a dict with per-level lists ``d``, ``C``, ``C2`` (level
    0 first) and the evaluation count ``evals``."""
    left, right = _u8(left), _u8(right)
    h, w = left.shape
    sizes = [level_size(w, h, k) for k in range(levels)]
    tot = sum(a * b for a, b in sizes)
    d = np.empty(tot, np.int16)
    c = np.empty(tot, np.float64)
    c2 = np.empty(tot, np.float64)
    ev = _load().oracle_disparity(_ptr(left), _ptr(right), w, h, max_disp, levels, window,
                                  radius, _ptr(d), _ptr(c), _ptr(c2))
    if ev < 0:
        raise ValueError("invalid arguments")
    out = {"d": [], "C": [], "C2": [], "evals": int(ev)}
    o = 0
    for a, b in sizes:
        out["d"].append(d[o:o + a * b].reshape(b, a))
        out["C"].append(c[o:o + a * b].reshape(b, a))
        out["C2"].append(c2[o:o + a * b].reshape(b, a))
        o += a * b
    return out


def softargmax_fwd(left, right, n: int, ndisp: int, T: float, eps: float, want_rho=False):
    """Soft-argmax ZNCC level, FP64.  left/right: (B, H, W) float.  Returns d_soft
    (B, H, W) and, if asked, rho (B, H, W, ndisp) with -inf at inadmissible z."""
    left = np.ascontiguousarray(left, dtype=np.float64)
    right = np.ascontiguousarray(right, dtype=np.float64)
    if left.ndim == 2:
        left, right = left[None], right[None]
    b, h, w = left.shape
    ds = np.empty((b, h, w), np.float64)
    rho = np.empty((b, h, w, ndisp), np.float64) if want_rho else None
    _load().oracle_softargmax_fwd(_ptr(left), _ptr(right), b, h, w, n, ndisp, T, eps,
                                  _ptr(ds), _ptr(rho) if want_rho else None)
    return (ds, rho) if want_rho else ds


def softargmax_bwd(left, right, n: int, ndisp: int, T: float, eps: float, g_d):
    left = np.ascontiguousarray(left, dtype=np.float64)
    right = np.ascontiguousarray(right, dtype=np.float64)
    g_d = np.ascontiguousarray(g_d, dtype=np.float64)
    if left.ndim == 2:
        left, right, g_d = left[None], right[None], g_d[None]
    b, h, w = left.shape
    gl = np.empty_like(left)
    gr = np.empty_like(left)
    _load().oracle_softargmax_bwd(_ptr(left), _ptr(right), b, h, w, n, ndisp, T, eps,
                                  _ptr(g_d), _ptr(gl), _ptr(gr))
    return gl, gr


# --- gated steps of the full method (alpha refinement, beta fallback, selective median) ---
ALPHA_REFINE, BETA_FALLBACK, SELECTIVE_MEDIAN = 1, 2, 4
FULL_METHOD = ALPHA_REFINE | BETA_FALLBACK | SELECTIVE_MEDIAN
WINDOW_HALVING = 8     # per-level block size halving (Sec. III)


def level_half_width(n0: int, k: int) -> int:
    """Window half-width at level k with per-level halving: max(1, n0 >> k)."""
    return int(_load().oracle_level_half_width(n0, k))


def bicubic_at(cost, cy: float, cx: float) -> float:
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    h, w = cost.shape
    return float(_load().oracle_bicubic_at(_ptr(cost), w, h, cy, cx))


def upsample_cost(cost, width: int, height: int) -> np.ndarray:
    """Bicubic cost prior of Sec. III-C at the finer level's size."""
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    h, w = cost.shape
    out = np.empty((height, width), np.float64)
    _load().oracle_upsample_cost(_ptr(cost), w, h, width, height, _ptr(out))
    return out


def match_level_beta(a_img, b_img, n: int, dk: int, r: int, prior, cprior, beta: float):
    """Eq. 8-9 (both branches).  Returns (d, C, C2, evals, fallback mask, C_hat)."""
    a_img, b_img = _u8(a_img), _u8(b_img)
    h, w = a_img.shape
    prior = np.ascontiguousarray(prior, dtype=np.int16)
    cprior = np.ascontiguousarray(cprior, dtype=np.float64)
    hp, wp = prior.shape
    d = np.empty((h, w), np.int16)
    c = np.empty((h, w), np.float64)
    c2 = np.empty((h, w), np.float64)
    fb = np.empty((h, w), np.uint8)
    ch = np.empty((h, w), np.float64)
    ev = _load().oracle_match_level_beta(_ptr(a_img), _ptr(b_img), w, h, n, dk, r, _ptr(prior),
                                         _ptr(cprior), wp, hp, beta, _ptr(d), _ptr(c), _ptr(c2),
                                         _ptr(fb), _ptr(ch))
    return d, c, c2, int(ev), fb.astype(bool), ch


def alpha_refine(a_img, b_img, n: int, dk: int, alpha: float, d, cost, cost2=None):
    """Eq. 5-7 on a coarsest-level result.  Returns (d, C, C2, refined mask) (new arrays)."""
    a_img, b_img = _u8(a_img), _u8(b_img)
    h, w = a_img.shape
    d = np.array(d, dtype=np.int16, copy=True, order="C")
    c = np.array(cost, dtype=np.float64, copy=True, order="C")
    c2 = np.full((h, w), -np.inf) if cost2 is None else np.array(cost2, dtype=np.float64, copy=True, order="C")
    ref = np.empty((h, w), np.uint8)
    _load().oracle_alpha_refine(_ptr(a_img), _ptr(b_img), w, h, n, dk, alpha, _ptr(d), _ptr(c), _ptr(c2),
                                _ptr(ref))
    return d, c, c2, ref.astype(bool)


def selective_median(d, cost, alpha: float) -> np.ndarray:
    """Eq. 10."""
    d = np.ascontiguousarray(d, dtype=np.int16)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    h, w = d.shape
    out = np.empty_like(d)
    _load().oracle_selective_median(_ptr(d), _ptr(cost), w, h, alpha, _ptr(out))
    return out


def disparity_full(left, right, max_disp: int, levels: int, window: int, radius: int,
                   alpha: float = 0.9, beta: float = 0.9, flags: int = FULL_METHOD):
    """The full method (plain method plus the gated steps selected by ``flags``)."""
    left, right = _u8(left), _u8(right)
    h, w = left.shape
    sizes = [level_size(w, h, k) for k in range(levels)]
    tot = sum(a * b for a, b in sizes)
    d = np.empty(tot, np.int16)
    c = np.empty(tot, np.float64)
    c2 = np.empty(tot, np.float64)
    ev = _load().oracle_disparity_full(_ptr(left), _ptr(right), w, h, max_disp, levels, window, radius,
                                       alpha, beta, flags, _ptr(d), _ptr(c), _ptr(c2))
    if ev < 0:
        raise ValueError("invalid arguments")
    out = {"d": [], "C": [], "C2": [], "evals": int(ev)}
    o = 0
    for a, b in sizes:
        out["d"].append(d[o:o + a * b].reshape(b, a))
        out["C"].append(c[o:o + a * b].reshape(b, a))
        out["C2"].append(c2[o:o + a * b].reshape(b, a))
        o += a * b
    return out
