"""ctypes binding of libmsbm.so (the C ABI in include/msbm.h), same names as the C calls.

Loading fails loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libmsbm.so")

MSBM_OK = 0
MSBM_ERR_INVALID_ARG = 1
MSBM_ERR_ALIGNMENT = 2
MSBM_ERR_OOM = 3
MSBM_ERR_CUDA = 4
MSBM_ERR_TIMEOUT = 5
MSBM_ERR_UNSUPPORTED = 6

MSBM_FLAG_NO_GRAPH = 1
MSBM_FLAG_TEST_TIMEOUT = 2
MSBM_FLAG_ALPHA_REFINE = 4
MSBM_FLAG_BETA_FALLBACK = 8
MSBM_FLAG_SELECTIVE_MEDIAN = 16
MSBM_FLAGS_FULL_METHOD = 28
MSBM_FLAG_WINDOW_HALVING = 32
MSBM_FLAG_BATCH_GROUPED = 64

# Every function the header declares, with its ctypes signature.
c_void_p, c_int32, c_uint32, c_size_t = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_size_t
P = ctypes.POINTER


class msbm_params(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("max_disp", c_int32),
                ("levels", c_int32), ("window", c_int32), ("radius", c_int32),
                ("flags", c_uint32), ("alpha", ctypes.c_float), ("beta", ctypes.c_float)]


SIGNATURES = {
    "msbm_version": ([], ctypes.c_int),
    "msbm_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "msbm_create": ([P(msbm_params), c_void_p, P(c_void_p)], ctypes.c_int),
    "msbm_destroy": ([c_void_p], ctypes.c_int),
    "msbm_set_stream": ([c_void_p, c_void_p], ctypes.c_int),
    "msbm_level_shape": ([c_void_p, c_int32, P(c_int32), P(c_int32), P(c_int32)], ctypes.c_int),
    "msbm_pyramid": ([c_void_p, c_void_p, c_void_p, c_size_t], ctypes.c_int),
    "msbm_level_image": ([c_void_p, c_int32, c_int32, c_void_p], ctypes.c_int),
    "msbm_match_level": ([c_void_p, c_int32, c_void_p, c_void_p, c_void_p], ctypes.c_int),
    "msbm_disparity": ([c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], ctypes.c_int),
    "msbm_disparity_host": ([c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], ctypes.c_int),
    "msbm_disparity_host_frames": ([c_void_p, c_int32, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p], ctypes.c_int),
    "msbm_pipe_probe": ([c_int32, c_int32, c_int32, c_void_p, P(ctypes.c_float), P(ctypes.c_double)], ctypes.c_int),
    "msbm_level_result": ([c_void_p, c_int32, c_void_p, c_void_p], ctypes.c_int),
    "msbm_profile_disparity": ([c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p,
                                P(ctypes.c_float), c_int32], ctypes.c_int),
    "msbm_sync": ([c_void_p], ctypes.c_int),
    "msbm_alpha_refine": ([c_void_p, c_int32, c_void_p, c_void_p], ctypes.c_int),
    "msbm_selective_median": ([c_void_p, c_int32, c_void_p, c_void_p, c_void_p], ctypes.c_int),
    "msbm_match_level_beta": ([c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], ctypes.c_int),
    "msbm_eval_count": ([c_void_p, P(ctypes.c_int64), c_int32], ctypes.c_int),
    "msbm_pass_kernel_count": ([c_void_p, P(c_int32)], ctypes.c_int),
    "msbm_set_level_tuning": ([c_void_p, c_int32, c_int32, c_int32], ctypes.c_int),
    "msbm_batch_create": ([P(msbm_params), c_int32, c_void_p, c_void_p, c_void_p, P(c_void_p)], ctypes.c_int),
    "msbm_batch_run": ([c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p], ctypes.c_int),
    "msbm_batch_sync": ([c_void_p], ctypes.c_int),
    "msbm_batch_eval_count": ([c_void_p, P(ctypes.c_int64), c_int32], ctypes.c_int),
    "msbm_batch_level_result": ([c_void_p, c_int32, c_int32, c_void_p, c_void_p], ctypes.c_int),
    "msbm_batch_info": ([c_void_p, P(ctypes.c_int64), P(c_int32), P(c_int32)], ctypes.c_int),
    "msbm_batch_destroy": ([c_void_p], ctypes.c_int),
    "msbm_zncc_softargmax_fwd": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                                  ctypes.c_float, ctypes.c_float, c_void_p, c_void_p, c_void_p, c_void_p],
                                 ctypes.c_int),
    "msbm_zncc_softargmax_workspace_bytes": ([c_int32, c_int32, c_int32, c_int32, c_int32], c_size_t),
    "msbm_zncc_softargmax_bwd": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                                  ctypes.c_float, ctypes.c_float, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_size_t, c_void_p], ctypes.c_int),
    "msbm_zncc_softargmax_saved_bytes": ([c_int32, c_int32, c_int32, c_int32, c_int32], c_size_t),
    "msbm_zncc_softargmax_fwd_saved": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                                        ctypes.c_float, ctypes.c_float, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_size_t, c_void_p], ctypes.c_int),
    "msbm_zncc_softargmax_bwd_saved": ([c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32,
                                        ctypes.c_float, ctypes.c_float, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p],
                                       ctypes.c_int),
    "msbm_flat_disparity_noalloc": ([c_void_p, c_void_p, c_size_t, c_int32, c_int32, c_int32, c_int32,
                                     c_void_p, c_void_p, c_void_p, c_void_p], ctypes.c_int),
}

_lib = None
_lock = threading.Lock()


class MsbmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib.msbm_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else msg)


def load(path: str | None = None):
    """Load libmsbm.so (built by ``paper_1901_09593_gb300.build``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            so = path or SO_PATH
            if not os.path.exists(so):
                raise RuntimeError(f"libmsbm.so is not built ({so}); run "
                                   "`python -m paper_1901_09593_gb300.build` (needs nvcc)")
            lib = ctypes.CDLL(so)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def check(status: int, what: str = "") -> None:
    if status != MSBM_OK:
        raise MsbmError(status, what)
