"""CPU checks of the C ABI: the library builds, loads, and exports every function that
include/msbm.h declares; argument validation answers before any device work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(msbm_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1901_09593_gb300 import _lib, build
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["msbm_create", "msbm_pyramid", "msbm_match_level", "msbm_disparity",
                     "msbm_destroy", "msbm_disparity_host", "msbm_sync"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1901_09593_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_status_strings_and_version(lib):
    assert lib.msbm_version() >= 10000
    assert lib.msbm_status_string(0) == b"ok"
    assert lib.msbm_status_string(5) == b"device wait timed out"
    assert lib.msbm_status_string(99) == b"unknown status"


@pytest.mark.parametrize("field,value", [
    ("width", 0), ("height", -1), ("width", 16385), ("max_disp", 0), ("max_disp", 5000),
    ("levels", 0), ("levels", 13), ("window", 4), ("window", 1), ("window", 15),
    ("radius", -1), ("radius", 17), ("flags", 1 << 7)])
def test_create_rejects_bad_params_before_device_work(lib, field, value):
    from paper_1901_09593_gb300 import _lib
    p = _lib.msbm_params(64, 48, 16, 2, 5, 2, 0)
    setattr(p, field, value)
    out = ctypes.c_void_p(123)
    st = lib.msbm_create(ctypes.byref(p), None, ctypes.byref(out))
    assert st == _lib.MSBM_ERR_INVALID_ARG
    assert out.value is None


def test_null_arguments_are_rejected(lib):
    from paper_1901_09593_gb300 import _lib
    p = _lib.msbm_params(64, 48, 16, 2, 5, 2, 0)
    assert lib.msbm_create(ctypes.byref(p), None, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_create(None, None, ctypes.byref(ctypes.c_void_p())) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_pyramid(None, None, None, 0) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_match_level(None, 0, None, None, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_disparity(None, None, None, 0, None, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_sync(None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_destroy(None) == _lib.MSBM_OK


def test_create_without_gpu_reports_unsupported(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1901_09593_gb300 import _lib
    p = _lib.msbm_params(64, 48, 16, 2, 5, 2, 0)
    out = ctypes.c_void_p()
    assert lib.msbm_create(ctypes.byref(p), None, ctypes.byref(out)) == _lib.MSBM_ERR_UNSUPPORTED


def test_context_fails_loudly_when_library_missing(tmp_path):
    from paper_1901_09593_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def _no_gpu():
    torch = pytest.importorskip("torch")
    return not torch.cuda.is_available()


# non-null placeholders: these calls reject their arguments before touching any pointer
_FAKE = ctypes.c_void_p(4096)


@pytest.mark.parametrize("field,value", [
    ("width", 0), ("height", 16385), ("max_disp", 0), ("max_disp", 4097), ("levels", 0),
    ("levels", 13), ("window", 11), ("window", 6), ("radius", 17), ("flags", 4)])
def test_batch_create_rejects_bad_pair_params(lib, field, value):
    from paper_1901_09593_gb300 import _lib
    pairs = (_lib.msbm_params * 3)(*[_lib.msbm_params(64 + 32 * i, 48, 16, 2, 5, 2, 0) for i in range(3)])
    setattr(pairs[1], field, value)
    out = ctypes.c_void_p(123)
    assert lib.msbm_batch_create(pairs, 3, None, None, None, ctypes.byref(out)) == _lib.MSBM_ERR_INVALID_ARG
    assert out.value is None


def test_batch_create_rejects_bad_counts_and_tuning(lib):
    from paper_1901_09593_gb300 import _lib
    pairs = (_lib.msbm_params * 2)(*[_lib.msbm_params(64, 48, 16, 2, 5, 2, 0) for _ in range(2)])
    out = ctypes.c_void_p()
    bad = _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_batch_create(pairs, 0, None, None, None, ctypes.byref(out)) == bad
    assert lib.msbm_batch_create(pairs, 4097, None, None, None, ctypes.byref(out)) == bad
    assert lib.msbm_batch_create(None, 2, None, None, None, ctypes.byref(out)) == bad
    assert lib.msbm_batch_create(pairs, 2, None, None, None, None) == bad
    sx = (ctypes.c_int32 * 2)(1, 3)
    assert lib.msbm_batch_create(pairs, 2, sx, None, None, ctypes.byref(out)) == bad
    zb = (ctypes.c_int32 * 2)(0, 48)
    assert lib.msbm_batch_create(pairs, 2, None, zb, None, ctypes.byref(out)) == bad
    if _no_gpu():
        ok_sx, ok_zb = (ctypes.c_int32 * 2)(1, 2), (ctypes.c_int32 * 2)(0, 64)
        assert lib.msbm_batch_create(pairs, 2, ok_sx, ok_zb, None, ctypes.byref(out)) == _lib.MSBM_ERR_UNSUPPORTED
    assert lib.msbm_batch_destroy(None) == _lib.MSBM_OK


def test_softargmax_workspace_bytes_formula_and_invalid_sizes(lib):
    # the backward's workspace: one float per (image, pixel, candidate), six floats per
    # pixel and four per position of the window-extended image, each part rounded up to 256
    # bytes
    al = lambda v: (v + 255) // 256 * 256
    for b, h, w, win, nd in [(1, 5, 9, 3, 4), (8, 480, 640, 5, 64), (2, 7, 13, 9, 256)]:
        n = win // 2
        want = al(b * nd * h * w * 4) + 6 * al(b * h * w * 4) + al(b * (h + 2 * n) * (w + 2 * n) * 16)
        assert lib.msbm_zncc_softargmax_workspace_bytes(b, h, w, win, nd) == want
    for args in [(0, 5, 9, 3, 4), (65536, 5, 9, 3, 4), (1, 0, 9, 3, 4), (1, 5, 16385, 3, 4),
                 (1, 5, 9, 1, 4), (1, 5, 9, 4, 4), (1, 5, 9, 11, 4), (1, 5, 9, 3, 0), (1, 5, 9, 3, 257)]:
        assert lib.msbm_zncc_softargmax_workspace_bytes(*args) == 0, args


@pytest.mark.parametrize("change", ["null_left", "batch", "height", "window_even", "window_big", "ndisp",
                                    "temperature", "temperature_nan", "eps", "null_out"])
def test_softargmax_rejects_bad_arguments_before_device_work(lib, change):
    from paper_1901_09593_gb300 import _lib
    a = dict(L=_FAKE, R=_FAKE, B=2, H=16, W=24, win=5, nd=8, T=0.1, eps=1e-6, out=_FAKE)
    a.update({"null_left": {"L": None}, "batch": {"B": 0}, "height": {"H": 16385}, "window_even": {"win": 4},
              "window_big": {"win": 11}, "ndisp": {"nd": 257}, "temperature": {"T": 0.0},
              "temperature_nan": {"T": float("nan")}, "eps": {"eps": -1.0}, "null_out": {"out": None}}[change])
    st = lib.msbm_zncc_softargmax_fwd(a["L"], a["R"], a["B"], a["H"], a["W"], a["win"], a["nd"], a["T"], a["eps"],
                                      a["out"], _FAKE, _FAKE, None)
    assert st == _lib.MSBM_ERR_INVALID_ARG
    st = lib.msbm_zncc_softargmax_bwd(a["L"], a["R"], a["B"], a["H"], a["W"], a["win"], a["nd"], a["T"], a["eps"],
                                      _FAKE, _FAKE, _FAKE, _FAKE, a["out"], _FAKE, _FAKE, 1 << 30, None)
    assert st == _lib.MSBM_ERR_INVALID_ARG


def test_softargmax_backward_checks_its_workspace(lib):
    from paper_1901_09593_gb300 import _lib
    need = lib.msbm_zncc_softargmax_workspace_bytes(1, 8, 16, 3, 4)
    args = [_FAKE, _FAKE, 1, 8, 16, 3, 4, 0.1, 0.0, _FAKE, _FAKE, _FAKE, _FAKE, _FAKE, _FAKE]
    assert lib.msbm_zncc_softargmax_bwd(*args, None, need, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_bwd(*args, _FAKE, need - 1, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_bwd(*args, ctypes.c_void_p(4096 + 128), need, None) == _lib.MSBM_ERR_ALIGNMENT


def test_softargmax_saved_bytes_formula_and_checks(lib):
    # the kept forward: one float per (image, z, pixel), then two float2 per pixel, each part
    # rounded up to 256 bytes
    from paper_1901_09593_gb300 import _lib
    al = lambda v: (v + 255) // 256 * 256
    for b, h, w, win, nd in [(1, 5, 9, 3, 4), (8, 480, 640, 7, 64)]:
        assert lib.msbm_zncc_softargmax_saved_bytes(b, h, w, win, nd) == al(b * nd * h * w * 4) + 2 * al(b * h * w * 8)
    assert lib.msbm_zncc_softargmax_saved_bytes(1, 5, 9, 4, 4) == 0
    need = lib.msbm_zncc_softargmax_saved_bytes(1, 8, 16, 3, 4)
    fwd = [_FAKE, _FAKE, 1, 8, 16, 3, 4, 0.1, 0.0, _FAKE, _FAKE, _FAKE]
    assert lib.msbm_zncc_softargmax_fwd_saved(*fwd, None, need, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_fwd_saved(*fwd, _FAKE, need - 1, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_fwd_saved(*fwd, ctypes.c_void_p(4096 + 64), need, None) == _lib.MSBM_ERR_ALIGNMENT
    ws = lib.msbm_zncc_softargmax_workspace_bytes(1, 8, 16, 3, 4)
    bwd = [_FAKE, _FAKE, 1, 8, 16, 3, 4, 0.1, 0.0, _FAKE, _FAKE, _FAKE, _FAKE]
    assert lib.msbm_zncc_softargmax_bwd_saved(*bwd, None, need, _FAKE, _FAKE, _FAKE, ws, None) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_bwd_saved(*bwd, _FAKE, need - 1, _FAKE, _FAKE, _FAKE, ws, None) == \
        _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_zncc_softargmax_bwd_saved(*bwd, ctypes.c_void_p(4096 + 32), need, _FAKE, _FAKE, _FAKE, ws,
                                              None) == _lib.MSBM_ERR_ALIGNMENT


def test_noalloc_rejects_bad_arguments_and_oversized_images_before_device_work(lib):
    from paper_1901_09593_gb300 import _lib
    f = lib.msbm_flat_disparity_noalloc
    bad = _lib.MSBM_ERR_INVALID_ARG
    assert f(None, _FAKE, 64, 64, 48, 16, 5, _FAKE, None, None, None) == bad
    assert f(_FAKE, _FAKE, 64, 64, 48, 16, 5, None, None, None, None) == bad
    assert f(_FAKE, _FAKE, 63, 64, 48, 16, 5, _FAKE, None, None, None) == bad       # pitch < width
    assert f(_FAKE, _FAKE, 64, 64, 48, 0, 5, _FAKE, None, None, None) == bad
    assert f(_FAKE, _FAKE, 64, 64, 48, 4097, 5, _FAKE, None, None, None) == bad
    assert f(_FAKE, _FAKE, 64, 64, 48, 16, 15, _FAKE, None, None, None) == bad
    assert f(_FAKE, _FAKE, 64, 64, 48, 16, 4, _FAKE, None, None, None) == bad
    assert f(_FAKE, _FAKE, 16385, 16385, 48, 16, 5, _FAKE, None, None, None) == bad
    # two apron buffers of round_up(W + 32, 128) x (H + 16) bytes must fit the 16 MiB array
    assert f(_FAKE, _FAKE, 4096, 4096, 2160, 64, 5, _FAKE, None, None, None) == _lib.MSBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("flags,alpha,beta,ok", [
    (4, float("nan"), 0.9, False), (16, 2.0, 0.9, False), (8, 0.9, -2.5, False), (8, 0.9, float("nan"), False),
    (0, float("nan"), float("nan"), True), (28, 0.9, 0.9, True), (4, -1.99, 5.0, True)])
def test_create_checks_the_thresholds_its_flags_use(lib, flags, alpha, beta, ok):
    from paper_1901_09593_gb300 import _lib
    p = _lib.msbm_params(64, 48, 16, 2, 5, 2, flags, alpha, beta)
    out = ctypes.c_void_p()
    st = lib.msbm_create(ctypes.byref(p), None, ctypes.byref(out))
    if not ok:
        assert st == _lib.MSBM_ERR_INVALID_ARG
    else:
        assert st != _lib.MSBM_ERR_INVALID_ARG
        if st == _lib.MSBM_OK:
            lib.msbm_destroy(out)


C_CONSUMER = r"""
#include <stdio.h>
#include "msbm.h"
int main(void) {
    msbm_params p = {64, 48, 16, 2, 5, 2, 0u, 0.9f, 0.9f};
    msbm_ctx *ctx = NULL;
    p.window = 4;   /* even: rejected before any device work */
    msbm_status s = msbm_create(&p, NULL, &ctx);
    printf("%d %s %d %d\n", msbm_version() >= 10000, msbm_status_string(s), ctx == NULL,
           (int)msbm_zncc_softargmax_workspace_bytes(1, 8, 16, 3, 4));
    return s == MSBM_ERR_INVALID_ARG ? 0 : 1;
}
"""


def test_header_serves_a_plain_c_program(lib, tmp_path):
    # the boundary is a C ABI: a C11 program includes the header with every warning an error,
    # links the library and calls it
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    from paper_1901_09593_gb300 import build
    src, exe = tmp_path / "consumer.c", tmp_path / "consumer"
    src.write_text(C_CONSUMER)
    subprocess.check_call([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                           os.path.join(ROOT, "include"), str(src), "-o", str(exe), build.SO,
                           "-Wl,-rpath," + os.path.dirname(build.SO)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    al = lambda v: (v + 255) // 256 * 256
    want = al(8 * 16 * 4 * 4) + 6 * al(8 * 16 * 4) + al((8 + 2) * (16 + 2) * 16)
    assert r.stdout.split() == ["1", "invalid", "argument", "1", str(want)], r.stdout
