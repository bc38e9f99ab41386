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
