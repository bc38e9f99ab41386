"""The issue-rate probes behind the matching stages' roofline denominators (msbm_pipe_probe,
through the C ABI): the operation count follows the documented formula, the runs take time,
and no rate exceeds the SM's issue bound (one warp instruction per clock per sub-partition,
128 lanes per clock per SM, at the GPU's maximum clock)."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_every_probe_runs_and_stays_under_the_issue_bound():
    import torch

    from paper_1901_09593_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_mhz = 2070.0      # the GB300's maximum SM clock; the probe changes no clock
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for kind in range(5):
        ms, ops = ctypes.c_float(), ctypes.c_double()
        assert lib.msbm_pipe_probe(kind, sms * 8, 2000, st, ctypes.byref(ms), ctypes.byref(ops)) == _lib.MSBM_OK
        assert ops.value == sms * 8 * 256 * 2000 * 128
        assert ms.value > 0
        rate = ops.value / (ms.value * 1e-3)
        assert rate <= 1.05 * sms * 128 * max_mhz * 1e6, (kind, rate)
        assert rate >= 0.01 * sms * 128 * max_mhz * 1e6, (kind, rate)


def test_probe_rejects_bad_arguments():
    from paper_1901_09593_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    ms, ops = ctypes.c_float(), ctypes.c_double()
    assert lib.msbm_pipe_probe(5, 1, 1, None, ctypes.byref(ms), ctypes.byref(ops)) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_pipe_probe(0, 0, 1, None, ctypes.byref(ms), ctypes.byref(ops)) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_pipe_probe(0, 1, 0, None, ctypes.byref(ms), ctypes.byref(ops)) == _lib.MSBM_ERR_INVALID_ARG
    assert lib.msbm_pipe_probe(0, 1, 1, None, None, ctypes.byref(ops)) == _lib.MSBM_ERR_INVALID_ARG
