"""Allocation-free flat matching (msbm_flat_disparity_noalloc) against the FP64 oracle and
the allocating context path.

The entry point serves callers that cannot call cudaMalloc (a real-time loop that cannot
take the device-wide synchronisation an allocation may cause, or a framework that owns all
device memory through its own pool).  Its scratch is a fixed device array inside the
library, shared by every call, so this test makes several calls in a row with different
image sizes and checks each one against the oracle (costs within 1e-4, disparities equal
outside counted near-ties) and against the context path (msbm_disparity with K = 1) under
the same bar.  One call is 1400 x 1000, where the context path also runs the full-range
tile kernel.  This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1901_09593_gb300 import scenes
from tests.gpu_util import COST_TOL, TIE_TOL, compare_level

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _noalloc(lib, L, R, W, H, D, win, d, c, status, stream):
    return lib.msbm_flat_disparity_noalloc(_p(L), _p(R), L.stride(0), W, H, D, win, _p(d), _p(c),
                                           _p(status), ctypes.c_void_p(stream))


def test_noalloc_flat_matches_oracle_and_context_path_on_calls_in_a_row():
    import torch

    from paper_1901_09593_gb300 import Context, _lib, build
    build.build()
    oracle.build()
    lib = _lib.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream

    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 0)
    big = scenes.make_pair(scenes.SPECS["bench_1400x1000"], 0)
    rng = np.random.default_rng(11)
    rand_l = rng.integers(0, 256, (97, 150)).astype(np.uint8)
    rand_r = rng.integers(0, 256, (97, 150)).astype(np.uint8)
    cases = [(sc.left, sc.right, 32, 5), (rand_l, rand_r, 48, 7), (big.left, big.right, 64, 7),
             (sc.left, sc.right, 32, 5)]

    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for left, right, D, win in cases:
        H, W = left.shape
        L = torch.from_numpy(left).cuda()
        R = torch.from_numpy(right).cuda()
        d = torch.empty((H, W), dtype=torch.int16, device="cuda")
        c = torch.empty((H, W), dtype=torch.float32, device="cuda")
        assert _noalloc(lib, L, R, W, H, D, win, d, c, status, stream) == _lib.MSBM_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        d_np, c_np = d.cpu().numpy(), c.cpu().numpy()
        what = f"no-alloc {W}x{H} D={D} {win}x{win}"
        do, co, c2, _ = oracle.match_level(left, right, win // 2, D)
        compare_level(d_np, c_np, do, co, c2, what)

        ctx = Context(W, H, D, 1, win, 0)
        d_ref, c_ref = ctx.disparity(L, R)
        ctx.sync()
        d_ref_np, c_ref_np = d_ref.cpu().numpy(), c_ref.cpu().numpy()
        assert np.abs(c_np - c_ref_np).max() <= COST_TOL, what
        near = (co - c2) < TIE_TOL
        assert not ((d_np != d_ref_np) & ~near).any(), what
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1901_09593_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    st = lib.msbm_flat_disparity_noalloc(dummy, dummy, 4096, 4096, 2160, 64, 7, dummy, None, None, None)
    assert st == _lib.MSBM_ERR_UNSUPPORTED
