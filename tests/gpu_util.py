"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

COST_TOL = 1e-4      # |C_gpu - C_oracle| bound (FP32 final divide vs FP64)
TIE_TOL = 1e-4       # oracle best - second below this: a near-tie, disparity may differ


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def compare_level(d_gpu, c_gpu, d_or, c_or, c2_or, what=""):
    """Costs within COST_TOL everywhere; disparities equal except at counted near-ties.
    Returns the number of near-tie pixels where the disparities differ."""
    d_gpu = np.asarray(d_gpu)
    c_gpu = np.asarray(c_gpu, dtype=np.float64)
    err = np.abs(c_gpu - c_or)
    assert np.all(np.isfinite(c_gpu)), what
    assert err.max() <= COST_TOL, f"{what}: max cost error {err.max():.3g}"
    near = (c_or - c2_or) < TIE_TOL
    bad = (d_gpu != d_or) & ~near
    assert not bad.any(), f"{what}: {int(bad.sum())} disparities differ outside near-ties " \
                          f"(first at {np.argwhere(bad)[:3].tolist()})"
    return int(((d_gpu != d_or) & near).sum())
