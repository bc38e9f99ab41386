"""Batched persistent launch against the FP64 oracle, through the C ABI.

Every level of every batched pair is compared element by element with the oracle fed the
batch's own coarser map as the prior, so both sides search the same candidate sets: costs
within 1e-4 and disparities equal except where the oracle's best and second-best costs
differ by less than 1e-4 (counted).  The batch is also compared with the single-pair
context path: costs within one rounding of the rsqrt order (the batched tile applies the
two factors in the other order) wherever the disparities agree, and the same disparities
at every pixel whose prior cell agrees, except at counted near-ties.  The dependency-wait
timeout path is exercised by withholding the first stage (test hook).  The autotuner's
choices only change speed."""
import numpy as np
import pytest

import oracle
from paper_1901_09593_gb300 import scenes
from tests.gpu_util import TIE_TOL, compare_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09593_gb300 import build
    build.build()
    oracle.build()


def _levels_of_batch(b, i, spec, d0, c0):
    """[(d, c)] of pair i, level 0 first (host arrays)."""
    K = spec[3]
    out = [(d0.cpu().numpy(), c0.cpu().numpy())]
    for k in range(1, K):
        d, c = b.level_result(i, k)
        out.append((d.cpu().numpy(), c.cpu().numpy()))
    return out


def _levels_of_context(spec, L, R, sx=None, zblock=0):
    from paper_1901_09593_gb300 import Context
    w, h, d, k, win, r = spec
    ctx = Context(w, h, d, k, win, r)
    if sx is not None:
        ctx.set_level_tuning(k - 1, sx, zblock)
    dd, cc = ctx.disparity(L, R)
    ctx.sync()
    out = [(dd.cpu().numpy(), cc.cpu().numpy())]
    for j in range(1, k):
        dj, cj = ctx.level_result(j)
        out.append((dj.cpu().numpy(), cj.cpu().numpy()))
    ctx.close()
    return out


def _check_against_oracle(levels, spec, left, right, what):
    """Each level vs the oracle given the batch's own coarser map.  Returns (near-tie
    disagreements, oracle near-tie masks per level)."""
    w, h, D, K, win, r = spec
    pa, pb = oracle.pyramid(left, K), oracle.pyramid(right, K)
    ties, near = 0, [None] * K
    for k in range(K - 1, -1, -1):
        dk = oracle.level_disp(D, k)
        if k == K - 1:
            do, co, c2, _ = oracle.match_level(pa[k], pb[k], win // 2, dk)
        else:
            do, co, c2, _ = oracle.match_level(pa[k], pb[k], win // 2, dk, r, levels[k + 1][0])
        ties += compare_level(levels[k][0], levels[k][1], do, co, c2, f"{what} level {k}")
        near[k] = (co - c2) < TIE_TOL
    return ties, near


def _check_against_context(bl, cl, near, what):
    """Batch vs context path: same disparity wherever the prior cell agrees, except at the
    oracle's near-ties; costs within 1e-6 wherever the disparities agree."""
    K = len(bl)
    for k in range(K - 1, -1, -1):
        db, cb = bl[k]
        dc, cc = cl[k]
        if k == K - 1:
            same_prior = np.ones(db.shape, bool)
        else:
            h, w = db.shape
            pb, pc = bl[k + 1][0], cl[k + 1][0]
            yy, xx = np.mgrid[0:h, 0:w]
            same_prior = pb[yy // 2, xx // 2] == pc[yy // 2, xx // 2]
        bad = (db != dc) & same_prior & ~near[k]
        assert not bad.any(), f"{what} level {k}: {int(bad.sum())} disparities differ from the context path"
        eq = db == dc
        assert np.abs(cb[eq] - cc[eq]).max(initial=0.0) <= 1e-6, f"{what} level {k}: cost"


def _pairs(specs, seed):
    import torch
    rng = np.random.default_rng(seed)
    Ls, Rs = [], []
    for (w, h, *_r) in specs:
        Ls.append(rng.integers(0, 256, (h, w), dtype=np.uint8))
        Rs.append(rng.integers(0, 256, (h, w), dtype=np.uint8))
    return Ls, Rs, [torch.from_numpy(a).cuda() for a in Ls], [torch.from_numpy(a).cuda() for a in Rs]


def _check_batch(b, specs, Lh, Rh, Ld, Rd, d, c, sx=None, zb=None, context=True):
    ties = 0
    for i, spec in enumerate(specs):
        bl = _levels_of_batch(b, i, spec, d[i], c[i])
        t, near = _check_against_oracle(bl, spec, Lh[i], Rh[i], f"pair {i} {spec}")
        ties += t
        if context:
            cl = _levels_of_context(spec, Ld[i], Rd[i])
            _check_against_context(bl, cl, near, f"pair {i} {spec}")
    return ties


MODES = pytest.mark.parametrize("grouped", [False, True], ids=["persistent", "grouped"])


def _mode(grouped):
    from paper_1901_09593_gb300 import _lib
    return _lib.MSBM_FLAG_BATCH_GROUPED if grouped else 0


@MODES
def test_mixed_batch_matches_oracle_and_single_pair_path(grouped):
    from paper_1901_09593_gb300 import Batch
    specs = [(160, 120, 32, 3, 5, 2), (320, 240, 64, 3, 7, 2), (257, 130, 40, 2, 3, 1), (64, 40, 16, 1, 9, 0),
             (1, 1, 1, 1, 3, 0), (33, 17, 50, 4, 7, 3), (200, 96, 48, 2, 5, 5), (700, 400, 96, 6, 5, 2)]
    Lh, Rh, Ls, Rs = _pairs(specs, 0)
    sx = [1, 2, 1, 1, 1, 2, 2, 1]
    zb = [0, 32, 64, 0, 0, 0, 32, 0]
    b = Batch(specs, sx, zb, flags=_mode(grouped))
    d, c = b.run(Ls, Rs)
    b.sync()
    assert b.info()["items"] > 0
    _check_batch(b, specs, Lh, Rh, Ls, Rs, d, c)
    # a second run with new outputs (pointer table re-upload) gives the same maps
    d2, c2 = b.run(Ls, Rs)
    b.sync()
    for i in range(len(specs)):
        np.testing.assert_array_equal(d2[i].cpu().numpy(), d[i].cpu().numpy())
        np.testing.assert_array_equal(c2[i].cpu().numpy(), c[i].cpu().numpy())


@MODES
def test_batch_with_large_coarsest_range_uses_full_range_tiles(grouped):
    # coarsest levels above 64 candidates select the batch kernel build with the full-range
    # tile (tile width and z-block from the caller)
    from paper_1901_09593_gb300 import Batch
    specs = [(300, 60, 160, 1, 5, 2), (240, 100, 300, 2, 7, 2), (96, 64, 24, 2, 5, 1)]
    Lh, Rh, Ls, Rs = _pairs(specs, 11)
    b = Batch(specs, [2, 1, 1], [64, 0, 32], flags=_mode(grouped))
    d, c = b.run(Ls, Rs)
    b.sync()
    _check_batch(b, specs, Lh, Rh, Ls, Rs, d, c)


def test_scene_batch_matches_oracle_on_levels():
    from paper_1901_09593_gb300 import Batch
    import torch
    spec = scenes.SPECS["small_320x240"]
    scs = [scenes.make_pair(spec, s) for s in range(3)]
    specs = [(spec.width, spec.height, spec.max_disp, spec.levels, spec.window, spec.radius)] * 3
    b = Batch(specs)
    Ls = [torch.from_numpy(s.left).cuda() for s in scs]
    Rs = [torch.from_numpy(s.right).cuda() for s in scs]
    d, c = b.run(Ls, Rs)
    b.sync()
    _check_batch(b, specs, [s.left for s in scs], [s.right for s in scs], Ls, Rs, d, c)


@MODES
def test_mixed_size_batch_of_48_benchmark_pairs(grouped):
    # the 48 seeded mixed-size pairs the batch benchmark runs: every level of every pair
    # against the oracle, and against the single-pair path
    from paper_1901_09593_gb300 import Batch, autotune
    import torch
    specs_s = scenes.make_batch_specs(48, 0)
    specs = [(s.width, s.height, s.max_disp, s.levels, s.window, s.radius) for s in specs_s]
    sx, zb = autotune.tune_batch(specs)
    assert all(v in (1, 2) for v in sx)
    scs = [scenes.make_pair(s, 1000 + i) for i, s in enumerate(specs_s)]
    Ls = [torch.from_numpy(s.left).cuda() for s in scs]
    Rs = [torch.from_numpy(s.right).cuda() for s in scs]
    b = Batch(specs, sx, zb, flags=_mode(grouped))
    d, c = b.run(Ls, Rs)
    b.sync()
    evals = b.eval_count()
    ties = _check_batch(b, specs, [s.left for s in scs], [s.right for s in scs], Ls, Rs, d, c)
    npx = sum(w * h for (w, h, *_r) in specs)
    assert ties <= 1e-3 * npx, ties
    for i, s in enumerate(specs_s):
        bad = scenes.bad_rate(d[i].cpu().numpy(), scs[i].gt, scs[i].mask, 1.0)
        assert bad < 0.25, (i, bad)
    assert evals > 0


def test_sampled_oracle_levels_from_batch_output():
    # a flat (K = 1) batched pair checked against the oracle directly
    from paper_1901_09593_gb300 import Batch
    import torch
    rng = np.random.default_rng(3)
    a = rng.integers(0, 256, (64, 150), dtype=np.uint8)
    bb = rng.integers(0, 256, (64, 150), dtype=np.uint8)
    spec = (150, 64, 48, 1, 7, 2)
    b = Batch([spec], [2], [64])
    d, c = b.run([torch.from_numpy(a).cuda()], [torch.from_numpy(bb).cuda()])
    b.sync()
    do, co, c2, _ = oracle.match_level(a, bb, 3, 48)
    compare_level(d[0].cpu().numpy(), c[0].cpu().numpy(), do, co, c2, "batched flat")


@MODES
def test_withheld_dependency_times_out_and_reports(grouped):
    # persistent mode: the queue withholds its first stage and every dependent wait gives up;
    # grouped mode: every tile's TMA wait gives up at once
    from paper_1901_09593_gb300 import Batch, _lib
    specs = [(96, 64, 16, 2, 5, 2), (64, 48, 16, 2, 5, 1)]
    Lh, Rh, Ls, Rs = _pairs(specs, 5)
    b = Batch(specs, flags=_lib.MSBM_FLAG_TEST_TIMEOUT | _mode(grouped))
    b.run(Ls, Rs)
    with pytest.raises(_lib.MsbmError) as ei:
        b.sync()
    assert ei.value.status == _lib.MSBM_ERR_TIMEOUT
    b.close()
    ok = Batch(specs, flags=_mode(grouped))
    d, c = ok.run(Ls, Rs)
    ok.sync()
    _check_batch(ok, specs, Lh, Rh, Ls, Rs, d, c)


def test_autotuner_choices_do_not_change_results():
    from paper_1901_09593_gb300 import Context, autotune
    import torch
    res = autotune.tune_full_level(350, 250, 64, 7, reps=3, cache_path=None)
    assert res["sx"] in (1, 2, 4) and res["zblock"] % 32 == 0 and len(res["table"]) >= 3
    rng = np.random.default_rng(9)
    a = torch.from_numpy(rng.integers(0, 256, (250, 350), dtype=np.uint8)).cuda()
    b = torch.from_numpy(rng.integers(0, 256, (250, 350), dtype=np.uint8)).cuda()
    outs = []
    for sx, zb in [(1, 32), (2, 96), (4, 64), (res["sx"], res["zblock"])]:
        ctx = Context(350, 250, 64, 1, 7, 0)
        ctx.set_level_tuning(0, sx, zb)
        d, c = ctx.disparity(a, b)
        ctx.sync()
        outs.append((d.cpu().numpy(), c.cpu().numpy()))
    for d, c in outs[1:]:
        np.testing.assert_array_equal(d, outs[0][0])
        np.testing.assert_array_equal(c, outs[0][1])
