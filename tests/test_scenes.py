"""The seeded input generator (the synthetic stand-in for the paper's stereo benchmark pairs,
Sec. IV) follows its recipe: deterministic per seed, exact warps for integer disparities,
the photometric change applied to the right view only, ground truth and mask rules, the
mixed-batch size rule, and the bad-pixel rate."""
import dataclasses

import numpy as np
import pytest

from paper_1901_09593_gb300 import scenes

SMALL = scenes.SceneSpec(96, 64, 4, 16, 2, 5, 2, 0.0, False)


def test_make_pair_is_deterministic_per_seed():
    a, b, c = scenes.make_pair(SMALL, 3), scenes.make_pair(SMALL, 3), scenes.make_pair(SMALL, 4)
    for f in ("left", "right", "gt", "mask", "labels"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.left, c.left)
    assert a.left.dtype == np.uint8 and a.right.dtype == np.uint8


def test_integer_shift_scene_warps_exactly():
    # constant integer disparity per region, no noise: every masked left pixel is found
    # unchanged in the right view at column x - gt (left reference, Eq. 1 sign reading)
    for seed in range(3):
        sc = scenes.make_pair(SMALL, seed)
        ys, xs = np.nonzero(sc.mask)
        assert len(ys) > 0.3 * sc.mask.size
        g = sc.gt[ys, xs].astype(np.int64)
        np.testing.assert_array_equal(sc.right[ys, xs - g], sc.left[ys, xs])


def test_photometric_change_applies_to_the_right_view_only():
    spec = dataclasses.replace(SMALL, gain=1.2, offset=-10.0)
    sc, plain = scenes.make_pair(spec, 7), scenes.make_pair(SMALL, 7)
    np.testing.assert_array_equal(sc.left, plain.left)
    ys, xs = np.nonzero(sc.mask)
    g = sc.gt[ys, xs].astype(np.int64)
    want = np.clip(np.rint(1.2 * sc.left[ys, xs].astype(np.float64) - 10.0), 0, 255)
    np.testing.assert_array_equal(sc.right[ys, xs - g], want.astype(np.uint8))


@pytest.mark.parametrize("spec", [SMALL, scenes.SceneSpec(128, 80, 6, 32, 3, 7, 2, 3.0, True)])
def test_ground_truth_and_mask_rules(spec):
    sc = scenes.make_pair(spec, 11)
    n = spec.window // 2
    assert np.all(sc.gt == np.rint(sc.gt))
    assert sc.gt.min() >= 0 and sc.gt.max() <= spec.max_disp - 1
    assert not sc.mask[:n].any() and not sc.mask[-n:].any()
    assert not sc.mask[:, :n].any() and not sc.mask[:, -n:].any()
    xx = np.broadcast_to(np.arange(spec.width)[None, :], sc.gt.shape)
    assert np.all(xx[sc.mask] - sc.gt[sc.mask] >= 0)
    assert sc.mask.mean() > 0.3
    assert sc.labels.min() >= 0 and sc.labels.max() < spec.regions


def test_slanted_planes_vary_within_a_region():
    spec = scenes.SceneSpec(256, 160, 3, 64, 3, 5, 2, 0.0, True)
    sc = scenes.make_pair(spec, 2)
    varied = [np.ptp(sc.gt[(sc.labels == r) & sc.mask]) for r in range(spec.regions)
              if ((sc.labels == r) & sc.mask).sum() > 100]
    assert varied and max(varied) >= 1


def test_texture_spans_the_full_range():
    t = scenes.make_texture(np.random.Generator(np.random.PCG64(0)), 40, 50)
    assert t.min() == 0.0 and abs(t.max() - 255.0) < 1e-9


def test_float_pair_is_in_unit_range():
    spec = scenes.SceneSpec(80, 48, 4, 16, 1, 5, 0, 0.01, True)
    sc = scenes.make_float_pair(spec, 1)
    assert sc.left.dtype == np.float64 and sc.right.dtype == np.float64
    assert sc.left.min() >= 0 and sc.left.max() <= 1 and sc.right.min() >= 0 and sc.right.max() <= 1
    assert sc.gt.min() >= 0 and sc.gt.max() <= spec.max_disp - 1


def test_mixed_batch_size_rule():
    # D = W / 5 to the nearest multiple of 16 (half up); K the deepest pyramid whose
    # coarsest width ceil(W / 2^(K-1)) is still >= 160; window 5 or 7
    rule = {320: (240, 64, 2), 640: (480, 128, 3), 1280: (720, 256, 4), 1400: (1000, 288, 4),
            1920: (1080, 384, 4)}
    specs = scenes.make_batch_specs(200, 0)
    assert specs == scenes.make_batch_specs(200, 0)
    seen = set()
    for s in specs:
        h, d, k = rule[s.width]
        assert (s.height, s.max_disp, s.levels) == (h, d, k)
        assert s.window in (5, 7) and s.radius == 2 and s.slanted
        seen.add(s.width)
    assert seen == set(rule)


def test_bad_rate_by_hand():
    d = np.array([[0, 3, 5], [7, 9, 2]], np.int16)
    gt = np.array([[0.0, 1.0, 5.0], [9.0, 9.0, 0.0]])
    mask = np.array([[True, True, True], [True, False, True]])
    # masked errors 0, 2, 0, 2, 2: three above 1, none above 2
    assert scenes.bad_rate(d, gt, mask, 1.0) == pytest.approx(3 / 5)
    assert scenes.bad_rate(d, gt, mask, 2.0) == 0.0
    assert scenes.bad_rate(d, gt, np.zeros_like(mask), 1.0) == 0.0
