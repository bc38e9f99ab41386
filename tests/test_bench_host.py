"""Host-side accounting of bench.py (CPU): the evaluation counts it divides by agree with
the oracle's own counts, the roofline denominators and work units are what the design
states, and the measured-traffic record is only used while its sources are unchanged."""
import numpy as np
import pytest

import bench
import oracle
from paper_1901_09593_gb300 import scenes


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _pair(h, w, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 256, size=(h, w), dtype=np.uint8)
    b = np.roll(a, 3, axis=1)
    return a, b


def test_full_evals_matches_oracle_count():
    # Eq. 3-4: every pixel evaluates 0 <= z <= min(D_k - 1, x)
    for h, w, dk in ((5, 7, 3), (9, 12, 20), (4, 30, 8)):
        a, b = _pair(h, w, h * w)
        *_, ev = oracle.match_level(a, b, 1, dk)
        assert bench.full_evals(w, h, dk) == ev


def test_restricted_evals_matches_oracle_count():
    # Eq. 8-9 first branch: dhat -/+ r around 2 * prior(y/2, x/2), clipped to the admissible range
    rng = np.random.default_rng(5)
    for h, w, dk, r in ((6, 9, 8, 1), (11, 14, 12, 2), (8, 20, 5, 3)):
        a, b = _pair(h, w, h + w)
        prior = rng.integers(0, (dk + 1) // 2 + 2, size=((h + 1) // 2, (w + 1) // 2)).astype(np.int16)
        *_, ev = oracle.match_level(a, b, 1, dk, r, prior)
        assert bench.restricted_evals(prior, w, h, dk, r) == ev


def test_alu_peak_and_ops_per_eval():
    assert bench.alu_peak_tops(152, 2070.0) == pytest.approx(152 * 128 * 2070e6 / 1e12)
    # one dp4a per 4 window bytes per row plus 5 lane-ops: 7 x 7 -> 7 * 2 + 5
    assert bench.ops_per_eval_restricted(7) == 19
    assert bench.ops_per_eval_restricted(5) == 5 * 2 + 5
    assert bench.ops_per_eval_restricted(9) == 9 * 3 + 5


def test_stage_work_units():
    spec = scenes.SPECS["bench_1400x1000"]
    wh = [oracle.level_size(spec.width, spec.height, k) for k in range(spec.levels)]
    ev = [10, 20, 30, 40]
    bound, work, unit = bench.stage_work("pyramid", spec, wh, ev)
    assert (bound, unit) == ("hbm", "B") and work > 2 * spec.width * spec.height
    # statistics: one right-image byte read and 8 plane bytes written per pixel of levels 0..K-2
    assert bench.stage_work("statistics", spec, wh, ev) == ("hbm", sum(9 * w * h for w, h in wh[:-1]), "B")
    # matching stages count the window's dp4a (7 x 7: 7 rows x 2 words) per evaluation
    assert bench.dp4a_per_eval(7) == 14 and bench.dp4a_per_eval(9) == 27 and bench.dp4a_per_eval(5) == 10
    assert bench.stage_work("full_level3", spec, wh, ev) == ("dp4a", 40 * 14, "dp4a")
    assert bench.stage_work("restricted_level1", spec, wh, ev) == ("dp4a", 20 * 14, "dp4a")


def test_equal_or_better_picks_fastest_admissible_method():
    methods = {"a": {"frames_per_s": 100.0, "bad1": 0.02},
               "b": {"frames_per_s": 50.0, "bad1": 0.01},
               "c": {"frames_per_s": 80.0, "bad1": 0.015}}
    got = bench.equal_or_better(methods, 10.0, 0.015)
    assert got["method"] == "c" and got["speedup"] == pytest.approx(8.0)
    assert bench.equal_or_better(methods, 10.0, 0.001) is None


def test_measured_traffic_only_for_recorded_kernels():
    assert bench.measured_traffic("no_such_kernel") is None
    rec = bench.MEASURED_TRAFFIC["restricted_level0"]
    got = bench.measured_traffic("restricted_level0")
    assert got is None or got == rec["bytes"]


def test_reference_rows_bound_the_reference_run():
    # whole frames while they fit the budget
    assert bench.reference_rows(1000, 4, 0.2, 100, 150.0) == 1000
    # otherwise a band from the top, a multiple of 2^(K-1) rows, sized to the budget
    rows = bench.reference_rows(1000, 4, 0.2, 2000, 150.0)
    assert rows % 8 == 0 and rows <= 1000 * 150.0 / (2000 * 0.2) and rows > 1000 * 150.0 / (2000 * 0.2) - 8
    assert bench.reference_rows(1000, 4, 5.0, 10000, 1.0) == 8


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    # under torchrun every rank but 0 exits at once, printing nothing
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]) == 0
    assert capsys.readouterr().out == ""


def test_warmup_below_three_is_refused():
    with pytest.raises(SystemExit):
        bench.main(["--warmup", "2"])
