"""The oracle's pins catch plausible mistakes (CPU).

Each mutant below is a copy of ``oracle/msbm_oracle.c`` with ONE planted mistake of the kind
that a restatement of the paper could plausibly contain: a dropped term, a wrong sign or
index, an off-by-one window or span, the other tie-break, the paper's literal prior without
the factor 2.  The pin suites (``tests/test_oracle_*.py`` without the regression fixture,
which compares the oracle with its own recorded output) run against every mutant in a
subprocess and must fail; the unmodified copy must pass, so that a broken harness cannot
look like a caught mistake.  Mutants only change arithmetic, never a buffer size, so every
mutant still runs within its buffers.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "msbm_oracle.c")
PIN_SUITES = ["tests/test_oracle_pyramid.py", "tests/test_oracle_zncc.py", "tests/test_oracle_wta.py",
              "tests/test_oracle_softargmax.py", "tests/test_oracle_gated.py"]

# (name, planted mistake, text in the oracle, replacement, which occurrence of the text)
MUTANTS = [
    # pyramid (Sec. III, Fig. 1; binomial reading)
    ("pyr_truncates", "pyramid truncates instead of rounding", "(s + 128) >> 8", "s >> 8", 0),
    ("pyr_weights", "binomial weights 1 4 4 4 1", "{1, 4, 6, 4, 1}", "{1, 4, 4, 4, 1}", 0),
    ("pyr_phase", "decimation keeps odd columns", "clampi(2 * x + b, 0, W - 1)", "clampi(2 * x + 1 + b, 0, W - 1)", 0),
    ("pyr_rows_phase", "decimation keeps odd rows", "clampi(2 * y + a, 0, H - 1)", "clampi(2 * y + 1 + a, 0, H - 1)", 0),
    ("level_disp_floor", "D_k = floor(D / 2^k)", "(int)((D + (1L << k) - 1) >> k)", "(int)(D >> k)", 0),
    # ZNCC (Eq. 1-2)
    ("zncc_plus_z", "right window at x + z", "long long b = B[(long)yy * W + clampi(x - z + j, 0, W - 1)];",
     "long long b = B[(long)yy * W + clampi(x + z + j, 0, W - 1)];", 0),
    ("zncc_window_short", "window columns -n .. n-1", "for (int j = -n; j <= n; ++j) {\n            long long a",
     "for (int j = -n; j < n; ++j) {\n            long long a", 0),
    ("zncc_no_mean", "cross term without the mean product", "double c = (double)(N * Sab - Sa * Sb);",
     "double c = (double)(N * Sab);", 0),
    ("zncc_va_twice", "denominator Va * Va", "sqrt((double)Va * (double)Vb)", "sqrt((double)Va * (double)Va)", 0),
    ("zncc_vb_mixed", "Vb from Sa", "long long Vb = N * Sbb - Sb * Sb;", "long long Vb = N * Sbb - Sa * Sb;", 0),
    ("zncc_rows_unclamped_b", "right rows read one row lower", "long long b = B[(long)yy * W",
     "long long b = B[(long)clampi(yy + 1, 0, H - 1) * W", 0),
    # WTA and the hierarchy (Eq. 3-4, 8-9)
    ("wta_ties_last", "ties go to the largest z", "if (rho > best) { second = best; best = rho; bz = z; }",
     "if (rho >= best) { second = best; best = rho; bz = z; }", 0),
    ("wta_no_second", "second-best value never updated", "else if (rho > second) second = rho;", ";", 0),
    ("wta_inadmissible", "candidates past the left border", "int zmax = Dk - 1 < x ? Dk - 1 : x;\n            int lo",
     "int zmax = Dk - 1;\n            int lo", 0),
    ("prior_no_factor2", "prior not scaled to the finer level", "int dh = clampi(2 * (int)prior[(long)py * Wp + px], 0, zmax);",
     "int dh = clampi((int)prior[(long)py * Wp + px], 0, zmax);", 0),
    ("prior_round_up", "prior sampled at (y+1)/2", "int py = clampi(y / 2, 0, Hp - 1)", "int py = clampi((y + 1) / 2, 0, Hp - 1)", 0),
    ("span_open", "span dhat - r .. dhat + r - 1", "hi = dh + r > zmax ? zmax : dh + r;", "hi = dh + r - 1 > zmax ? zmax : dh + r - 1;", 0),
    ("span_low", "span starts at dhat - r + 1", "lo = dh - r < 0 ? 0 : dh - r;", "lo = dh - r + 1 < 0 ? 0 : dh - r + 1;", 0),
    ("driver_level_disp", "level k searches D_{k+1} candidates", "n, oracle_level_disp(D, k),\n", "n, oracle_level_disp(D, k + 1),\n", 0),
    # differentiable level (Eq. 2 with epsilon; soft-argmax and its backward)
    ("eps_inside", "epsilon added once under the root", "return Sab / sqrt((Saa + eps) * (Sbb + eps));",
     "return Sab / sqrt(Saa * Sbb + eps);", 0),
    ("softmax_no_T", "softmax without the temperature", "double e = exp(rho[z] / T - m);\n                        s += e;",
     "double e = exp(rho[z] - m);\n                        s += e;", 0),
    ("bwd_no_centering", "dd/drho without the -d_soft term", "double grho = g * p * (z - dsoft) / T;",
     "double grho = g * p * z / T;", 0),
    ("bwd_drop_rho_term", "drho/da without the rho term", "double da = bc[t] / sq - r_ * ac[t] / (Saa + eps);",
     "double da = bc[t] / sq;", 0),
    ("bwd_wrong_var", "drho/db normalised by Saa", "double db = ac[t] / sq - r_ * bc[t] / (Sbb + eps);",
     "double db = ac[t] / sq - r_ * bc[t] / (Saa + eps);", 0),
    ("bwd_right_column", "right gradient sent to x + z", "gB[(long)yy * W + clampi(x - z + j, 0, W - 1)]",
     "gB[(long)yy * W + clampi(x + j, 0, W - 1)]", 0),
    ("sa_fwd_inadmissible", "soft-argmax over candidates past the left border",
     "int zmax = ndisp - 1 < x ? ndisp - 1 : x;", "int zmax = ndisp - 1;", 0),
    ("sa_bwd_inadmissible", "backward over candidates past the left border",
     "int zmax = ndisp - 1 < x ? ndisp - 1 : x;", "int zmax = ndisp - 1;", 1),
    ("sa_mean_biased", "window mean over N - 1", "ma /= N; mb /= N;", "ma /= N - 1; mb /= N - 1;", 0),
    ("bwd_p_without_T", "backward softmax without the temperature", "double p = exp(rho[z] / T - m) / s;",
     "double p = exp(rho[z] - m) / s;", 0),
    ("bwd_left_mirrored", "left gradient sent to the mirrored window column",
     "gA[(long)yy * W + clampi(x + j, 0, W - 1)] += grho * da;", "gA[(long)yy * W + clampi(x - j, 0, W - 1)] += grho * da;", 0),
    # gated steps (Sec. III-B, III-C, III-D)
    ("cubic_kernel", "cubic kernel with a = -3/4", "if (t < 1.0) return (1.5 * t - 2.5) * t * t + 1.0;",
     "if (t < 1.0) return (1.25 * t - 2.25) * t * t + 1.0;", 0),
    ("cubic_phase", "fine pixel at coarse (y/2 + 1/4)", "oracle_bicubic_at(Cc, Wc, Hc, 0.5 * y, 0.5 * x)",
     "oracle_bicubic_at(Cc, Wc, Hc, 0.5 * y + 0.25, 0.5 * x + 0.25)", 0),
    ("beta_inverted", "beta gate inverted", "int full = !(ch > beta);", "int full = ch > beta;", 0),
    ("alpha_window", "alpha average over 2 x 3", "for (int m = y - 1; m <= y + 1; ++m)", "for (int m = y - 1; m <= y; ++m)", 0),
    ("alpha_gate", "alpha refines confident pixels", "if (Cin[o] > alpha) continue;", "if (!(Cin[o] > alpha)) continue;", 0),
    ("median_upper", "upper median for an even count", "d_out[o] = (int16_t)v[(cnt - 1) / 2];", "d_out[o] = (int16_t)v[cnt / 2];", 0),
    ("median_voters", "every neighbour votes", "if (C[p] > alpha) v[cnt++] = d_in[p];", "v[cnt++] = d_in[p];", 0),
    ("median_3x3", "3 x 3 median neighbourhood", "for (int m = y - 2; m <= y + 2; ++m)\n                for (int q = x - 2; q <= x + 2; ++q)",
     "for (int m = y - 1; m <= y + 1; ++m)\n                for (int q = x - 1; q <= x + 1; ++q)", 0),
    ("halving_shift", "window halves one level early", "int n = n0 >> k;", "int n = n0 >> (k + 1);", 0),
    ("beta_axes", "cost prior sampled with x and y swapped", "oracle_bicubic_at(Cprior, Wp, Hp, 0.5 * y, 0.5 * x)",
     "oracle_bicubic_at(Cprior, Wp, Hp, 0.5 * x, 0.5 * y)", 0),
    # the full method's driver (Fig. 1 with the gates)
    ("full_median_beta", "median gated by beta", "oracle_selective_median(dk, ck, Wk, Hk, alpha, tmp);",
     "oracle_selective_median(dk, ck, Wk, Hk, beta, tmp);", 0),
    ("full_gate_alpha", "fallback gated by alpha", "beta, dk, ck, c2k, NULL, NULL);", "alpha, dk, ck, c2k, NULL, NULL);", 0),
    ("full_alpha_evals", "alpha evaluations counted as full 3 x 3", "cnt *= (x > 0) + 1 + (x < Wk - 1);", "cnt *= 3;", 0),
    ("full_no_halving", "window halving flag ignored", "n = (flags & 8) ? oracle_level_half_width(n0, k) : n0;",
     "n = n0;", 0),
]


def _mutate(text, old, new, occurrence):
    at = -1
    for _ in range(occurrence + 1):
        at = text.find(old, at + 1)
        if at < 0:
            raise AssertionError(f"oracle text not found (occurrence {occurrence}): {old!r}")
    return text[:at] + new + text[at + len(old):]


def _run_pins(src_path):
    env = dict(os.environ, MSBM_ORACLE_VARIANT_SRC=src_path, OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-m", "pytest", *PIN_SUITES, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    failed = [ln.split(" ")[1] for ln in p.stdout.splitlines() if ln.startswith("FAILED ")]
    return p.returncode, failed, p.stdout[-2000:] + p.stderr[-2000:]


def test_mutant_table_is_well_formed():
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    text = open(SRC).read()
    for name, _, old, new, occ in MUTANTS:
        assert old != new, name
        _mutate(text, old, new, occ)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    text = open(SRC).read()
    jobs = [("unmodified", text)] + [(m[0], _mutate(text, m[2], m[3], m[4])) for m in MUTANTS]
    paths = []
    for name, body in jobs:
        d = tmp_path_factory.mktemp(name)
        path = os.path.join(d, "msbm_oracle.c")
        with open(path, "w") as f:
            f.write(body)
        paths.append((name, path))
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda np_: (np_[0], _run_pins(np_[1])), paths))
    return dict(res)


def test_unmodified_copy_passes_every_pin(outcomes):
    rc, failed, tail = outcomes["unmodified"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_mutant(outcomes, name):
    rc, failed, tail = outcomes[name]
    # exit status 1: tests ran and at least one failed (not a crash, not a collection error)
    assert rc == 1 and failed, f"mutant {name} survived or crashed (rc={rc}):\n{tail}"
