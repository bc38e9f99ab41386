"""The oracle runs clean under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

A copy of ``oracle/msbm_oracle.c`` is built with ``-fsanitize=address,undefined`` (every
finding aborts) and the pin suites run against it in a subprocess with the sanitizer
runtimes preloaded.  A control copy with a planted out-of-bounds read of the binomial
weights must abort, so that a sanitizer that is not active cannot pass for a clean run."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "msbm_oracle.c")
PIN_SUITES = ["tests/test_oracle_pyramid.py", "tests/test_oracle_zncc.py", "tests/test_oracle_wta.py",
              "tests/test_oracle_softargmax.py", "tests/test_oracle_gated.py"]
FLAGS = ["-O1", "-g", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fsanitize=address,undefined",
         "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]


def _runtime(name):
    gcc = shutil.which("gcc")
    if not gcc:
        return None
    p = subprocess.run([gcc, f"-print-file-name={name}"], capture_output=True, text=True)
    path = p.stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def _run(tmp_path, text):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc sanitizer runtimes not available")
    src = os.path.join(tmp_path, "msbm_oracle.c")
    so = os.path.join(tmp_path, "liboracle_variant.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", *FLAGS, "-o", so, src, "-lm"])
    os.utime(so)                                  # newer than its source: the variant loader keeps it
    env = dict(os.environ, MSBM_ORACLE_VARIANT_SRC=src, LD_PRELOAD=f"{asan}:{ubsan}",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1", UBSAN_OPTIONS="halt_on_error=1",
               OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, "-m", "pytest", *PIN_SUITES, "-x", "-q", "-p", "no:cacheprovider",
                        "--capture=no"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return p.returncode, p.stdout + p.stderr


def test_pins_pass_on_the_sanitized_oracle(tmp_path):
    rc, out = _run(str(tmp_path), open(SRC).read())
    assert rc == 0, out[-3000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out


def test_sanitizer_catches_a_planted_overflow(tmp_path):
    text = open(SRC).read()
    old = "s += (long)c[a + 2] * c[b + 2]"
    assert old in text
    rc, out = _run(str(tmp_path), text.replace(old, "s += (long)c[a + 3] * c[b + 2]"))
    assert rc != 0 and ("AddressSanitizer" in out or "runtime error" in out), out[-3000:]
