"""Writes the oracle regression fixture ``oracle_small.txt``.

The paper prints no worked numeric example, so this fixture is not a pin of the method:
it records the oracle's own output on a small seeded input so that the test suite can
check that the oracle gives identical results on every machine it is built on (x86 and
Arm).  It calls only ``oracle`` and the seeded scene generator.
Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1901_09593_gb300 import scenes  # noqa: E402


def fixture_lines():
    sc = scenes.make_pair(scenes.SPECS["small_320x240"], 21)
    a, b = sc.left[100:132, 150:214].copy(), sc.right[100:132, 150:214].copy()
    lines = ["# oracle regression fixture: small_320x240 seed 21, crop rows 100:132 cols 150:214",
             "# D=32 K=3 window=5 radius=2; level-2 pyramid of the left crop, then level-0 d and C"]
    pyr = oracle.pyramid(a, 3)
    lines.append("pyr2 " + " ".join(str(int(v)) for v in pyr[2].ravel()))
    out = oracle.disparity(a, b, 32, 3, 5, 2)
    lines.append("evals %d" % out["evals"])
    lines.append("d0 " + " ".join(str(int(v)) for v in out["d"][0].ravel()))
    lines.append("C0 " + " ".join("%.12f" % v for v in out["C"][0].ravel()))
    return lines


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_small.txt"), "w") as f:
        f.write("\n".join(fixture_lines()) + "\n")
