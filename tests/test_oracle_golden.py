"""The oracle reproduces its recorded regression fixture on this machine (the fixture was
written by tests/golden/make_golden.py; it checks cross-machine determinism, it is not a
pin of the method)."""
import os

import numpy as np


def test_oracle_reproduces_fixture(oracle_mod):
    from tests.golden.make_golden import fixture_lines
    here = os.path.join(os.path.dirname(__file__), "golden", "oracle_small.txt")
    stored = open(here).read().strip().split("\n")
    fresh = fixture_lines()
    assert stored[:4] == fresh[:4]
    assert stored[4] == fresh[4]
    c_s = np.array(stored[5].split()[1:], float)
    c_f = np.array(fresh[5].split()[1:], float)
    np.testing.assert_allclose(c_f, c_s, atol=1e-11)
