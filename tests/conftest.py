import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libmsbm.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def _oracle_variant(src):
    """A private copy of the oracle package built from another C source (the mutation test
    points MSBM_ORACLE_VARIANT_SRC at a copy of the oracle with one planted mistake)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("oracle_variant", os.path.join(ROOT, "oracle", "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = src
    mod._OUT_DIR = os.path.dirname(os.path.abspath(src))
    mod._SO = os.path.join(mod._OUT_DIR, "liboracle_variant.so")
    mod.build()
    return mod


@pytest.fixture(scope="session")
def oracle_mod():
    src = os.environ.get("MSBM_ORACLE_VARIANT_SRC")
    if src:
        return _oracle_variant(src)
    import oracle
    oracle.build()
    return oracle
