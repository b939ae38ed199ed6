import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def small32():
    import gen
    w = gen.WORKLOADS["small32"]
    return w, gen.make_library(w["library"]), gen.make_grid(w["grid"])


@pytest.fixture(scope="session")
def screen_sample():
    """The 20k-ligand screening recipe cut to its first 64 ligands."""
    import gen
    w = gen.scaled("screen20k", 64)
    return w, gen.make_library(w["library"]), gen.make_grid(w["grid"])


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.lib()
    return oracle
