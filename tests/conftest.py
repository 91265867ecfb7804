import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libbm.so")


@pytest.fixture(scope="session")
def bmlib():
    """The built library (compiled in-tree on first use) and its binding."""
    from paper_2512_14193_gb300 import build as B
    B.build()
    from paper_2512_14193_gb300 import bm
    bm.lib()
    return bm


@pytest.fixture()
def handle(bmlib):
    h = bmlib.bm_create(0)
    yield h
    bmlib.bm_destroy(h)
