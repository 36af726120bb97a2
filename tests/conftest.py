import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def cat_lib():
    """Builds (if stale) and loads libcatalan.so."""
    from paper_2601_11621_gb300 import build, capi
    build.build()
    return capi


@pytest.fixture(scope="session")
def ctx(cat_lib):
    """A libcatalan context on cuda:0 (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cat_lib.Context(0)
    yield c
    c.close()
