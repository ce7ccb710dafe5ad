import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_sessionstart(session):
    # libpint.so is built in-tree (nvcc cross-compiles without a GPU)
    import __graft_entry__
    __graft_entry__._build_module().build()


@pytest.fixture(scope="session")
def P():
    import paper_2504_02117_gb300 as mod
    return mod


@pytest.fixture(scope="session")
def ctx(P):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = P.pint_create(0)
    yield c
    P.pint_destroy(c)
