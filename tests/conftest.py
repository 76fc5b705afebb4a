import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def semlib():
    """The CUDA library, built in-tree if stale (nvcc cross-compiles without a GPU)."""
    import paper_2312_09888_gb300 as S
    S.build_library()
    S.get_lib()
    return S


@pytest.fixture(scope="session")
def gpu(semlib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    return semlib


@pytest.fixture
def sess(gpu):
    s = gpu.Session(0)
    yield s
    s.close()
