import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle():
    import oracle as o
    return o.default()


@pytest.fixture(scope="session")
def lslib():
    from paper_1511_07207_gb300 import binding
    return binding.load()


@pytest.fixture(scope="session")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="session")
def ctx(gpu, lslib):
    import torch
    from paper_1511_07207_gb300 import binding
    h = binding.ls_create(0, torch.cuda.current_stream(gpu))
    yield h
    binding.ls_destroy(h)
