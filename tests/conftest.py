import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def gpu_lib():
    """Built libadvisor on a CUDA device (the CUDA path must be the one that runs)."""
    import torch
    from paper_2301_03636_gb300 import advisor, build
    assert torch.cuda.is_available(), "gpu tests need a CUDA device"
    build.build()
    return advisor.lib()
