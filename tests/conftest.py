import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library through its Python binding; the test fails loudly if it
    cannot load or no GPU is visible."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("a gpu-marked test ran without a visible CUDA device")
    from paper_2002_08014_gb300 import binding
    binding.load()
    return binding
