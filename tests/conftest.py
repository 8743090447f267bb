import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="session")
def gpu():
    """The CUDA library and a context on device 0 (skips where no GPU is present)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_00292_gb300 import build as grt_build
    from paper_2603_00292_gb300.objects import Context

    grt_build.build()
    ctx = Context(0)
    yield ctx
    torch.cuda.synchronize()
    ctx.close()
