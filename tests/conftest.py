import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def ctx():
    """A liblrfg context on cuda:0 (builds the library first if needed)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected without a CUDA device")
    from paper_1902_07455_gb300 import build
    build.build()
    import paper_1902_07455_gb300 as lr
    c = lr.Context(0)
    yield c
    c.close()
