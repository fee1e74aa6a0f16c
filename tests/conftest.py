import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and libcheb.so")


@pytest.fixture(scope="session")
def ctx():
    """One libcheb context on cuda:0 for the GPU tests (builds the library if needed)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_04688_gb300 import build as B
    B.build()
    import paper_2307_04688_gb300 as cb
    c = cb.Context(0)
    yield c
    c.device_status()
    c.close()
