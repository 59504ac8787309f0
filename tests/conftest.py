import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _clear_device_status(request):
    """The library's device status word is sticky across calls: clear it
    before every GPU test so that each test reads only its own flags."""
    if "gpu" in request.keywords:
        import torch
        if torch.cuda.is_available():
            from paper_2602_05179_gb300 import api
            torch.cuda.synchronize()
            api.status()
    yield
