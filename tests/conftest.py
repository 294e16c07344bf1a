import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~10 s")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped (not failed) when no device is present, so the CPU
    # suite can be collected everywhere; -m gpu on a machine with a GPU runs them.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
