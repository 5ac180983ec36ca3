import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libsp2.so")
    config.addinivalue_line("markers", "slow: long-running full-size check (opt in with SP2_SLOW=1)")


def have_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    gpu = have_gpu()
    slow = os.environ.get("SP2_SLOW") == "1"
    for it in items:
        if "gpu" in it.keywords and not gpu:
            it.add_marker(pytest.mark.skip(reason="no CUDA device"))
        if "slow" in it.keywords and not slow:
            it.add_marker(pytest.mark.skip(reason="set SP2_SLOW=1"))
