import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: large inputs; still part of the default run")


# Upper bound on one test's wall time where pytest-timeout is installed (the
# slowest test takes about 20 s): a test that stops making progress fails
# after it instead of holding the run, and the GPU, until an outer limit.
TEST_TIME_LIMIT_S = 600


def pytest_collection_modifyitems(config, items):
    if config.pluginmanager.hasplugin("timeout"):
        for item in items:
            if item.get_closest_marker("timeout") is None:
                item.add_marker(pytest.mark.timeout(TEST_TIME_LIMIT_S))
    # GPU tests cannot run without a device; skip them loudly rather than fail on import.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover - torch missing entirely
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
