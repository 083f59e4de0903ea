import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("SV_PARITY_REPORT")
    if not path:
        return
    try:
        import bars
    except ImportError:
        return
    if bars.RECORDS:
        import json
        with open(path, "w") as f:
            json.dump(bars.RECORDS, f, indent=1)
