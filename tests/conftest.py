import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("FDTD_PARITY_LOG")
    if not path:
        return
    import json

    from tests.helpers import PARITY_LOG

    with open(path, "a") as f:
        for r in PARITY_LOG:
            f.write(json.dumps(r) + "\n")
