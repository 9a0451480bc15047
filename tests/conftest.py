import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


_ACCURACY: dict = {}


@pytest.fixture(scope="session")
def accuracy_record():
    """Collects per-workload error figures; with BSF_ACCURACY_OUT set they are
    written there as JSON when the session ends."""
    return _ACCURACY


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("BSF_ACCURACY_OUT")
    if path and _ACCURACY:
        import json
        with open(path, "w") as fh:
            json.dump(_ACCURACY, fh, indent=1, sort_keys=True)
