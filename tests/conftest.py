import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


_REPORT = {}


@pytest.fixture(scope="session")
def report():
    """Measured parity errors; merged into the JSON file named by the
    environment variable SPH_PARITY_REPORT (when set) at the end of the
    session: the measured margins of every parity test, kept to compare
    runs and to set tolerances from."""
    return _REPORT


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("SPH_PARITY_REPORT")
    if _REPORT and path:
        import json
        old = {}
        if os.path.exists(path):
            with open(path) as f:
                old = json.load(f)
        old.update(_REPORT)
        with open(path, "w") as f:
            json.dump(old, f, indent=1, sort_keys=True)
