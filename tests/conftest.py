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
    """Measured parity errors; written to gpurun_out/parity_errors.json (when
    that folder exists) at the end of the session, for the design notes."""
    return _REPORT


def pytest_sessionfinish(session, exitstatus):
    out = os.path.join(ROOT, "gpurun_out")
    if _REPORT and os.path.isdir(out):
        import json
        with open(os.path.join(out, "parity_errors.json"), "w") as f:
            json.dump(_REPORT, f, indent=1, sort_keys=True)
