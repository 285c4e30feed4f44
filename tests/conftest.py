import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def oracle():
    import oracle as o

    o.build()
    return o


@pytest.fixture(scope="session")
def parity_report():
    """Collects per-workload error statistics of the full-size parity tests; when the
    environment names a file in QMC_PARITY_REPORT they are written there as JSON at
    the end of the session (pytest's own output keeps only pass or fail)."""
    import json

    stats = {}
    yield stats
    path = os.environ.get("QMC_PARITY_REPORT")
    if path and stats:
        with open(path, "w") as f:
            json.dump(stats, f, indent=1, sort_keys=True)
