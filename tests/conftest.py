import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(autouse=True)
def _no_failed_address_checks(request):
    """Under the address-checked library (MPDO_LIBRARY=bounds) every GPU test must end with no failed
    address check in any kernel it launched."""
    yield
    if os.environ.get("MPDO_LIBRARY") != "bounds" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2508_07610_gb300 import mpdo as G

    rep = G.bounds_read()
    assert rep["failures"] == 0, f"failed address checks: {rep}"
