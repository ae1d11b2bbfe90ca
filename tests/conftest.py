import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libfsc.so")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session", autouse=True)
def bounds_check_clean():
    """With FSC_LIBRARY=checked (the build with index checks), the whole session must end with no
    out-of-range index recorded by any kernel."""
    yield
    if os.environ.get("FSC_LIBRARY") != "checked":
        return
    import paper_2310_10939_gb300 as fsc
    rep = fsc.bounds_report()
    assert rep is None, f"out-of-range index recorded: {rep}"
