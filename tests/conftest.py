import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_built():
    import oracle
    oracle.build()
    return oracle


def pytest_sessionfinish(session, exitstatus):
    """Write the deviations recorded by precision_bounds.check16 when
    FE_DEVIATION_LOG names a file."""
    path = os.environ.get("FE_DEVIATION_LOG")
    if not path:
        return
    try:
        import json
        from precision_bounds import DEVIATIONS
    except ImportError:
        return
    with open(path, "w") as f:
        json.dump(DEVIATIONS, f, indent=1)
