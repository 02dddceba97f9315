import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _checked_build_report():
    """With the checked library (UFC_CHECKED=1), every test ends with a
    synchronize of the shared contexts, which reports a failed index test of
    any kernel the test ran (the record is per device)."""
    yield
    if os.environ.get("UFC_CHECKED") != "1":
        return
    api = sys.modules.get("paper_1801_05745_gb300.api")
    if api is None:
        return
    for ctx in list(api._ctxs.values()):
        if ctx.h:
            ctx.synchronize()
