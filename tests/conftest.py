import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libmppi")
    config.addinivalue_line("markers", "slow: long-running test")


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle as O
    O.build()
    return O


@pytest.fixture(autouse=True)
def _clear_literal_misses():
    try:
        import parity_util
    except ImportError:
        yield
        return
    parity_util.LITERAL_MISSES.clear()
    yield


@pytest.hookimpl(hookwrapper=True)
def pytest_runtest_makereport(item, call):
    """A test whose only shortfall is a nominal-control miss beyond binary32
    reach (parity_util.compare decides it from the oracle alone) is reported
    as XFAIL with the literal errors, not as a pass."""
    outcome = yield
    rep = outcome.get_result()
    if rep.when != "call" or not rep.passed:
        return
    pu = sys.modules.get("parity_util")
    if pu is not None and pu.LITERAL_MISSES:
        rep.outcome = "skipped"
        rep.wasxfail = "nominal beyond binary32 reach: " + "; ".join(pu.LITERAL_MISSES)
