import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libodp.so")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    try:
        import parity_log
    except ImportError:
        return
    if parity_log.NOTES:
        terminalreporter.section("parity numbers")
        for test, text in parity_log.NOTES:
            terminalreporter.write_line("%s: %s" % (test, text))
