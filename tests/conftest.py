import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libasci")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """Print the parity reports filed during the session: per comparison the
    number of keys, the worst error / tolerance and how many keys needed the
    fallback (cancellation and denominator) bound."""
    from tests._parity import REPORTS
    if not REPORTS:
        return
    terminalreporter.write_sep("-", "parity report (keys, worst err/tol, keys beyond 1e-11 |S|)")
    for label, n, worst, nfb in REPORTS:
        terminalreporter.write_line(f"{label}: {n} keys, worst {worst:.3g}, fallback {nfb}")
