import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O


def pytest_terminal_summary(terminalreporter):
    """Rays waived from exact integer parity, per test and rule (threshold,
    tolerance_flip, perturbation; see parity.py)."""
    try:
        from parity import WAIVERS
    except ImportError:
        return
    terminalreporter.section("integer-parity waivers")
    if not WAIVERS:
        terminalreporter.write_line("none")
        return
    for test, c in sorted(WAIVERS.items()):
        terminalreporter.write_line(f"{test}: " + ", ".join(f"{k} {v}" for k, v in sorted(c.items())))
