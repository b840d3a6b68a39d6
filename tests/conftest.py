import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN


def pytest_terminal_summary(terminalreporter):
    """Print the parity exclusion counts of every GPU parity check that ran."""
    mod = sys.modules.get("tests.parity_util")
    reports = getattr(mod, "REPORTS", None) if mod else None
    if not reports:
        return
    terminalreporter.write_sep("-", "parity exclusions (FP64 near-ties; bound 5 % of queries)")
    for name, rep in reports:
        terminalreporter.write_line(f"{name}: {rep}")
