import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300 / sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="session")
def two_plate_fdm():
    """Whole-structure finite-difference rows of the two-plate structure (master 0)
    at h = 0.05 um (with its discrete energy) and h = 0.025 um (about 45 s)."""
    from paper_2507_09730_gb300 import workloads as W
    from tests import fdm_reference as F
    s = W.tiny_two_plate()
    c1, u1 = F.capacitance_row(s, 0, 0.05, energy=True)
    c2 = F.capacitance_row(s, 0, 0.025, rtol=1e-8)
    return s, (c1, u1), c2
