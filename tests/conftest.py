import os
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if REPO not in sys.path:
    sys.path.insert(0, REPO)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload")


@pytest.fixture(scope="session", autouse=True)
def _native_host_builds():
    """Builds the host-side C modules (input generators, CPU oracle)."""
    from paper_2111_09947_gb300 import _build
    from oracle import build as oracle_build
    _build.build_synth()
    oracle_build.build()
