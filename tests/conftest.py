import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session", autouse=True)
def _build_cpu_parts():
    """The oracle and the scene generator are plain C compiled with gcc on first use."""
    import oracle
    import synth
    oracle.build()
    synth.build()
