import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled CUDA library")


@pytest.fixture(scope="session", autouse=True)
def _built_host_libs():
    """Compile the host-side helpers (generator and oracle) once per session."""
    import oracle
    from paper_2410_15451_gb300 import synth

    synth.build()
    oracle.build()
    yield
