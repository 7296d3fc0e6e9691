import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libpes.so")
    config.addinivalue_line("markers", "slow: long-running (full-size parity)")


@pytest.fixture(scope="session", autouse=True)
def _native_cpu_libs():
    """Build the CPU-side native pieces (workload generator, oracle) once."""
    from paper_2102_00514_gb300 import build
    import oracle
    build.build_synth()
    oracle.build()
    yield
