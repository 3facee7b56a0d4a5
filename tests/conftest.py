import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) GPU and the CUDA library")
    config.addinivalue_line("markers", "slow: long CPU run (oracle at full size)")


@pytest.fixture(scope="session")
def sphere320_oracle():
    """Oracle of the 320-triangle sphere, fully assembled (about 15 s on 8 cores)."""
    from oracle.oracle import Oracle
    from workloads import workload

    w = workload("sphere320")
    o = Oracle(w.verts, w.tris, w.dt)
    o.assemble()
    return w, o


@pytest.fixture(scope="session")
def sphere320_march(sphere320_oracle):
    w, o = sphere320_oracle
    return o.march(w.pulses[0], w.Nt)
