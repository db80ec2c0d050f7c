import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


@pytest.fixture(scope="session")
def c1_small():
    """A reduced C1-shaped workload (mixture of Gaussians, d=96, d'=32) that
    the oracle finishes in seconds: (index, queries, reduced FP32 rows, V)."""
    from paper_2503_21206_b300 import index_build, synth
    w = synth.WORKLOADS["c1_mixture_20k_d96"]
    return index_build.build_workload(w, n=4000, nq=64)
