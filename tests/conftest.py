import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as O
    O.lib()
    return O


@pytest.fixture
def gp():
    """Factory of GpuProblem contexts on cuda:0, destroyed after the test."""
    from gpu_util import GpuProblem
    made = []

    def make(problem):
        g = GpuProblem(problem)
        made.append(g)
        return g

    yield make
    for g in made:
        g.close()
