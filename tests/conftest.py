import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


def make_problem(shells=1, nc=8, nf=16, t=1.0, tp=-0.25, mu=None, U=3.0, ncy=None, nfy=None,
                 **kw):
    """Oracle problem on the given grids (van Hove filling unless mu given)."""
    import workloads as W
    from oracle.model import Problem
    mu = 4.0 * tp if mu is None else mu
    return Problem(t, tp, mu, U, W.bonds_for_shells(shells), nc, ncy or nc, nf, nfy or nf,
                   **kw).check()


@pytest.fixture
def problem_factory():
    return make_problem
