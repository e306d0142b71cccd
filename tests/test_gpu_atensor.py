"""Projections from the precomputed tensors A^{B,B'} (App. C, Sec. 2.5)
against the oracle's projections (Eqs. proj_VP/VC/VD) and the on-the-fly
path, through the C ABI, for FP64 and mixed-precision contexts, with and
without feedback, on square and rectangular coarse grids."""
import numpy as np
import pytest

import workloads as W
from tests.conftest import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_1604_06296_gb300 import build
    build.build()
    return t


CASES = [  # shells, nc, ncy, precision, feedback
    (1, 4, None, "fp64", True),
    (1, 8, None, "fp64", True),
    (2, 6, None, "fp64", True),
    (1, 6, 4, "fp64", True),
    (2, 4, None, "fp64", False),
    (1, 8, None, "bf16x3", True),
    (2, 6, None, "3xtf32", True),
]


@pytest.mark.parametrize("shells,nc,ncy,prec,feedback", CASES)
def test_atensor_projections_match_oracle(torch, shells, nc, ncy, prec, feedback):
    from oracle import projections as pj
    from paper_1604_06296_gb300 import Solver
    nf = 4 * max(nc, ncy or nc)
    prob = make_problem(shells=shells, nc=nc, ncy=ncy, nf=nf, U=2.7, feedback=feedback)
    s = Solver(1.0, -0.25, -1.0, 2.7, W.bonds_for_shells(shells), nc, nf, precision=prec,
               feedback=feedback, ncy=ncy)
    nl, nff = s.nl, s.nff
    cols = nl * nff * nff
    elem = 8 if prec == "fp64" else 4
    assert s.atensor_bytes() == elem * (3 * cols * cols + 4 * cols)
    s.atensor_build()
    tol = 1e-12 if prec == "fp64" else 2e-6
    for seed in (21, 22):
        y = W.random_state(seed, nl, nff, 0.3)
        ref = pj.project(prob, y)
        yd = torch.from_numpy(y).cuda()
        got = s.project_atensor(yd).cpu().numpy()
        fly = s.project(yd).cpu().numpy()
        sc = np.abs(ref).max()
        assert np.abs(got - ref).max() <= tol * sc
        assert np.abs(got - fly).max() <= tol * sc
    s.close()


def test_atensor_refusals(torch):
    from paper_1604_06296_gb300 import Solver, TufrgError
    s = Solver(1.0, -0.25, -1.0, 3.0, W.bonds_for_shells(1), 4, 16)
    y = s.zeros(3)
    with pytest.raises(TufrgError) as e:      # before the tensors exist
        s.project_atensor(y)
    assert e.value.status == -7
    s.close()
    big = Solver(1.0, -0.25, -1.0, 3.0, W.bonds_for_shells(3), 8, 32)   # 13 form factors
    with pytest.raises(TufrgError) as e:
        big.atensor_bytes()
    assert e.value.status == -1
    with pytest.raises(TufrgError):
        big.atensor_build()
    big.close()
