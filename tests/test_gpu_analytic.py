"""Analytic-xi mode on the GPU: fine grids whose points p +- l/2 fall between
grid points (nf not a multiple of 2 nc), where the FP64 loops take
xi(p +- l/2) of Eq. (hubb-disp) from per-row cosine tables.  Loops, the
right-hand side and RK4 steps against the oracle (which evaluates xi at
p +- l/2 directly for any grid), square and rectangular grids; tensor-core
precisions and the refinement refuse such grids."""
import numpy as np
import pytest

import workloads as W
from tests.conftest import make_problem

pytestmark = pytest.mark.gpu

T, TP, MU, U = 1.0, -0.3, -1.2, 3.0


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_1604_06296_gb300 import build
    build.build()
    return t


CASES = [  # shells, nc, ncy, nf, nfy
    (1, 8, None, 36, None),
    (2, 6, None, 40, None),
    (1, 6, 8, 40, 36),
]


def _pair(shells, nc, ncy, nf, nfy):
    from paper_1604_06296_gb300 import Solver
    prob = make_problem(shells=shells, nc=nc, ncy=ncy, nf=nf, nfy=nfy, t=T, tp=TP, mu=MU, U=U)
    sv = Solver(T, TP, MU, U, W.bonds_for_shells(shells), nc, nf, precision="fp64", ncy=ncy,
                nfy=nfy)
    assert nf % (2 * nc) != 0           # the grids of these cases are not aligned
    return prob, sv


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("shells,nc,ncy,nf,nfy", CASES)
def test_analytic_loops_match_oracle(torch, shells, nc, ncy, nf, nfy):
    from oracle import loops as lp
    prob, sv = _pair(shells, nc, ncy, nf, nfy)
    for om in (0.9, 0.08):
        got = sv.loops(om).cpu().numpy()
        ref = np.stack(lp.chi_dot(prob, om))
        for ch in range(2):
            assert _rel(got[ch], ref[ch]) <= 1e-10
    sv.close()


@pytest.mark.parametrize("shells,nc,ncy,nf,nfy", CASES)
def test_analytic_rhs_matches_oracle(torch, shells, nc, ncy, nf, nfy):
    from oracle import rhs as orhs
    prob, sv = _pair(shells, nc, ncy, nf, nfy)
    y = W.random_state(3, prob.nl, prob.nff, 0.3)
    got = sv.rhs(0.2, torch.from_numpy(y).cuda()).cpu().numpy()
    assert _rel(got, orhs.rhs(prob, 0.2, y)) <= 1e-10
    sv.close()


def test_analytic_rk4_flow_matches_oracle(torch):
    from oracle import flow as ofl
    prob, sv = _pair(1, 8, None, 36, None)
    lam0, lam1, steps = 4.0, 0.8, 4
    h = (np.log(lam1) - np.log(lam0)) / steps
    y, res, _ = sv.flow(lambda0=lam0, lambda_min=lam1, threshold=1e9, h0=abs(h), method="rk4")
    _, yref = ofl.rk4(ofl.log_rhs(prob), np.log(lam0),
                      np.zeros((3, prob.nl, prob.nff, prob.nff)), h, steps)
    assert res["n_accepted"] == steps and not res["diverged"]
    assert _rel(y.cpu().numpy(), yref) <= 1e-9
    sv.close()


def test_unaligned_grids_refused_by_table_only_paths(torch):
    from paper_1604_06296_gb300 import Solver, TufrgError
    b = W.bonds_for_shells(1)
    for prec in ("bf16x3", "3xtf32"):
        with pytest.raises(TufrgError) as e:
            Solver(T, TP, MU, U, b, 8, 36, precision=prec)
        assert e.value.status == -1
    sv = Solver(T, TP, MU, U, b, 8, 36, precision="fp64")
    with pytest.raises(TufrgError) as e:
        sv.set_refinement(s=3)
    assert e.value.status == -7
    sv.close()
