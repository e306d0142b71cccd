"""Fermi-surface-refined loop integration on the GPU (Sec. 3, the adaptive
cubature's role) against the oracle's refined loops, through the C ABI: the
loops of every l (FP64 and BF16x3 contexts, square and rectangular grids,
s = 3 and 5), the right-hand side with the refined loops, the scale switch
Lambda_on, switching the refinement off again, and invalid settings."""
import numpy as np
import pytest

import workloads as W
from tests.conftest import make_problem

pytestmark = pytest.mark.gpu

BOUND = {"fp64": 1e-10, "bf16x3": 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_1604_06296_gb300 import build
    build.build()
    return t


def _pair(prob, s, kappa, lam_on, om):
    from oracle import refine as rf
    return rf.chi_dot_refined(prob, om, s=s, kappa=kappa, lam_on=lam_on)


CASES = [  # shells, nc, ncy, nf, precision, s, kappa, om
    (1, 4, None, 32, "fp64", 3, 8.0, 0.1),
    (1, 4, None, 32, "fp64", 5, 4.0, 0.05),
    (2, 6, None, 24, "fp64", 3, 6.0, 0.08),
    (1, 6, 4, 24, "fp64", 3, 8.0, 0.1),
    (1, 4, None, 32, "bf16x3", 5, 8.0, 0.1),
    (2, 8, None, 32, "bf16x3", 3, 6.0, 0.06),
]


@pytest.mark.parametrize("shells,nc,ncy,nf,prec,s,kappa,om", CASES)
def test_refined_loops_match_oracle(torch, shells, nc, ncy, nf, prec, s, kappa, om):
    from oracle import loops as lp
    from paper_1604_06296_gb300 import Solver
    prob = make_problem(shells=shells, nc=nc, ncy=ncy, nf=nf, tp=-0.3)
    sv = Solver(1.0, -0.3, -1.2, 3.0, W.bonds_for_shells(shells), nc, nf, precision=prec,
                ncy=ncy)
    plain = lp.chi_dot(prob, om)
    sv.set_refinement(s=s, kappa=kappa, lambda_on=1.0)
    got = sv.loops(om).cpu().numpy()
    ref = _pair(prob, s, kappa, 1.0, om)
    for ch in range(2):
        sc = np.abs(ref[ch]).max()
        assert np.abs(got[ch] - ref[ch]).max() <= BOUND[prec] * sc
        # the refinement moves the loops by more than the tolerance
        assert np.abs(ref[ch] - plain[ch]).max() > 10 * BOUND[prec] * sc
    # above Lambda_on nothing is refined
    sv.set_refinement(s=s, kappa=kappa, lambda_on=0.5 * om)
    got = sv.loops(om).cpu().numpy()
    for ch in range(2):
        assert np.abs(got[ch] - plain[ch]).max() <= BOUND[prec] * np.abs(plain[ch]).max()
    # off again
    sv.set_refinement(s=1)
    got = sv.loops(om).cpu().numpy()
    for ch in range(2):
        assert np.abs(got[ch] - plain[ch]).max() <= BOUND[prec] * np.abs(plain[ch]).max()
    sv.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_rhs_with_refined_loops_matches_oracle(torch, prec):
    from oracle import projections as pj
    from oracle import rhs as orhs
    from paper_1604_06296_gb300 import Solver
    om = 0.07
    prob = make_problem(shells=1, nc=6, nf=24, tp=-0.3, U=3.0)
    sv = Solver(1.0, -0.3, -1.2, 3.0, W.bonds_for_shells(1), 6, 24, precision=prec)
    sv.set_refinement(s=3, kappa=8.0)
    y = W.random_state(9, prob.nl, prob.nff, 0.3)
    pp, ph = _pair(prob, 3, 8.0, np.inf, om)
    ref = orhs.products(pj.project(prob, y), pp, ph)
    got = sv.rhs(om, torch.from_numpy(y).cuda()).cpu().numpy()
    tol = 1e-10 if prec == "fp64" else 2e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    sv.close()


def test_refinement_rejects_bad_settings(torch):
    from paper_1604_06296_gb300 import Solver, TufrgError
    sv = Solver(1.0, -0.3, -1.2, 3.0, W.bonds_for_shells(1), 4, 32)
    for args in ((2, 8.0, 1.0), (11, 8.0, 1.0), (3, -1.0, 1.0), (3, 8.0, -1.0),
                 (3, float("nan"), 1.0)):
        with pytest.raises(TufrgError) as e:
            sv.set_refinement(*args)
        assert e.value.status == -1
    sv.close()


def test_refined_loops_production_size_sampled(torch):
    """The production point (coarse 24x24, Nff 13, fine 480x480, BF16x3) with
    refinement s = 5, kappa = 8 at Lambda = 0.03: the loops of every l on the
    GPU against the oracle's refined loops at six l (zone boundary, interior,
    near the pairing momentum 0)."""
    from oracle import refine as rf
    from paper_1604_06296_gb300 import Solver
    c = W.config("cfg2")
    tp = c["tp"]
    prob = make_problem(shells=c["shells"], nc=c["nc"], nf=c["nf"], t=c["t"], tp=tp, mu=4 * tp,
                        U=c["U"])
    sv = Solver(c["t"], tp, 4 * tp, c["U"], W.bonds_for_shells(c["shells"]), c["nc"], c["nf"],
                precision="bf16x3")
    sv.set_refinement(s=5, kappa=8.0, lambda_on=0.1)
    om = 0.03
    got = sv.loops(om).cpu().numpy()
    ls = np.array([0, 13, 150, 288, 301, 575])
    pp, ph = rf.chi_dot_refined(prob, om, s=5, kappa=8.0, lam_on=0.1, l_index=ls)
    for ch, ref in enumerate((pp, ph)):
        assert np.abs(got[ch][ls] - ref).max() <= 1e-5 * np.abs(ref).max()
    sv.close()
