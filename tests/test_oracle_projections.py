"""Pins of the oracle's projections (Eqs. proj_VP/VC/VD, proj-P/C/D, proj_pos).

* the position-space route equals the literal double sum over the coarse
  grid for all six cross pairs, including grids small enough to alias;
* the full projected interaction B[V] equals the assembled V^B;
* own channel B[Phi^B] = B and bare V0 -> U e0 e0^T (initial condition);
* A-tensor pair relations of App. C;
* App. B: no weight on f_n whose bond exceeds |R_m| + |R_c| + |R_c'|.
"""
import numpy as np
import pytest

import workloads as W
from oracle import projections as pj
from tests.conftest import make_problem

CASES = [(1, 4), (1, 6), (2, 6), (3, 6), (3, 8), (4, 6), (5, 6)]


@pytest.mark.parametrize("shells,nc", CASES)
def test_position_space_equals_literal_definition(shells, nc):
    prob = make_problem(shells=shells, nc=nc)
    y = W.random_state(11 + shells, prob.nl, prob.nff)
    for (T, S) in pj.SIGNATURES:
        B = y[pj.CHANNELS.index(S)]
        ref = pj.project_pair_bruteforce(prob, T, S, B)
        got = pj.project_pair(prob, T, S, B)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("shells,nc", [(1, 4), (2, 6), (3, 8)])
def test_assembled_couplings_equal_projected_full_interaction(shells, nc):
    prob = make_problem(shells=shells, nc=nc, U=2.7)
    y = W.random_state(5, prob.nl, prob.nff)
    assert np.allclose(pj.project(prob, y), pj.project_bruteforce(prob, y), atol=1e-12)


@pytest.mark.parametrize("shells,nc", [(1, 4), (3, 6), (5, 8)])
def test_own_channel_identity(shells, nc):
    prob = make_problem(shells=shells, nc=nc)
    y = W.random_state(7, prob.nl, prob.nff)
    for ci, ch in enumerate(pj.CHANNELS):
        assert np.allclose(pj.project_pair_bruteforce(prob, ch, ch, y[ci]), y[ci], atol=1e-13)


def test_bare_interaction_is_onsite_u_in_every_channel():
    # initial condition of the flow: P = C = D = 0  ->  V^B = U e0 e0^T
    prob = make_problem(shells=3, nc=6, U=3.0)
    V = pj.project(prob, np.zeros((3, prob.nl, prob.nff, prob.nff)))
    e = np.zeros((prob.nff, prob.nff))
    e[0, 0] = 3.0
    assert np.allclose(V, e[None, None], atol=1e-15)


def test_a_tensor_pair_relations():
    # App. C: A^{P,C} = pi_n A^{P,D}, A^{C,P} = pi_n' A^{D,P}, A^{D,C} = A^{C,D}
    prob = make_problem(shells=4, nc=6)
    par = prob.basis.parity
    X = W.random_state(2, prob.nl, prob.nff)[0]
    pc = pj.project_pair(prob, "P", "C", X)
    pd = pj.project_pair(prob, "P", "D", X)
    assert np.allclose(pc, pd * par[None, None, :], atol=1e-13)
    cp = pj.project_pair(prob, "C", "P", X)
    dp = pj.project_pair(prob, "D", "P", X * par[None, None, :])
    assert np.allclose(cp, dp, atol=1e-13)
    assert np.allclose(pj.project_pair(prob, "D", "C", X), pj.project_pair(prob, "C", "D", X),
                       atol=1e-13)


def test_bond_length_bound_of_appendix_b():
    prob = make_problem(shells=5, nc=10)
    R = prob.basis.bonds
    shell_len = {s: np.sqrt(r2) for s, r2 in enumerate([0, 1, 2, 4, 5, 8])}
    ln = np.array([shell_len[s] for s in prob.basis.shells])
    rng = np.random.default_rng(4)
    for c, cp in [(0, 0), (0, 1), (1, 5), (2, 7)]:
        X = np.zeros((prob.nl, prob.nff, prob.nff))
        X[:, c, cp] = X[:, cp, c] = rng.standard_normal(prob.nl)
        for T, S in [("D", "P"), ("D", "C"), ("P", "C"), ("C", "P")]:
            out = pj.project_pair(prob, T, S, X)
            bound = ln[:, None] + ln[c] + ln[cp] + 1e-9
            forbidden = ln[None, :] > bound
            assert np.abs(out[:, forbidden]).max() <= 1e-13 * max(np.abs(out).max(), 1e-30)
