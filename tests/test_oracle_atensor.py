"""Pins of the oracle's precomputed projection tensors (App. C, Sec. 2.5).

* the pair relations A^{P,D} = pi_n A^{P,C}, A^{D,P} = pi_n' A^{C,P},
  A^{C,D} = A^{D,C} between tensors built independently for all six pairs,
  so that storing three of them loses nothing;
* the couplings assembled from the three stored tensors equal the oracle's
  projections (Eqs. proj_VP/VC/VD) for random states, with and without
  feedback;
* point-group covariance A(S q, S l) = C C C C A(q, l) (App. C) for q and l
  inside the zone (the folding reading of the half-momentum convention
  breaks it on the zone boundary, as for the state itself);
* the index symmetries of App. C for (P, C) under exchange of the form-factor
  indices and momentum inversion, inside the zone.
"""
import numpy as np
import pytest

import workloads as W
from oracle import atensor as at
from oracle import formfactors as ffm
from oracle import projections as pj
from tests.conftest import make_problem


@pytest.fixture(scope="module")
def small():
    prob = make_problem(shells=1, nc=4)
    return prob, {pair: at.a_tensor(prob, *pair) for pair in pj.SIGNATURES}


def test_pair_relations_between_independently_built_tensors(small):
    prob, A = small
    par = prob.basis.parity
    sc = max(np.abs(a).max() for a in A.values())
    assert sc > 0.1
    assert np.abs(A[("P", "D")] - par[None, None, :, None, None, None] * A[("P", "C")]).max() \
        <= 1e-14 * sc
    assert np.abs(A[("D", "P")] - par[None, None, None, None, None, :] * A[("C", "P")]).max() \
        <= 1e-14 * sc
    assert np.abs(A[("C", "D")] - A[("D", "C")]).max() <= 1e-14 * sc
    A3 = {pair: A[pair] for pair in at.STORED}
    for pair in pj.SIGNATURES:
        assert np.abs(at.pair_tensor(prob, A3, *pair) - A[pair]).max() <= 1e-14 * sc


@pytest.mark.parametrize("shells,nc,feedback", [(1, 4, True), (2, 4, True), (1, 6, True),
                                                (1, 4, False)])
def test_assembly_from_stored_tensors_equals_projections(shells, nc, feedback):
    prob = make_problem(shells=shells, nc=nc, U=2.6, feedback=feedback)
    A3 = at.stored_tensors(prob)
    for seed in (3, 4):
        y = W.random_state(seed, prob.nl, prob.nff)
        ref = pj.project(prob, y)
        got = at.project_with_tensors(prob, y, A3)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _index(prob):
    return {tuple(u): i for i, u in enumerate(prob.l_units)}


def test_point_group_covariance_inside_the_zone(small):
    prob, A = small
    lu = prob.l_units
    index = _index(prob)
    inner = np.nonzero(np.all(np.abs(lu) < prob.ncx, axis=1))[0]
    for pair in at.STORED:
        a = A[pair]
        sc = np.abs(a).max()
        for S in ffm.POINT_GROUP:
            C = prob.basis.rep_matrix(S)
            for li in inner:
                lj = index[tuple(S @ lu[li])]
                for qi in inner:
                    qj = index[tuple(S @ lu[qi])]
                    rot = np.einsum("mi,nj,ak,bl,ijkl->mnab", C, C, C, C, a[li, :, :, qi])
                    assert np.abs(a[lj, :, :, qj] - rot).max() <= 1e-13 * sc


def test_index_symmetries_of_the_pc_tensor_inside_the_zone(small):
    prob, A = small
    a = A[("P", "C")]
    par = prob.basis.parity
    pmn = par[:, None] * par[None, :]
    lu = prob.l_units
    index = _index(prob)
    inner = np.nonzero(np.all(np.abs(lu) < prob.ncx, axis=1))[0]
    sc = np.abs(a).max()
    for li in inner:
        lm = index[tuple(-lu[li])]
        for qi in inner:
            qm = index[tuple(-lu[qi])]
            blk = a[li, :, :, qi]                   # [m][n][m'][n']
            neg_q = a[li, :, :, qm]
            # A_{n,m,m',n'}(q, l) = pi_m pi_n A_{m,n,m',n'}(-q, l)
            assert np.abs(np.swapaxes(blk, 0, 1) - pmn[:, :, None, None] * neg_q).max() \
                <= 1e-13 * sc
            # A_{m,n,n',m'}(q, l) = pi_m pi_n A_{m,n,m',n'}(-q, l)
            assert np.abs(np.swapaxes(blk, 2, 3) - pmn[:, :, None, None] * neg_q).max() \
                <= 1e-13 * sc
            # A(-q, -l) = pi_m pi_n pi_m' pi_n' A(q, l)
            p4 = pmn[:, :, None, None] * pmn[None, None, :, :]
            assert np.abs(a[lm, :, :, qm] - p4 * blk).max() <= 1e-13 * sc
