"""App. C invariants of the flowing state with full inter-channel feedback:
B_mn = B_nm, P = pi_m pi_n P, C(-l) = C(l), D(-l) = D(l), and C4v
covariance B(S l) = C^S B(l) C^S^T for l inside the zone (the folding reading
of the half-momentum convention breaks covariance on the zone boundary)."""
import numpy as np

from oracle import flow as fl
from oracle import formfactors as ffm
from tests.conftest import make_problem


def test_flow_state_invariants():
    prob = make_problem(shells=2, nc=6, nf=24, tp=-0.3)
    y = fl.flow(prob, 10.0, 0.05, 1e9, rtol=1e-9, atol=1e-11).y
    sc = np.abs(y).max()
    assert sc > 0.5
    assert np.abs(y - np.swapaxes(y, -1, -2)).max() <= 1e-14 * sc
    par = prob.basis.parity
    odd = (par[:, None] * par[None, :]) < 0
    assert np.abs(y[0][:, odd]).max() <= 1e-14 * sc
    lu = prob.l_units
    index = {tuple(u): i for i, u in enumerate(lu)}
    interior = np.all(np.abs(lu) < prob.ncx, axis=1)
    for li in np.nonzero(interior)[0]:
        lj = index[tuple(-lu[li])]
        assert np.abs(y[1:, lj] - y[1:, li]).max() <= 1e-14 * sc
    for S in ffm.POINT_GROUP:
        C = prob.basis.rep_matrix(S)
        for li in np.nonzero(interior)[0]:
            lj = index[tuple(S @ lu[li])]
            assert np.abs(y[:, lj] - C @ y[:, li] @ C.T).max() <= 1e-13 * sc


def test_flowing_state_projections_and_rhs_covariant_on_boundary_subgroup():
    """App. C covariance on the zone boundary: for every element g that maps
    l into [-pi, pi)^2 without a fold, the flowing state, its projections
    and its right-hand side satisfy X(g l) = C^g X(l) C^g^T (to rounding);
    the elements that need a fold do not (the half momentum moves by pi)."""
    from oracle import projections
    from oracle import rhs as orhs
    prob = make_problem(shells=2, nc=6, nf=24, tp=-0.3)
    y = fl.flow(prob, 10.0, 0.3, 1e9, rtol=1e-9, atol=1e-11).y
    V = projections.project(prob, y)
    dy = orhs.rhs(prob, 0.3, y)
    lu = prob.l_units
    n = prob.ncx
    index = {tuple(u): i for i, u in enumerate(lu)}
    boundary = np.nonzero(np.any(lu == -n, axis=1))[0]
    for X in (y, V, dy):
        sc = np.abs(X).max()
        held, broken = 0, 0.0
        for S in ffm.POINT_GROUP:
            C = prob.basis.rep_matrix(S)
            for li in boundary:
                v = S @ lu[li]
                lj = index[tuple(((v + n) % (2 * n)) - n)]
                err = np.abs(X[:, lj] - C @ X[:, li] @ C.T).max() / sc
                if np.all((v >= -n) & (v < n)):
                    assert err <= 1e-13
                    held += 1
                else:
                    broken = max(broken, err)
        assert held == 4 * (2 * n - 2) + 2
        assert broken > 1e-3
