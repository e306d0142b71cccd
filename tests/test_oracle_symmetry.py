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
