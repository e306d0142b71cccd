"""Pins of the oracle's flow integration (Sec. 3/4) and of the products
(Eqs. matmul-P/C/D) through closed-form ladders.

* Butcher order conditions of the Dormand-Prince tableau (order 5 for the
  propagating weights, 4 for the embedded ones): any mistyped coefficient
  fails them;
* exact solutions of linear ODEs, threshold crossing, checkpoints;
* exactness of the cubic Hermite interpolant on cubics;
* projections switched off: every channel is a ladder with closed form
  V^P = (V0^-1 + Dchi^pp)^-1, V^C = (V0^-1 + Dchi^ph)^-1,
  2 V^D - V^C = (V0^-1 - Dchi^ph)^-1, Dchi = chi(L) - chi(L0) from the
  non-derivative loop; for V0 = U e0 e0^T only the 00 element flows.
"""
import numpy as np
import pytest

from oracle import flow as fl
from oracle import loops
from tests.conftest import make_problem


def _tableau():
    A = np.zeros((7, 7))
    for i, row in enumerate(fl.DP_A):
        A[i, :len(row)] = row
    return A, fl.DP_C


def _conditions(b, A, c, order):
    e = np.ones_like(c)
    Ac = A @ c
    conds = [(b @ e, 1), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ Ac, 1 / 6),
             (b @ c ** 3, 1 / 4), (b @ (c * Ac), 1 / 8), (b @ (A @ c ** 2), 1 / 12),
             (b @ (A @ Ac), 1 / 24),
             (b @ c ** 4, 1 / 5), (b @ (c ** 2 * Ac), 1 / 10), (b @ (c * (A @ c ** 2)), 1 / 15),
             (b @ (c * (A @ Ac)), 1 / 30), (b @ Ac ** 2, 1 / 20), (b @ (A @ c ** 3), 1 / 20),
             (b @ (A @ (c * Ac)), 1 / 40), (b @ (A @ (A @ c ** 2)), 1 / 60),
             (b @ (A @ (A @ Ac)), 1 / 120)]
    n = {1: 1, 2: 2, 3: 4, 4: 8, 5: 17}[order]
    return conds[:n]


def test_tableau_order_conditions():
    A, c = _tableau()
    assert np.allclose(A.sum(1), c, atol=1e-15)
    for got, want in _conditions(fl.DP_B, A, c, 5):
        assert abs(got - want) < 1e-14
    for got, want in _conditions(fl.DP_BSTAR, A, c, 4):
        assert abs(got - want) < 1e-14
    # the embedded solution is genuinely of lower order
    assert max(abs(g - w) for g, w in _conditions(fl.DP_BSTAR, A, c, 5)) > 1e-6
    # first-same-as-last: last stage row equals the propagating weights
    assert np.allclose(A[6, :6], fl.DP_B[:6])


def test_dopri5_linear_ode_and_checkpoints():
    rates = np.array([0.5, -1.0, 2.0, 0.0])
    f = lambda s, y: rates * y
    y0 = np.array([1.0, 2.0, -1.0, 3.0])
    res = fl.dopri5(f, 0.0, y0, -2.0, 0.1, 1e-10, 1e-12, checkpoints=[-0.5, -1.3])
    assert not res.crossed and np.isclose(res.s, -2.0)
    assert np.allclose(res.y, y0 * np.exp(rates * -2.0), rtol=1e-8)
    for sc, yc in res.checkpoints.items():
        assert np.allclose(yc, y0 * np.exp(rates * sc), rtol=1e-7)
    assert len(res.checkpoints) == 2


def test_threshold_crossing():
    f = lambda s, y: -y          # y = y0 exp(-s) grows as s decreases
    res = fl.dopri5(f, 0.0, np.array([1.0, 0.5]), -10.0, 0.05, 1e-10, 1e-12, threshold=40.0)
    assert res.crossed
    assert abs(res.s - (-np.log(40.0))) < 1e-7
    assert np.isclose(np.max(np.abs(res.y)), 40.0, rtol=1e-7)


def test_hermite_exact_on_cubics():
    p = np.poly1d([0.7, -1.2, 0.3, 2.0])
    dp = p.deriv()
    s0, s1 = 0.3, -0.4
    for s in np.linspace(s1, s0, 7):
        assert np.isclose(fl.hermite(s0, p(s0), dp(s0), s1, p(s1), dp(s1), s), p(s), atol=1e-14)


def test_rk4_fourth_order():
    f = lambda s, y: np.cos(s) * y
    exact = np.exp(np.sin(1.0))
    errs = [abs(fl.rk4(f, 0.0, np.array([1.0]), 1.0 / n, n)[1][0] - exact) for n in (10, 20)]
    assert 14 < errs[0] / errs[1] < 18


def _ladder_flow(prob, lam0, lam1):
    res = fl.flow(prob, lam0, lam1, threshold=1e9, rtol=1e-11, atol=1e-13, h0=-0.02)
    assert not res.diverged
    return res.y


@pytest.mark.parametrize("tp", [-0.1, -0.3])
def test_onsite_ladder_closed_form(tp):
    prob = make_problem(shells=1, nc=4, nf=16, tp=tp, U=2.0, feedback=False)
    lam0, lam1 = 10.0, 0.3
    y = _ladder_flow(prob, lam0, lam1)
    c1, c0 = np.stack(loops.chi(prob, lam1)), np.stack(loops.chi(prob, lam0))
    dpp, dph = (c1 - c0)[0][:, 0, 0], (c1 - c0)[1][:, 0, 0]
    U = prob.U
    assert np.allclose(U - y[0, :, 0, 0], U / (1 + U * dpp), rtol=1e-8)
    assert np.allclose(U + y[1, :, 0, 0], U / (1 + U * dph), rtol=1e-8)
    assert np.allclose(U + y[2, :, 0, 0], U / (1 - U ** 2 * dph ** 2), rtol=1e-8)
    rest = y.copy()
    rest[:, :, 0, 0] = 0.0
    assert np.abs(rest).max() == 0.0


def test_matrix_ladder_closed_form():
    rng = np.random.default_rng(9)
    nff = 5
    a = rng.standard_normal((nff, nff))
    V0 = 0.4 * (a @ a.T / nff + np.eye(nff))    # symmetric positive definite bare matrix
    prob = make_problem(shells=1, nc=4, nf=16, tp=-0.2, feedback=False, bare=V0)
    lam0, lam1 = 8.0, 0.8
    y = _ladder_flow(prob, lam0, lam1)
    c1, c0 = np.stack(loops.chi(prob, lam1)), np.stack(loops.chi(prob, lam0))
    dpp, dph = c1[0] - c0[0], c1[1] - c0[1]
    inv0 = np.linalg.inv(V0)
    VP = np.linalg.inv(inv0[None] + dpp)
    VC = np.linalg.inv(inv0[None] + dph)
    K = np.linalg.inv(inv0[None] - dph)
    assert np.allclose(V0 - y[0], VP, atol=1e-8)
    assert np.allclose(V0 + y[1], VC, atol=1e-8)
    assert np.allclose(V0 + y[2], 0.5 * (K + VC), atol=1e-8)


def test_ladder_critical_scale():
    prob = make_problem(shells=1, nc=4, nf=32, tp=-0.25, U=3.0, feedback=False)
    lam0, thr = 10.0, 20.0
    res = fl.flow(prob, lam0, 1e-3, thr, rtol=1e-10, atol=1e-12)
    assert res.diverged
    c0 = np.stack(loops.chi(prob, lam0))[:, :, 0, 0]
    U = prob.U

    def excess(lam):
        d = np.stack(loops.chi(prob, lam))[:, :, 0, 0] - c0
        b = np.concatenate([U - U / (1 + U * d[0]), U / (1 + U * d[1]) - U,
                            U / (1 - U ** 2 * d[1] ** 2) - U])
        return np.max(np.abs(b)) - thr

    lo, hi = res.lambda_c * 0.9, res.lambda_c * 1.1     # excess(lo) > 0 > excess(hi)
    assert excess(lo) > 0 > excess(hi)
    for _ in range(60):
        mid = np.sqrt(lo * hi)
        if excess(mid) > 0:
            lo = mid
        else:
            hi = mid
    assert abs(res.lambda_c / mid - 1) < 1e-6
    assert res.classification["kind"] == "magnetic" and res.classification["m"] == 0
