"""Pins of the oracle's loops (Eq. chis) against independent mathematics.

* numerical frequency quadrature of Re[G G] and of d/dOmega Re[G G] with the
  Omega-cutoff propagator (the closed forms in oracle.loops are derived, not
  printed in the paper);
* a full brute-force loop on a tiny grid, frequency integrals by quadrature;
* Omega -> 0 limits (BCS, Lindhard) and the Omega -> infinity sum rule;
* int chi_dot dOmega = Delta chi (checks J = dK/dOmega at the loop level);
* App. C: symmetry, parity selection and C4v covariance of chi.
"""
import numpy as np
import pytest
from scipy.integrate import quad, quad_vec

from oracle import formfactors as ffm
from oracle import loops
from tests.conftest import make_problem


def _gg(p0, a, b, om, channel, derivative):
    th = p0 * p0 / (p0 * p0 + om * om)
    dth = -2 * om * p0 * p0 / (p0 * p0 + om * om) ** 2
    num = 2 * th * dth if derivative else th * th
    second = -1j * p0 - b if channel == "pp" else 1j * p0 - b
    return (num / ((1j * p0 - a) * second)).real / (2 * np.pi)


def _quad_weight(a, b, om, channel, derivative):
    pts = sorted({abs(a), abs(b), om})
    f = lambda p0: 2 * _gg(p0, a, b, om, channel, derivative)   # even in p0
    val = 0.0
    edges = [0.0] + pts
    for lo, hi in zip(edges[:-1], edges[1:]):
        if hi <= lo:
            continue
        val += quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    val += quad(f, edges[-1], np.inf, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
    return val


CASES = [(0.3, 0.7, 0.5), (-0.3, 0.7, 0.5), (0.3, -1.2, 2.0), (-0.4, -0.1, 0.05),
         (0.2, 0.2, 0.3), (0.2, -0.2, 0.3), (0.0, 0.5, 0.7), (0.0, 0.0, 0.4),
         (1e-3, -2e-3, 0.01), (3.0, 2.9, 0.02)]


@pytest.mark.parametrize("a,b,om", CASES)
@pytest.mark.parametrize("derivative", [False, True])
def test_weights_match_frequency_quadrature(a, b, om, derivative):
    wpp, wph = loops.weights(np.array(a), np.array(b), om, derivative)
    qpp = _quad_weight(a, b, om, "pp", derivative)
    qph = _quad_weight(a, b, om, "ph", derivative)
    scale = max(abs(qpp), abs(qph), 1e-300)
    assert abs(wpp - qpp) <= 1e-10 * scale
    assert abs(wph - qph) <= 1e-10 * scale


def test_weights_match_naive_quotients_away_from_singular_points():
    rng = np.random.default_rng(3)
    a, b = rng.uniform(-3, 3, (2, 2000))
    keep = (np.abs(a + b) > 0.05) & (np.abs(a - b) > 0.05)
    a, b = a[keep], b[keep]
    for om in (0.01, 0.3, 5.0):
        for d in (False, True):
            s = loops.weights(a, b, om, d)
            n = loops.weights_naive(a, b, om, d)
            for x, y in zip(s, n):
                assert np.allclose(x, y, rtol=1e-11, atol=0)


def test_zero_scale_limits_bcs_and_lindhard():
    om = 1e-10
    a = np.array([0.3, -0.5, 0.3, 0.4])
    b = np.array([0.3, -0.5, -0.7, 0.9])
    pp, ph = loops.weights(a, b, om, derivative=False)
    # BCS: 1/(|a|+|b|) for equal signs, 0 otherwise; Lindhard: -1/|b-a| across, 0 same side
    assert np.allclose(pp, [1 / 0.6, 1 / 1.0, 0.0, 1 / 1.3], rtol=1e-8, atol=1e-8)
    assert np.allclose(ph, [0.0, 0.0, -1 / 1.0, 0.0], rtol=1e-8, atol=1e-8)


def test_large_scale_sum_rule():
    prob = make_problem(shells=2, nc=4, nf=16, tp=-0.3)
    om = 1e6
    pp, ph = loops.chi_dot(prob, om)
    eye = np.eye(prob.nff)[None]
    assert np.allclose(om ** 2 * pp, -eye / 4, atol=2e-5)
    assert np.allclose(om ** 2 * ph, eye / 4, atol=2e-5)


def _tiny_problem():
    import workloads as W
    from oracle.model import Problem
    return Problem(1.0, -0.25, -1.0, 3.0, W.bonds_for_shells(1), 4, 4, 8, 8)


def test_full_loop_against_quadrature_on_tiny_grid():
    prob = _tiny_problem()
    om = 0.37
    p = prob.p_values
    f = prob.basis.values(p[:, 0], p[:, 1])
    pp, ph = loops.chi_dot(prob, om)
    cache = {}
    for li, (lx, ly) in enumerate(prob.l_values):
        xa = prob.xi(p[:, 0] + lx / 2, p[:, 1] + ly / 2)
        xb = prob.xi(p[:, 0] - lx / 2, p[:, 1] - ly / 2)
        wq = {"pp": np.empty(len(p)), "ph": np.empty(len(p))}
        for i in range(len(p)):
            key = (round(xa[i], 13), round(xb[i], 13))
            if key not in cache:
                cache[key] = (_quad_weight(xa[i], xb[i], om, "pp", True),
                              _quad_weight(xa[i], xb[i], om, "ph", True))
            wq["pp"][i], wq["ph"][i] = cache[key]
        for ch, mine in (("pp", pp), ("ph", ph)):
            ref = (f * wq[ch]) @ f.T / prob.nf
            assert np.abs(mine[li] - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-12)


def test_integrated_derivative_equals_loop_difference():
    prob = make_problem(shells=1, nc=4, nf=16)
    sel = [0, 5, 10]
    lo, hi = 0.2, 1.5
    dpp, dph = quad_vec(lambda lam: np.stack(loops.chi_dot(prob, lam, sel)), lo, hi,
                        epsabs=1e-13, epsrel=1e-12)[0]
    c_hi, c_lo = np.stack(loops.chi(prob, hi, sel)), np.stack(loops.chi(prob, lo, sel))
    assert np.allclose(dpp, c_hi[0] - c_lo[0], atol=1e-10)
    assert np.allclose(dph, c_hi[1] - c_lo[1], atol=1e-10)


def test_symmetry_and_parity_selection():
    prob = make_problem(shells=3, nc=6, nf=24, tp=-0.35)
    par = prob.basis.parity
    odd = (par[:, None] * par[None, :]) < 0
    for om in (0.05, 1.0):
        for chi in loops.chi_dot(prob, om):
            scale = np.abs(chi).max()
            assert np.allclose(chi, np.swapaxes(chi, 1, 2), atol=1e-15 * scale)
            assert np.abs(chi[:, odd]).max() <= 1e-14 * scale


def test_point_group_covariance_interior_l():
    prob = make_problem(shells=4, nc=8, nf=32, tp=-0.3)
    pp, ph = loops.chi_dot(prob, 0.2)
    lu = prob.l_units
    interior = np.all(np.abs(lu) < prob.ncx, axis=1)
    index = {tuple(u): i for i, u in enumerate(lu)}
    for S in ffm.POINT_GROUP:
        C = prob.basis.rep_matrix(S)
        for li in np.nonzero(interior)[0]:
            lj = index[tuple(S @ lu[li])]
            for chi in (pp, ph):
                assert np.allclose(chi[lj], C @ chi[li] @ C.T, atol=1e-13 * np.abs(chi).max())


def test_point_group_covariance_boundary_l():
    """App. C covariance on the zone boundary: chi(g l) = C chi(l) C^T holds
    for the elements g that map l into [-pi, pi)^2 without a fold (those
    that keep a -pi component at -pi), and fails for the others (the fold
    of +pi to -pi moves the half momentum l/2 by pi)."""
    prob = make_problem(shells=3, nc=6, nf=24, tp=-0.3)
    pp, ph = loops.chi_dot(prob, 0.3)
    lu = prob.l_units
    n = prob.ncx
    index = {tuple(u): i for i, u in enumerate(lu)}
    boundary = np.nonzero(np.any(lu == -n, axis=1))[0]
    held, broken = 0, 0
    for S in ffm.POINT_GROUP:
        C = prob.basis.rep_matrix(S)
        for li in boundary:
            v = S @ lu[li]
            lj = index[tuple(((v + n) % (2 * n)) - n)]
            err = max(np.abs(chi[lj] - C @ chi[li] @ C.T).max() / np.abs(chi).max()
                      for chi in (pp, ph))
            if np.all((v >= -n) & (v < n)):
                assert err <= 1e-13
                held += 1
            else:
                broken += err > 1e-3
    # (-pi, q): 4 elements each; (-pi, -pi): 2 (e and the diagonal mirror)
    assert held == 4 * (2 * n - 2) + 2
    assert broken > 0
