"""Form-factor projected loops (oracle; test infrastructure).

Eq. (chis), Sec. 2.4:
    chi^pp_mn(l) = int dp G(l/2 + p) G(l/2 - p) f_m(p) f_n(p)
    chi^ph_mn(l) = int dp G(p + l/2) G(p - l/2) f_m(p) f_n(p)
at bosonic frequency l0 = 0 (frequency dependence neglected, Sec. 3).
The dot is the derivative with respect to the scale Lambda = Omega.

Readings (the paper cites the Omega-cutoff of Husemann & Salmhofer without
printing it, Sec. 3):
  * regulator G_Omega(k0, k) = k0^2/(k0^2 + Omega^2) * 1/(i k0 - xi_k), T = 0;
  * int dp = int dp0/(2 pi) (1/Nf) sum_p over a uniform fine grid.

The frequency integral is done in closed form.  With
    K(xi, Omega) = int dp0/2pi Theta(p0)^2 xi/(p0^2 + xi^2)
                 = sgn(xi) |xi| (Omega + 2|xi|) / (4 (Omega + |xi|)^2),
    J(xi, Omega) = dK/dOmega = -xi (Omega + 3|xi|) / (4 (Omega + |xi|)^3),
partial fractions in p0 give, for xi_a = xi(a), xi_b = xi(b):
    pp weight = (K(a) + K(b)) / (xi_a + xi_b)
    ph weight = (K(a) - K(b)) / (xi_b - xi_a)
and the same with J for the scale derivatives.  Since xi(l/2 - p) = xi(p - l/2)
both loops use the same pair (xi(p + l/2), xi(p - l/2)).

These quotients are evaluated without cancellation by writing
K = sgn * k/4, J = -sgn * h/4 with
    k(x) = x (W + 2x)/(W + x)^2 = 2 - 3W/u + W^2/u^2,
    h(x) = x (W + 3x)/(W + x)^3 = 3/u - 5W/u^2 + 2W^2/u^3,   u = W + x,
whose divided differences follow from [1/u^n]_{x,y} exactly.

Pins (tests/test_oracle_loops.py): numerical frequency quadrature of
Re[G G] and of its Omega derivative (to 1e-10), Omega -> 0 limits (BCS
1/(2|xi|), Lindhard), the naive quotients away from singular points,
int chi_dot dOmega = Delta chi, symmetry, parity selection and C4v
covariance (App. C).
"""
from __future__ import annotations

import numpy as np


def K_freq(xi, om):
    """Frequency integral K(xi, Omega) (closed form, see module header)."""
    x = np.abs(xi)
    return np.sign(xi) * x * (om + 2 * x) / (4 * (om + x) ** 2)


def J_freq(xi, om):
    """J = dK/dOmega."""
    x = np.abs(xi)
    return -xi * (om + 3 * x) / (4 * (om + x) ** 3)


def _k_fun(x, om):
    return x * (om + 2 * x) / (om + x) ** 2


def _h_fun(x, om):
    return x * (om + 3 * x) / (om + x) ** 3


def _sum_quotient(phi, dphi0, x, y, om):
    """(phi(x) + phi(y)) / (x + y) for x, y >= 0; phi'(0) at x = y = 0."""
    s = x + y
    with np.errstate(invalid="ignore", divide="ignore"):
        q = (phi(x, om) + phi(y, om)) / s
    return np.where(s > 0, q, dphi0)


def _dd_k(x, y, om):
    """Divided difference k[x, y]."""
    u, v = om + x, om + y
    return 3 * om / (u * v) - om ** 2 * (u + v) / (u ** 2 * v ** 2)


def _dd_h(x, y, om):
    """Divided difference h[x, y]."""
    u, v = om + x, om + y
    return (-3 / (u * v) + 5 * om * (u + v) / (u ** 2 * v ** 2)
            - 2 * om ** 2 * (u * u + u * v + v * v) / (u ** 3 * v ** 3))


def weights(xa, xb, om, derivative=True):
    """Loop weights (w_pp, w_ph) for dispersion values xa, xb at scale om.

    derivative=True: weights of chi_dot (J); False: of chi (K).
    """
    x, y = np.abs(xa), np.abs(xb)
    same = (xa * xb) > 0
    if derivative:
        S = _sum_quotient(_h_fun, 1.0 / om ** 2, x, y, om)
        D = _dd_h(x, y, om)
        wpp = np.where(same, -S, -D) / 4
        wph = np.where(same, D, S) / 4
    else:
        S = _sum_quotient(_k_fun, 1.0 / om, x, y, om)
        D = _dd_k(x, y, om)
        wpp = np.where(same, S, D) / 4
        wph = np.where(same, -D, -S) / 4
    return wpp, wph


def weights_naive(xa, xb, om, derivative=True):
    """Plain quotients of K (or J); singular where xa + xb = 0 or xa = xb."""
    g = J_freq if derivative else K_freq
    return (g(xa, om) + g(xb, om)) / (xa + xb), (g(xa, om) - g(xb, om)) / (xb - xa)


def _loop(prob, om, derivative, l_index=None, l_chunk=32):
    """chi (or chi_dot) for all or selected l: two arrays [nl_sel][Nff][Nff]."""
    p = prob.p_values                                   # [Nf, 2]
    f = prob.f_fine                                     # [Nff, Nf]
    ls = np.arange(prob.nl) if l_index is None else np.asarray(l_index)
    # products f_m f_n as one [Nff^2][Nf] matrix when it is small
    ff = None
    if prob.nff ** 2 * prob.nf <= 2 ** 25:
        ff = (f[:, None, :] * f[None, :, :]).reshape(prob.nff ** 2, prob.nf)
    out_pp = np.empty((len(ls), prob.nff, prob.nff))
    out_ph = np.empty_like(out_pp)
    for c0 in range(0, len(ls), l_chunk):
        sel = ls[c0:c0 + l_chunk]
        half = 0.5 * prob.l_values[sel]                 # [L, 2]
        ax = p[:, 0, None] + half[None, :, 0]
        ay = p[:, 1, None] + half[None, :, 1]
        bx = p[:, 0, None] - half[None, :, 0]
        by = p[:, 1, None] - half[None, :, 1]
        wpp, wph = weights(prob.xi(ax, ay), prob.xi(bx, by), om, derivative)
        if ff is not None:
            # (1/Nf) sum_p f_m(p) f_n(p) w(p, l) as one matrix product
            out_pp[c0:c0 + len(sel)] = (ff @ wpp).T.reshape(-1, prob.nff, prob.nff) / prob.nf
            out_ph[c0:c0 + len(sel)] = (ff @ wph).T.reshape(-1, prob.nff, prob.nff) / prob.nf
        else:
            for j in range(len(sel)):
                out_pp[c0 + j] = (f * wpp[:, j]) @ f.T / prob.nf
                out_ph[c0 + j] = (f * wph[:, j]) @ f.T / prob.nf
    return out_pp, out_ph


def chi_dot(prob, om, l_index=None):
    """(chi_dot^pp, chi_dot^ph) of Eq. (chis): arrays [Nl][Nff][Nff]."""
    return _loop(prob, om, True, l_index)


def chi(prob, om, l_index=None):
    """(chi^pp, chi^ph) of Eq. (chis) (non-derivative), for the ladder pin."""
    return _loop(prob, om, False, l_index)
