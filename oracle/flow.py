"""Integration of the Lambda-flow, critical scale and classification
(oracle; test infrastructure).

Sec. 3: the exchange propagators obey first-order ODEs in Lambda, solved
with an explicit stepper (the paper names the Odeint library, not the
method or tolerances).  Sec. 4: the flow starts at a large scale with the
bare interaction (P = C = D = 0, so V^B = U e0 e0^T) and stops when the
largest |exchange propagator| exceeds a threshold; the instability is
classified by the channel, transfer momentum and form-factor symmetry of
that largest element.

Readings:
  * integration variable s = ln Lambda (dy/ds = Lambda dy/dLambda),
    integrated from ln Lambda0 downwards;
  * Dormand-Prince 5(4) with the published tableau (Dormand & Prince 1980),
    local extrapolation, error max-norm with atol + rtol max(|y_n|, |y_n+1|),
    step factor 0.9 err^(-1/5) clipped to [0.2, 5] (no growth right after a
    rejection);
  * dense output by the cubic Hermite interpolant of (y_n, f_n, y_n+1,
    f_n+1) (f_n+1 is the FSAL stage), used for checkpoints and for the
    critical scale;
  * Lambda_c: the scale at which max |B_mn(l)| over B in {P, C, D} first
    reaches the threshold, found by bisection on the interpolant;
  * a fixed-step classic RK4 mode is provided for step-by-step comparison.

Pins: order conditions of the tableau, exact solutions of linear ODEs,
exactness of the interpolant on cubics, and the closed-form ladders with
projections switched off (tests/test_oracle_flow.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rhs as rhsmod

DP_C = np.array([0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0, 1.0])
DP_A = [
    [],
    [1 / 5],
    [3 / 40, 9 / 40],
    [44 / 45, -56 / 15, 32 / 9],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
    [35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84],
]
DP_B = np.array([35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84, 0.0])
DP_BSTAR = np.array([5179 / 57600, 0.0, 7571 / 16695, 393 / 640, -92097 / 339200,
                     187 / 2100, 1 / 40])

FAC_SAFETY, FAC_MIN, FAC_MAX = 0.9, 0.2, 5.0


def hermite(s0, y0, f0, s1, y1, f1, s):
    """Cubic Hermite interpolant on [s0, s1] evaluated at s."""
    h = s1 - s0
    th = (s - s0) / h
    h00 = 2 * th ** 3 - 3 * th ** 2 + 1
    h10 = th ** 3 - 2 * th ** 2 + th
    h01 = -2 * th ** 3 + 3 * th ** 2
    h11 = th ** 3 - th ** 2
    return h00 * y0 + h10 * h * f0 + h01 * y1 + h11 * h * f1


@dataclass
class IntegrationResult:
    s: float                      # final s (crossing point if crossed)
    y: np.ndarray                 # state at s
    crossed: bool
    n_rhs: int
    n_accepted: int
    n_rejected: int
    checkpoints: dict = field(default_factory=dict)   # s_c -> y(s_c)
    steps: list = field(default_factory=list)         # accepted (s, h)


def _crossing(s0, y0, f0, s1, y1, f1, thr, iters=100):
    """Bisection for max|y(s)| = thr on the Hermite interpolant, s in [s1, s0]."""
    a, b = s0, s1                  # g(a) <= 0 < g(b)
    for _ in range(iters):
        m = 0.5 * (a + b)
        if np.max(np.abs(hermite(s0, y0, f0, s1, y1, f1, m))) > thr:
            b = m
        else:
            a = m
    return b


def dopri5(f, s0, y0, s_end, h0, rtol, atol, threshold=None, checkpoints=(),
           max_steps=100000):
    """Adaptive Dormand-Prince 5(4) from s0 towards s_end (either direction)."""
    direction = np.sign(s_end - s0)
    h = abs(h0) * direction
    s, y = s0, np.array(y0, dtype=np.float64)
    k1 = f(s, y)
    n_rhs, nacc, nrej = 1, 0, 0
    ck = sorted(checkpoints, reverse=(direction < 0))
    ck_out = {}
    steps = []
    last_rejected = False
    for _ in range(max_steps):
        if (s_end - s) * direction <= 0:
            break
        if (s + h - s_end) * direction > 0:
            h = s_end - s
        k = [k1]
        for i in range(1, 7):
            yi = y + h * sum(DP_A[i][j] * k[j] for j in range(i) if DP_A[i][j] != 0.0)
            k.append(f(s + DP_C[i] * h, yi))
        n_rhs += 6
        y_new = y + h * sum(DP_B[j] * k[j] for j in range(6) if DP_B[j] != 0.0)
        err_vec = h * sum((DP_B[j] - DP_BSTAR[j]) * k[j] for j in range(7)
                          if DP_B[j] != DP_BSTAR[j])
        scale = atol + rtol * np.maximum(np.abs(y), np.abs(y_new))
        err = float(np.max(np.abs(err_vec) / scale))
        if err <= 1.0:
            fac = FAC_MAX if err == 0.0 else min(FAC_MAX, max(FAC_MIN, FAC_SAFETY * err ** -0.2))
            if last_rejected:
                fac = min(fac, 1.0)
            s_new = s + h
            f_new = k[6]
            while ck and (s_new - ck[0]) * direction >= 0 and (ck[0] - s) * direction >= 0:
                sc = ck.pop(0)
                ck_out[sc] = hermite(s, y, k1, s_new, y_new, f_new, sc)
            nacc += 1
            steps.append((s, h))
            if threshold is not None and np.max(np.abs(y_new)) > threshold:
                sc = _crossing(s, y, k1, s_new, y_new, f_new, threshold)
                yc = hermite(s, y, k1, s_new, y_new, f_new, sc)
                return IntegrationResult(sc, yc, True, n_rhs, nacc, nrej, ck_out, steps)
            s, y, k1 = s_new, y_new, f_new
            h = h * fac
            last_rejected = False
        else:
            nrej += 1
            h = h * max(FAC_MIN, FAC_SAFETY * err ** -0.2)
            last_rejected = True
    return IntegrationResult(s, y, False, n_rhs, nacc, nrej, ck_out, steps)


def rk4(f, s0, y0, h, n_steps):
    """Classic fixed-step RK4: n_steps steps of size h."""
    s, y = s0, np.array(y0, dtype=np.float64)
    for _ in range(n_steps):
        k1 = f(s, y)
        k2 = f(s + h / 2, y + h / 2 * k1)
        k3 = f(s + h / 2, y + h / 2 * k2)
        k4 = f(s + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        s = s + h
    return s, y


def log_rhs(prob):
    """dy/ds with s = ln Lambda."""
    def f(s, y):
        lam = np.exp(s)
        return lam * rhsmod.rhs(prob, lam, y)
    return f


@dataclass
class FlowResult:
    lambda_c: float
    diverged: bool
    y: np.ndarray
    n_rhs: int
    n_accepted: int
    n_rejected: int
    checkpoints: dict            # Lambda -> y
    classification: dict | None


def classify(prob, y):
    """Channel, transfer momentum and form-factor symmetry of max |B| (Sec. 4)."""
    a = np.abs(y)
    ch, l, m, n = np.unravel_index(int(np.argmax(a)), a.shape)
    kind = {0: "pairing", 1: "magnetic", 2: "charge"}[int(ch)]
    return dict(channel=int(ch), kind=kind, l_index=int(l),
                l=tuple(prob.l_values[l]), m=int(m), n=int(n),
                symmetry=(prob.basis.symmetry(m), prob.basis.symmetry(n)),
                value=float(y[ch, l, m, n]))


def flow(prob, lambda0, lambda_min, threshold, rtol=1e-8, atol=1e-10, h0=-0.05,
         y0=None, checkpoints=(), max_steps=100000):
    """Flow from lambda0 down to lambda_min or to the critical scale."""
    if y0 is None:
        y0 = np.zeros((3, prob.nl, prob.nff, prob.nff))
    logs = {float(np.log(c)): float(c) for c in checkpoints}
    res = dopri5(log_rhs(prob), np.log(lambda0), y0, np.log(lambda_min), h0, rtol,
                 atol, threshold, list(logs), max_steps)
    cks = {logs[k]: v for k, v in res.checkpoints.items()}
    cls = classify(prob, res.y) if res.crossed else None
    return FlowResult(float(np.exp(res.s)), res.crossed, res.y, res.n_rhs,
                      res.n_accepted, res.n_rejected, cks, cls)
