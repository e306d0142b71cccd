"""Inter-channel projections V^P, V^C, V^D (oracle; test infrastructure).

Eqs. (proj_VP/VC/VD), Sec. 2.4:
    V^P = P[V0] - P        + P[Phi^C] + P[Phi^D]
    V^C = C[V0] - C[Phi^SC] + C        + C[Phi^D]
    V^D = D[V0] - D[Phi^SC] + D[Phi^C] + D
with the projection rules of Eqs. (proj-P/C/D), Sec. 2.3,
    P[F]_mn(l) = int dk dk' f_m(k) f_n(k') F(l/2 + k, l/2 - k, l/2 - k')
    C[F]_mn(l) = int dk dk' f_m(k) f_n(k') F(k + l/2, k' - l/2, k - l/2)
    D[F]_mn(l) = int dk dk' f_m(k) f_n(k') F(k + l/2, k' - l/2, k' + l/2)
and single-channel couplings rebuilt from exchange propagators by
Eqs. (app-PhiP/C/D) in the decomposition of Eq. (simple-deco):
    Phi^SC: l = k1 + k2,  args ((k1 - k2)/2, (k4 - k3)/2)
    Phi^C:  l = k1 - k3,  args ((k1 + k3)/2, (k2 + k4)/2)
    Phi^D:  l = k3 - k2,  args ((k1 + k4)/2, (k2 + k3)/2),   k4 = k1 + k2 - k3.

Readings (the half-momentum convention is not periodic in the zone and the
position-space form Eq. (proj_pos) evaluates form factors at half lattice
vectors):
  * each channel's bosonic momentum is folded into the half-open zone
    [-pi, pi)^2 and the fermionic arguments are formed from it:
        Phi^SC: l = fold(k1 + k2), args (k1 - l/2, l/2 - k3)
        Phi^C:  l = fold(k1 - k3), args (k3 + l/2, k2 + l/2)
        Phi^D:  l = fold(k3 - k2), args (k1 - l/2, k2 + l/2)
    which equal the paper's expressions when no fold occurs and make
    B[Phi^B] = B exact;
  * the k and k' integrals are averages over the coarse l grid itself, so
    that every folded bosonic momentum lands on the grid;
  * V0 is the on-site U: its projection onto every channel is U e0 e0^T.

``project_bruteforce`` evaluates these definitions literally (cost
Nl^3 Nff^2, tiny grids only).  ``project`` uses the position-space form: with
f_m(k) = sum_R c_m(R) exp(i k.R) the k sum becomes a Kronecker delta on bond
vectors and the source propagator enters through its Fourier series at the
(half-integer) position X, as in Eq. (proj_pos); it is checked term by term
against the literal definition (tests/test_oracle_projections.py).

Pins: own-channel identity B[Phi^B] = B, bare projection U e0 e0^T, the
A-tensor pair relations A^{P,C} = pi_n A^{P,D}, A^{C,P} = pi_n' A^{D,P},
A^{D,C} = A^{C,D} (App. C), vanishing past the bond-length bound (App. B),
C4v covariance.
"""
from __future__ import annotations

import numpy as np

from .model import fold_units

CHANNELS = ("P", "C", "D")


# --- literal definition ---------------------------------------------------

def _proj_args(target, lh, k, kp):
    """(k1, k2, k3) of Eqs. (proj-P/C/D); all momenta in integer units."""
    if target == "P":
        return lh + k, lh - k, lh - kp
    if target == "C":
        return k + lh, kp - lh, k - lh
    if target == "D":
        return k + lh, kp - lh, kp + lh
    raise ValueError(target)


def _param(source, k1, k2, k3, nc):
    """Folded bosonic momentum and fermionic args of Phi^source(k1, k2, k3)."""
    if source == "P":
        lb = fold_units(k1 + k2, nc)
        return lb, k1 - lb // 2, lb // 2 - k3
    if source == "C":
        lb = fold_units(k1 - k3, nc)
        return lb, k3 + lb // 2, k2 + lb // 2
    if source == "D":
        lb = fold_units(k3 - k2, nc)
        return lb, k1 - lb // 2, k2 + lb // 2
    raise ValueError(source)


def _l_index(prob, lu):
    ix = (lu[..., 0] + prob.ncx) // 2
    iy = (lu[..., 1] + prob.ncy) // 2
    return ix * prob.ncy + iy


def _rad(prob, u):
    return u[..., 0] * np.pi / prob.ncx, u[..., 1] * np.pi / prob.ncy


def project_pair_bruteforce(prob, target, source, B):
    """target[Phi^source] for exchange propagator B [Nl][Nff][Nff] (literal)."""
    nc = np.array([prob.ncx, prob.ncy])
    ku = prob.l_units
    nl = prob.nl
    K, KP = np.meshgrid(np.arange(nl), np.arange(nl), indexing="ij")
    k, kp = ku[K.ravel()], ku[KP.ravel()]
    fk = prob.basis.values(*_rad(prob, k))
    fkp = prob.basis.values(*_rad(prob, kp))
    out = np.empty((nl, prob.nff, prob.nff))
    for li in range(nl):
        lh = ku[li] // 2
        k1, k2, k3 = _proj_args(target, lh, k, kp)
        lb, q, qp = _param(source, k1, k2, k3, nc)
        assert np.all(lb % 2 == 0), "bosonic momentum off the coarse grid"
        fq = prob.basis.values(*_rad(prob, q))
        fqp = prob.basis.values(*_rad(prob, qp))
        phi = np.einsum("ap,pab,bp->p", fq, B[_l_index(prob, lb)], fqp)
        out[li] = (fk * phi) @ fkp.T / nl ** 2
    return out


def project_bruteforce(prob, y):
    """(V^P, V^C, V^D) = (P[V], C[V], D[V]) of the full interaction
    V = V0 - Phi^SC + Phi^C + Phi^D, all by the literal definition."""
    sign = {"P": -1.0, "C": 1.0, "D": 1.0}
    out = []
    for target in CHANNELS:
        v = np.broadcast_to(prob.bare_matrix(), (prob.nl, prob.nff, prob.nff)).copy()
        for ci, source in enumerate(CHANNELS):
            v += sign[source] * project_pair_bruteforce(prob, target, source, y[ci])
        out.append(v)
    return np.stack(out)


# --- position-space form ----------------------------------------------------
#
# For target channel T and source S the integrand f_m(k) f_n(k') f_a(q) f_b(q')
# has, after k' = s (l' - k) (l' the folded source momentum),
#     q  = k + l/2 - l'/2                       (all six cross pairs)
#     q' = sq k + bq l/2 + gq l'/2
# Expanding f_m, f_n, f_a, f_b in plane waves with bonds R1, R2, R3, R4:
#     k  coefficient: R1 - s R2 + R3 + sq R4       (sum over k: Kronecker delta
#                                                   modulo the coarse grid)
#     l' coefficient: X = s R2 + (-R3 + gq R4)/2  (Fourier series of S at X)
#     l  coefficient: Y = (R3 + bq R4)/2          (phase)
# Signatures (s, sq, bq, gq), derived from the rules above:
SIGNATURES = {
    ("P", "C"): (+1, -1, +1, +1),
    ("P", "D"): (-1, -1, +1, +1),
    ("C", "P"): (+1, -1, +1, +1),
    ("C", "D"): (-1, +1, -1, -1),
    ("D", "P"): (+1, +1, -1, -1),
    ("D", "C"): (-1, +1, -1, -1),
}


_TERMS_CACHE = {}


def _terms(prob, sig):
    """All bond tuples (b1, b2, b3, b4) with a nonzero k sum, with X and Y."""
    key = (prob.basis.bonds.tobytes(), prob.ncx, prob.ncy, sig)
    if key not in _TERMS_CACHE:
        _TERMS_CACHE[key] = _terms_uncached(prob, sig)
    return _TERMS_CACHE[key]


def _terms_uncached(prob, sig):
    s, sq, bq, gq = sig
    R = prob.basis.bonds
    nb = len(R)
    nc = np.array([prob.ncx, prob.ncy])
    b2, b3, b4 = np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij")
    b2, b3, b4 = b2.ravel(), b3.ravel(), b4.ravel()
    base = -s * R[b2] + R[b3] + sq * R[b4]          # R1 + base == 0 (mod nc)
    rows = []
    for b1 in range(nb):
        ok = np.all((R[b1][None, :] + base) % nc == 0, axis=1)
        idx = np.nonzero(ok)[0]
        rows.append(np.stack([np.full(len(idx), b1), b2[idx], b3[idx], b4[idx]], 1))
    t = np.concatenate(rows, 0)
    X = s * R[t[:, 1]] + 0.5 * (-R[t[:, 2]] + gq * R[t[:, 3]])
    Y = 0.5 * (R[t[:, 2]] + bq * R[t[:, 3]])
    return t, X, Y


def project_pair(prob, target, source, B, chunk=4096):
    """target[Phi^source] by the position-space form (see above)."""
    c = prob.basis.coefficients()                         # [Nff][Nb]
    nb = c.shape[1]
    Bt = np.einsum("ai,bj,lab->lij", c, c, B)             # bond-space B [Nl][Nb][Nb]
    t, X, Y = _terms(prob, SIGNATURES[(target, source)])
    lv = prob.l_values                                    # [Nl][2], in [-pi, pi)
    T = np.zeros((prob.nl, nb * nb), dtype=np.complex128)
    for c0 in range(0, len(t), chunk):
        tt, XX, YY = t[c0:c0 + chunk], X[c0:c0 + chunk], Y[c0:c0 + chunk]
        ph_x = np.exp(1j * (lv @ XX.T))                   # [Nl(l'), n]
        F = np.einsum("ln,ln->n", ph_x, Bt[:, tt[:, 2], tt[:, 3]])
        ph_y = np.exp(1j * (lv @ YY.T))                   # [Nl(l), n]
        contrib = ph_y * F[None, :] / prob.nl
        np.add.at(T.T, tt[:, 0] * nb + tt[:, 1], contrib.T)
    T = T.reshape(prob.nl, nb, nb)
    out = np.einsum("mi,nj,lij->lmn", c, c, T)
    return out.real


def project(prob, y):
    """(V^P, V^C, V^D) of Eqs. (proj_VP/VC/VD).  y = (P, C, D) [3][Nl][Nff][Nff]."""
    P, C, D = y
    bare = prob.bare_matrix()[None]
    if not prob.feedback:
        return np.stack([bare - P, bare + C, bare + D])
    VP = bare - P + project_pair(prob, "P", "C", C) + project_pair(prob, "P", "D", D)
    VC = bare - project_pair(prob, "C", "P", P) + C + project_pair(prob, "C", "D", D)
    VD = bare - project_pair(prob, "D", "P", P) + project_pair(prob, "D", "C", C) + D
    return np.stack([VP, VC, VD])
