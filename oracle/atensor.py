"""Precomputed projection tensors A^{B,B'} (oracle; test infrastructure).

App. C writes every cross projection as a linear map of the source channel's
exchange propagator,

    B[Phi^B']_mn(l) = sum_{q, m', n'} A^{B,B'}_{m,n,m',n'}(q, l) B'_{m'n'}(q),

with A independent of the scale (Sec. 2.5: the scale-independent parts of
the projections computed once and stored).  Here A is that map for the
oracle's projection (``projections.project_pair``, itself pinned against the
literal double sum): the column (q, m', n') is the projection of the unit
propagator at q, (m', n').  Layout: A[l][m][n][q][m'][n'].

Of the six cross pairs three are stored, (P, C), (C, P) and (D, C); the
others follow from the pair relations of App. C,

    A^{P,D} = pi_n A^{P,C},   A^{D,P} = pi_n' A^{C,P},   A^{C,D} = A^{D,C},

and the couplings are assembled as in Eqs. (proj_VP/VC/VD):

    V^P = U e0 e0^T - P + A^{P,C} C + A^{P,D} D
    V^C = U e0 e0^T - A^{C,P} P + C + A^{C,D} D
    V^D = U e0 e0^T - A^{D,P} P + A^{D,C} C + D.

Pins (tests/test_oracle_atensor.py): the pair relations between tensors
built independently for all six pairs, the assembly against
``projections.project`` on random states, the point-group covariance of App.
C for transfer momenta inside the zone, and the index symmetries of App. C.
"""
from __future__ import annotations

import numpy as np

from .projections import project_pair

STORED = (("P", "C"), ("C", "P"), ("D", "C"))


def a_tensor(prob, target, source):
    """A^{target,source}[l][m][n][q][m'][n'] column by column: the projection of
    each unit propagator (the projection is linear in the propagator)."""
    nl, nff = prob.nl, prob.nff
    A = np.empty((nl, nff, nff, nl, nff, nff))
    e = np.zeros((nl, nff, nff))
    for q in range(nl):
        for a in range(nff):
            for b in range(nff):
                e[q, a, b] = 1.0
                A[:, :, :, q, a, b] = project_pair(prob, target, source, e)
                e[q, a, b] = 0.0
    return A


def stored_tensors(prob):
    """The three stored pairs {(target, source): A}."""
    return {pair: a_tensor(prob, *pair) for pair in STORED}


def pair_tensor(prob, A3, target, source):
    """Any of the six cross pairs from the three stored ones (App. C)."""
    if (target, source) in A3:
        return A3[(target, source)]
    par = prob.basis.parity
    if (target, source) == ("P", "D"):      # A^{P,D} = pi_n A^{P,C}
        return par[None, None, :, None, None, None] * A3[("P", "C")]
    if (target, source) == ("D", "P"):      # A^{D,P} = pi_n' A^{C,P}
        return par[None, None, None, None, None, :] * A3[("C", "P")]
    if (target, source) == ("C", "D"):      # A^{C,D} = A^{D,C}
        return A3[("D", "C")]
    raise ValueError((target, source))


def apply(A, B):
    """sum_{q, m', n'} A[l][m][n][q][m'][n'] B[q][m'][n']."""
    return np.einsum("lmnqab,qab->lmn", A, B)


def project_with_tensors(prob, y, A3):
    """(V^P, V^C, V^D) from the stored tensors (Eqs. proj_VP/VC/VD)."""
    P, C, D = y
    bare = prob.bare_matrix()[None]
    if not prob.feedback:
        return np.stack([bare - P, bare + C, bare + D])

    def A(t, s):
        return pair_tensor(prob, A3, t, s)

    VP = bare - P + apply(A("P", "C"), C) + apply(A("P", "D"), D)
    VC = bare - apply(A("C", "P"), P) + C + apply(A("C", "D"), D)
    VD = bare - apply(A("D", "P"), P) + apply(A("D", "C"), C) + D
    return np.stack([VP, VC, VD])
