"""Fermi-surface-refined loop integration (oracle; test infrastructure).

Sec. 3: the paper evaluates each loop integral of Eq. (chis) with an
adaptive cubature (DCUHRE).  The uniform fine grid of ``loops`` is the
midpoint rule on Nf cells; at small scales the integrand of a cell whose
propagators lie near the Fermi surface varies on an energy scale Lambda
smaller than the cell, and the midpoint value is inaccurate there.

Reading (the paper gives no refinement rule): a cell p is refined for
transfer momentum l when Lambda < Lambda_on and one of the two propagators
xi(k + l/2), xi(k - l/2), evaluated at the cell's centre and four corners,
changes sign over the cell (the cell straddles the Fermi surface) or comes
within kappa Lambda of zero; its midpoint value is then replaced by the average over s x s
sub-points p + (2 pi / nf) ((i - (s-1)/2) / s, (j - (s-1)/2) / s),
i, j = 0 .. s-1, s odd:

    chi_dot_mn(l) = (1/Nf) sum_p [refined(p, l) ? (1/s^2) sum_sub g(sub) : g(p)],
    g(k) = f_m(k) f_n(k) w(xi(k + l/2), xi(k - l/2)).

With s odd the sub-points of all cells tile the uniform grid of s nf points
per direction (the centre sub-point is p itself), so refining every cell
gives the uniform rule on the finer grid exactly.  The flag decision uses the
FP64 dispersion at the centres and corners of the fine-grid cells.

Pins (tests/test_oracle_refine.py): every cell refined = the uniform rule on
s nf points (to rounding); no cell refined = the uniform rule on nf; at small
scales the refined loops are much closer to the fine-grid loops than the
unrefined ones; symmetry, parity selection and C4v covariance survive.
"""
from __future__ import annotations

import numpy as np

from .loops import chi_dot, weights


def refine_flags(prob, om, l_index, kappa, lam_on):
    """[len(l_index)][Nf] bool: cells refined for each selected l.  A cell is
    refined when one of its two propagators, over the cell's centre and four
    corners, changes sign (the cell straddles the Fermi surface) or comes
    within kappa Lambda of zero."""
    ls = np.asarray(l_index)
    flags = np.zeros((len(ls), prob.nf), dtype=bool)
    if not (om < lam_on) or kappa <= 0:
        return flags
    p = prob.p_values
    hx, hy = np.pi / prob.nfx, np.pi / prob.nfy           # half a cell
    pts = [(0.0, 0.0), (-hx, -hy), (-hx, hy), (hx, -hy), (hx, hy)]
    for j, li in enumerate(ls):
        half = 0.5 * prob.l_values[li]
        for sgn in (1.0, -1.0):
            x = np.stack([prob.xi(p[:, 0] + dx + sgn * half[0], p[:, 1] + dy + sgn * half[1])
                          for dx, dy in pts])              # [5][Nf]
            near = np.abs(x).min(axis=0) < kappa * om
            cross = (x.min(axis=0) < 0) & (x.max(axis=0) > 0)
            flags[j] |= near | cross
    return flags


def chi_dot_refined(prob, om, s=3, kappa=4.0, lam_on=np.inf, l_index=None):
    """(chi_dot^pp, chi_dot^ph) [len(l)][Nff][Nff] with the refined cells."""
    if s < 1 or s % 2 == 0:
        raise ValueError("s must be odd")
    ls = np.arange(prob.nl) if l_index is None else np.asarray(l_index)
    pp, ph = chi_dot(prob, om, ls)
    flags = refine_flags(prob, om, ls, kappa, lam_on)
    if s == 1 or not flags.any():
        return pp, ph
    hx, hy = 2 * np.pi / prob.nfx, 2 * np.pi / prob.nfy
    off = (np.arange(s) - (s - 1) / 2) / s
    ox, oy = np.meshgrid(off * hx, off * hy, indexing="ij")
    ox, oy = ox.ravel(), oy.ravel()                       # [s^2]
    p = prob.p_values
    fc = prob.f_fine                                      # [Nff][Nf]
    for j, li in enumerate(ls):
        cells = np.nonzero(flags[j])[0]
        if len(cells) == 0:
            continue
        half = 0.5 * prob.l_values[li]
        # midpoint values of the refined cells, to be replaced
        xa = prob.xi(p[cells, 0] + half[0], p[cells, 1] + half[1])
        xb = prob.xi(p[cells, 0] - half[0], p[cells, 1] - half[1])
        wpp, wph = weights(xa, xb, om)
        f = fc[:, cells]
        pp[j] -= (f * wpp) @ f.T / prob.nf
        ph[j] -= (f * wph) @ f.T / prob.nf
        # the sub-point averages
        kx = (p[cells, 0][:, None] + ox[None, :]).ravel()
        ky = (p[cells, 1][:, None] + oy[None, :]).ravel()
        xa = prob.xi(kx + half[0], ky + half[1])
        xb = prob.xi(kx - half[0], ky - half[1])
        wpp, wph = weights(xa, xb, om)
        f = prob.basis.values(kx, ky)
        pp[j] += (f * wpp) @ f.T / (prob.nf * s * s)
        ph[j] += (f * wph) @ f.T / (prob.nf * s * s)
    return pp, ph
