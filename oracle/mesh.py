"""Non-uniform, channel-specific bosonic meshes (oracle; test infrastructure).

Sec. 4 (and the mesh figure): production flows keep each exchange
propagator on its own momentum mesh, refined around the momenta where it is
expected to peak (992 points for P, 6632 for C and D).  Readings (the paper
gives the meshes only as a figure):

  * a mesh is a nested refinement of the coarse grid: the coarse cells whose
    centre lies within a radius of a given centre (periodic distance) are
    split into m x m sub-cells (m odd), each represented by its centre, with
    the cell's area as quadrature weight (weights sum to one).  Points are
    integer pairs j on the lattice l = -pi + 2 pi j / (nc m); a coarse point
    is j = m i, and the centre sub-point of a refined cell is the coarse point;
  * P lives on mesh_P, C and D on mesh_CD; the state holds every channel on
    the union of the two meshes, a channel's entries off its own mesh are
    zero and stay zero (their derivative is set to zero);
  * the Fourier values of a source propagator at the key positions X of the
    position-space projections (Eq. proj_pos) are quadratures over its mesh,
    sum_{l' in mesh_S} w_l' e^{i l'.X} Bt^S(l'), which on the uniform coarse
    grid (w = 1/Nl) are those of projections.project_pair; the phase sums are
    evaluated at every point of the union; the k and k' integrals of the
    projections stay averages over the coarse grid (the coarse grid's term
    lists);
  * the loops are evaluated at every point of the union (l/2 on the fine grid:
    nf a multiple of 2 nc m), the products of a channel at its own mesh.

Pins (tests/test_oracle_mesh.py): the uniform coarse mesh reproduces
projections.project and rhs.rhs; rhs_mesh_at equals rhs_mesh at its points; a mesh refined everywhere reproduces them on
the uniform grid of nc m points (coarse grids that do not alias the bond
sums, so the term lists agree); the quadrature weights sum to one per
channel; entries off a channel's mesh stay zero.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .loops import weights
from .projections import SIGNATURES, _terms
from .rhs import products


@dataclass
class Mesh:
    nc: int              # coarse grid per direction
    m: int               # refinement factor (odd)
    points: np.ndarray   # [N][2] integer lattice coordinates, l = -pi + 2 pi j / (nc m)
    w_p: np.ndarray      # [N] quadrature weights of mesh_P (zero off it)
    w_cd: np.ndarray     # [N] quadrature weights of mesh_CD

    @property
    def n(self) -> int:
        return len(self.points)

    @property
    def l_values(self) -> np.ndarray:
        return -np.pi + 2.0 * np.pi * self.points / (self.nc * self.m)


def _cells(nc, m, centres, radius):
    """{coarse (ix, iy): refined?} for a centre list [(lx, ly)] in radians."""
    g = -np.pi + 2.0 * np.pi * np.arange(nc) / nc
    out = {}
    for ix in range(nc):
        for iy in range(nc):
            ref = False
            for cx, cy in centres:
                dx = (g[ix] - cx + np.pi) % (2 * np.pi) - np.pi
                dy = (g[iy] - cy + np.pi) % (2 * np.pi) - np.pi
                ref = ref or np.hypot(dx, dy) <= radius
            out[(ix, iy)] = ref
    return out


def _cell_points(nc, m, cells):
    """{lattice point: weight} of one channel's mesh."""
    pts = {}
    c = (m - 1) // 2
    for (ix, iy), ref in cells.items():
        if ref:
            for a in range(m):
                for b in range(m):
                    pts[((m * ix + a - c) % (nc * m), (m * iy + b - c) % (nc * m))] = \
                        1.0 / (nc * nc * m * m)
        else:
            pts[(m * ix, m * iy)] = 1.0 / (nc * nc)
    return pts


def refined_mesh(nc, m, centres_p, centres_cd, radius):
    """Union of mesh_P (cells near centres_p refined) and mesh_CD."""
    if m < 1 or m % 2 == 0:
        raise ValueError("m must be odd")
    wp = _cell_points(nc, m, _cells(nc, m, centres_p, radius))
    wc = _cell_points(nc, m, _cells(nc, m, centres_cd, radius))
    keys = sorted(set(wp) | set(wc))
    pts = np.array(keys, dtype=np.int64).reshape(-1, 2)
    return Mesh(nc, m, pts, np.array([wp.get(k, 0.0) for k in keys]),
                np.array([wc.get(k, 0.0) for k in keys]))


def chi_dot_at(prob, om, lv):
    """(chi_dot^pp, chi_dot^ph) [len(lv)][Nff][Nff] at the momenta lv [N][2]
    (Eq. chis on the fine grid, as loops.chi_dot)."""
    p = prob.p_values
    f = prob.f_fine
    out_pp = np.empty((len(lv), prob.nff, prob.nff))
    out_ph = np.empty_like(out_pp)
    for j, l in enumerate(lv):
        h = 0.5 * l
        wpp, wph = weights(prob.xi(p[:, 0] + h[0], p[:, 1] + h[1]),
                           prob.xi(p[:, 0] - h[0], p[:, 1] - h[1]), om)
        out_pp[j] = (f * wpp) @ f.T / prob.nf
        out_ph[j] = (f * wph) @ f.T / prob.nf
    return out_pp, out_ph


def project_pair_mesh(prob, mesh, target, source, B, w):
    """target[Phi^source] at every mesh point, the source's Fourier values a
    quadrature over its mesh (weights w) -- the position-space form of
    projections.project_pair with the coarse grid's term lists."""
    c = prob.basis.coefficients()
    nb = c.shape[1]
    Bt = np.einsum("ai,bj,lab->lij", c, c, B)
    t, X, Y = _terms(prob, SIGNATURES[(target, source)])
    lv = mesh.l_values
    ph_x = np.exp(1j * (lv @ X.T))                       # [N(l')][terms]
    F = np.einsum("l,lt,lt->t", w, ph_x, Bt[:, t[:, 2], t[:, 3]])
    ph_y = np.exp(1j * (lv @ Y.T))                       # [N(l)][terms]
    T = np.zeros((mesh.n, nb * nb), dtype=np.complex128)
    np.add.at(T.T, t[:, 0] * nb + t[:, 1], (ph_y * F[None, :]).T)
    return np.einsum("mi,nj,lij->lmn", c, c, T.reshape(mesh.n, nb, nb)).real


def project_pair_mesh_at(prob, mesh, target, source, B, w, out):
    """project_pair_mesh at the mesh points out only (the source's quadrature
    still runs over its whole mesh)."""
    c = prob.basis.coefficients()
    nb = c.shape[1]
    Bt = np.einsum("ai,bj,lab->lij", c, c, B)
    t, X, Y = _terms(prob, SIGNATURES[(target, source)])
    lv = mesh.l_values
    F = np.einsum("l,lt,lt->t", w, np.exp(1j * (lv @ X.T)), Bt[:, t[:, 2], t[:, 3]])
    ph_y = np.exp(1j * (lv[out] @ Y.T))                  # [len(out)][terms]
    T = np.zeros((len(out), nb * nb), dtype=np.complex128)
    np.add.at(T.T, t[:, 0] * nb + t[:, 1], (ph_y * F[None, :]).T)
    return np.einsum("mi,nj,lij->lmn", c, c, T.reshape(len(out), nb, nb)).real


def rhs_mesh_at(prob, mesh, lam, y, out):
    """rhs_mesh at the mesh points out only: [3][len(out)][Nff][Nff]."""
    out = np.asarray(out)
    P, C, D = y
    bare = prob.bare_matrix()[None]
    wp, wc = mesh.w_p, mesh.w_cd
    if prob.feedback:
        VP = bare - P[out] + project_pair_mesh_at(prob, mesh, "P", "C", C, wc, out) \
            + project_pair_mesh_at(prob, mesh, "P", "D", D, wc, out)
        VC = bare - project_pair_mesh_at(prob, mesh, "C", "P", P, wp, out) + C[out] \
            + project_pair_mesh_at(prob, mesh, "C", "D", D, wc, out)
        VD = bare - project_pair_mesh_at(prob, mesh, "D", "P", P, wp, out) \
            + project_pair_mesh_at(prob, mesh, "D", "C", C, wc, out) + D[out]
    else:
        VP, VC, VD = bare - P[out], bare + C[out], bare + D[out]
    pp, ph = chi_dot_at(prob, lam, mesh.l_values[out])
    dy = products(np.stack([VP, VC, VD]), pp, ph)
    dy[0][mesh.w_p[out] == 0] = 0.0
    dy[1:, mesh.w_cd[out] == 0] = 0.0
    return dy


def project_mesh(prob, mesh, y):
    """(V^P, V^C, V^D) at every mesh point (Eqs. proj_VP/VC/VD)."""
    P, C, D = y
    bare = prob.bare_matrix()[None]
    if not prob.feedback:
        return np.stack([bare - P, bare + C, bare + D])
    wp, wc = mesh.w_p, mesh.w_cd
    VP = bare - P + project_pair_mesh(prob, mesh, "P", "C", C, wc) \
        + project_pair_mesh(prob, mesh, "P", "D", D, wc)
    VC = bare - project_pair_mesh(prob, mesh, "C", "P", P, wp) + C \
        + project_pair_mesh(prob, mesh, "C", "D", D, wc)
    VD = bare - project_pair_mesh(prob, mesh, "D", "P", P, wp) \
        + project_pair_mesh(prob, mesh, "D", "C", C, wc) + D
    return np.stack([VP, VC, VD])


def rhs_mesh(prob, mesh, lam, y):
    """dy/dLambda on the meshes: steps i-iii, each channel's derivative at
    its own mesh (zero elsewhere)."""
    V = project_mesh(prob, mesh, y)
    pp, ph = chi_dot_at(prob, lam, mesh.l_values)
    dy = products(V, pp, ph)
    dy[0][mesh.w_p == 0] = 0.0
    dy[1:, mesh.w_cd == 0] = 0.0
    return dy
