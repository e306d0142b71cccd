"""Model, momentum grids and problem container (oracle; test infrastructure).

Dispersion: Eq. (hubb-disp), Sec. 4 --
    eps(k) = -2 t (cos kx + cos ky) - 4 t' cos kx cos ky - mu.
The bare interaction is the on-site Hubbard U (Sec. 3/4).

Grids.  A uniform grid of n points per direction holds k_i = -pi + 2 pi i / n.
Coarse (bosonic l) momenta are stored as integers u = 2 i - n in units of
pi / n, so that l / 2 is an integer number of units and folding into the
half-open zone [-pi, pi) is exact integer arithmetic.

Parity pins: dispersion values at high-symmetry points and van Hove filling
(tests/test_oracle_model.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import cached_property

import numpy as np

from . import formfactors as ffmod


def dispersion(kx, ky, t, tp, mu):
    """Eq. (hubb-disp)."""
    return (-2.0 * t * (np.cos(kx) + np.cos(ky))
            - 4.0 * tp * np.cos(kx) * np.cos(ky) - mu)


def grid(n: int) -> np.ndarray:
    """k_i = -pi + 2 pi i / n, i = 0..n-1."""
    return -np.pi + 2.0 * np.pi * np.arange(n) / n


def fold_units(u, n):
    """Fold a momentum given in units of pi/n into [-n, n) (i.e. [-pi, pi))."""
    return ((np.asarray(u) + n) % (2 * n)) - n


def density(t, tp, mu, nfx, nfy):
    """n(mu) = (2/Nf) sum_k [eps0_k < mu], ties counted as one half."""
    kx = grid(nfx)[:, None]
    ky = grid(nfy)[None, :]
    e0 = dispersion(kx, ky, t, tp, 0.0)
    below = np.sum(e0 < mu) + 0.5 * np.sum(e0 == mu)
    return 2.0 * below / (nfx * nfy)


def mu_for_density(n, t, tp, nfx, nfy, iters=200):
    """Chemical potential for filling n by bisection on the fine grid."""
    lo, hi = -4.0 * abs(t) - 4.0 * abs(tp) - 1.0, 4.0 * abs(t) + 4.0 * abs(tp) + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if density(t, tp, mid, nfx, nfy) < n:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@dataclass
class Problem:
    """One (t, t', mu, U) point on given coarse and fine grids.

    bonds: int array [n][2] forming complete shells (see formfactors).
    feedback: True = full TUfRG projections (Eqs. proj_VP/VC/VD);
              False = inter-channel projections switched off
              (V^P = V0 - P, V^C = V0 + C, V^D = V0 + D).
    bare: optional symmetric Nff x Nff bare matrix that replaces U e0 e0^T
          (used only with feedback=False for the matrix-ladder pin).
    """
    t: float
    tp: float
    mu: float
    U: float
    bonds: np.ndarray
    ncx: int
    ncy: int
    nfx: int
    nfy: int
    feedback: bool = True
    bare: np.ndarray | None = field(default=None, repr=False)

    @cached_property
    def basis(self) -> ffmod.Basis:
        return ffmod.Basis.from_bonds(self.bonds)

    @property
    def nff(self) -> int:
        return self.basis.nff

    @property
    def nl(self) -> int:
        return self.ncx * self.ncy

    @property
    def nf(self) -> int:
        return self.nfx * self.nfy

    @cached_property
    def l_units(self) -> np.ndarray:
        """Coarse momenta in units of (pi/ncx, pi/ncy): [Nl][2], index ix*ncy+iy."""
        ux = 2 * np.arange(self.ncx) - self.ncx
        uy = 2 * np.arange(self.ncy) - self.ncy
        return np.stack(np.meshgrid(ux, uy, indexing="ij"), -1).reshape(-1, 2)

    @cached_property
    def l_values(self) -> np.ndarray:
        """Coarse momenta [Nl][2] in radians, in [-pi, pi)."""
        u = self.l_units
        return np.stack([u[:, 0] * np.pi / self.ncx, u[:, 1] * np.pi / self.ncy], -1)

    @cached_property
    def p_values(self) -> np.ndarray:
        """Fine-grid momenta [Nf][2] in radians, index ix*nfy+iy."""
        px, py = np.meshgrid(grid(self.nfx), grid(self.nfy), indexing="ij")
        return np.stack([px.ravel(), py.ravel()], -1)

    @cached_property
    def f_fine(self) -> np.ndarray:
        """Form factors on the fine grid [Nff][Nf] (scale independent)."""
        p = self.p_values
        return self.basis.values(p[:, 0], p[:, 1])

    def xi(self, kx, ky):
        return dispersion(kx, ky, self.t, self.tp, self.mu)

    def bare_matrix(self) -> np.ndarray:
        """Projection of V0 onto any channel: U delta_m0 delta_n0 (or `bare`)."""
        if self.bare is not None:
            return np.asarray(self.bare, dtype=np.float64)
        b = np.zeros((self.nff, self.nff))
        b[0, 0] = self.U
        return b

    def check(self):
        nmax = self.basis.max_component
        if min(self.ncx, self.ncy) < 2 * nmax + 1:
            raise ValueError("coarse grid too small for the form-factor basis")
        if self.ncx % 2 or self.ncy % 2:
            raise ValueError("coarse grid must have an even number of points")
        return self
