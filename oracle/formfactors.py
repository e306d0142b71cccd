"""Bond form factors adapted to the C4v point group (oracle; test infrastructure).

Sec. 3 (footnote on the basis): every form factor belongs to one bond length
and transforms under an irreducible representation of C4v (s, p, d, g).  A
truncation "at the n-th nearest neighbour" keeps all bonds of shells 0..n.
Sec. 2.3: for a Bravais lattice the form factors can be chosen real.

The basis is orthonormal under the Brillouin-zone average,
<f_m f_n> = (1/N) sum_k f_m(k) f_n(k) = delta_mn, and every function has a
definite parity f_m(-k) = pi_m f_m(k) (App. C).  Order within a shell is
A1, then B1/B2/A2, then the E pairs (x-like, y-like).

Reading (the paper names only the irreps): within a shell, the following
real functions are used (c = cos, s = sin, r2 = sqrt 2):
  shell 0 (0,0):      1
  shell 1 (1,0):      cx+cy, cx-cy, r2 sx, r2 sy
  shell 2 (1,1):      2 cx cy, 2 sx sy, 2 sx cy, 2 cx sy
  shell 3 (2,0):      c2x+c2y, c2x-c2y, r2 s2x, r2 s2y
  shell 4 (2,1):      r2(c2x cy + cx c2y), r2(c2x cy - cx c2y),
                      r2(s2x sy + sx s2y), r2(s2x sy - sx s2y),
                      2 s2x cy, 2 cx s2y, 2 sx c2y, 2 c2x sy
  shell 5 (2,2):      2 c2x c2y, 2 s2x s2y, 2 s2x c2y, 2 c2x s2y
  shell 6 (3,0):      c3x+c3y, c3x-c3y, r2 s3x, r2 s3y
Any orthogonal rotation within a shell gives a covariant flow; this choice
fixes the matrix elements reported by the classification.

Bond coefficients c_m(R) with f_m(k) = sum_R c_m(R) exp(i k.R) are obtained by
an exact discrete Fourier transform of these trigonometric polynomials.

Pins: orthonormality, parity, the shell counts Nff = 1, 5, 9, 13, 21, 25
(App. A: 8.9e6 = (992 + 2*6632) * 25^2 fixes Nff = 25 at 5th NN),
orthogonality of the point-group representation matrices C^S (App. C).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

R2 = np.sqrt(2.0)
_c, _s = np.cos, np.sin

# squared bond length of each shell
SHELL_R2 = [0, 1, 2, 4, 5, 8, 9]

IRREP_SYMMETRY = {"A1": "s", "B1": "d", "B2": "d", "A2": "g", "E": "p"}


def _shell_functions(sh):
    """List of (name, irrep, parity, f(kx, ky)) for one shell."""
    if sh == 0:
        return [("1", "A1", 1, lambda x, y: np.ones(np.broadcast(x, y).shape))]
    if sh in (1, 3, 6):
        n = {1: 1, 3: 2, 6: 3}[sh]
        return [
            (f"c{n}x+c{n}y", "A1", 1, lambda x, y: _c(n * x) + _c(n * y)),
            (f"c{n}x-c{n}y", "B1", 1, lambda x, y: _c(n * x) - _c(n * y)),
            (f"r2 s{n}x", "E", -1, lambda x, y: R2 * _s(n * x) + 0.0 * y),
            (f"r2 s{n}y", "E", -1, lambda x, y: R2 * _s(n * y) + 0.0 * x),
        ]
    if sh in (2, 5):
        n = {2: 1, 5: 2}[sh]
        return [
            (f"2c{n}xc{n}y", "A1", 1, lambda x, y: 2 * _c(n * x) * _c(n * y)),
            (f"2s{n}xs{n}y", "B2", 1, lambda x, y: 2 * _s(n * x) * _s(n * y)),
            (f"2s{n}xc{n}y", "E", -1, lambda x, y: 2 * _s(n * x) * _c(n * y)),
            (f"2c{n}xs{n}y", "E", -1, lambda x, y: 2 * _c(n * x) * _s(n * y)),
        ]
    if sh == 4:
        return [
            ("A1(2,1)", "A1", 1, lambda x, y: R2 * (_c(2 * x) * _c(y) + _c(x) * _c(2 * y))),
            ("B1(2,1)", "B1", 1, lambda x, y: R2 * (_c(2 * x) * _c(y) - _c(x) * _c(2 * y))),
            ("B2(2,1)", "B2", 1, lambda x, y: R2 * (_s(2 * x) * _s(y) + _s(x) * _s(2 * y))),
            ("A2(2,1)", "A2", 1, lambda x, y: R2 * (_s(2 * x) * _s(y) - _s(x) * _s(2 * y))),
            ("2s2xcy", "E", -1, lambda x, y: 2 * _s(2 * x) * _c(y)),
            ("2cxs2y", "E", -1, lambda x, y: 2 * _c(x) * _s(2 * y)),
            ("2sxc2y", "E", -1, lambda x, y: 2 * _s(x) * _c(2 * y)),
            ("2c2xsy", "E", -1, lambda x, y: 2 * _c(2 * x) * _s(y)),
        ]
    raise ValueError(f"shell {sh} not supported")


def shell_of(bond) -> int:
    r2 = int(bond[0]) ** 2 + int(bond[1]) ** 2
    if r2 not in SHELL_R2:
        raise ValueError(f"bond {tuple(bond)} is not in a supported shell")
    return SHELL_R2.index(r2)


def shell_vectors(sh):
    r2 = SHELL_R2[sh]
    m = int(np.ceil(np.sqrt(r2)))
    return {(x, y) for x in range(-m, m + 1) for y in range(-m, m + 1)
            if x * x + y * y == r2}


# The eight operations of C4v acting on momenta, k -> S k.
POINT_GROUP = [np.array(m, dtype=np.int64) for m in (
    [[1, 0], [0, 1]], [[0, -1], [1, 0]], [[-1, 0], [0, -1]], [[0, 1], [-1, 0]],
    [[-1, 0], [0, 1]], [[1, 0], [0, -1]], [[0, 1], [1, 0]], [[0, -1], [-1, 0]])]


@dataclass
class Basis:
    bonds: np.ndarray          # [Nb][2] int, in the caller's order
    n_shells: int
    names: list
    irreps: list
    parity: np.ndarray         # [Nff] +-1
    shells: np.ndarray         # [Nff] shell of each form factor
    funcs: list

    @classmethod
    def from_bonds(cls, bonds):
        bonds = np.asarray(bonds, dtype=np.int64).reshape(-1, 2)
        present = {tuple(int(v) for v in b) for b in bonds}
        if len(present) != len(bonds):
            raise ValueError("duplicate bonds")
        shells = sorted({shell_of(b) for b in bonds})
        n_shells = max(shells)
        for sh in range(n_shells + 1):
            if not shell_vectors(sh) <= present:
                raise ValueError(f"shell {sh} incomplete")
        names, irreps, par, shs, funcs = [], [], [], [], []
        for sh in range(n_shells + 1):
            for name, irr, p, f in _shell_functions(sh):
                names.append(name)
                irreps.append(irr)
                par.append(p)
                shs.append(sh)
                funcs.append(f)
        return cls(bonds, n_shells, names, irreps, np.array(par), np.array(shs), funcs)

    @property
    def nff(self):
        return len(self.funcs)

    @property
    def max_component(self):
        return int(np.max(np.abs(self.bonds)))

    def values(self, kx, ky):
        """f_m(k) for all m: array [Nff, *shape(k)]."""
        kx = np.asarray(kx, dtype=np.float64)
        ky = np.asarray(ky, dtype=np.float64)
        return np.stack([f(kx, ky) for f in self.funcs])

    def symmetry(self, m):
        return IRREP_SYMMETRY[self.irreps[m]]

    def coefficients(self):
        """c[m][b] with f_m(k) = sum_b c[m][b] exp(i k . R_b), R_b = bonds[b].

        Exact DFT of the trigonometric polynomials on a 16 x 16 grid.
        """
        if getattr(self, "_coeff", None) is not None:
            return self._coeff
        n = 16
        k = -np.pi + 2 * np.pi * np.arange(n) / n
        kx, ky = np.meshgrid(k, k, indexing="ij")
        f = self.values(kx, ky)                               # [Nff, n, n]
        c = np.empty((self.nff, len(self.bonds)), dtype=np.complex128)
        for b, (rx, ry) in enumerate(self.bonds):
            ph = np.exp(-1j * (kx * rx + ky * ry))
            c[:, b] = (f * ph).mean(axis=(1, 2))
        # all weight must sit on the listed bonds
        recon = np.einsum("mb,bxy->mxy", c,
                          np.exp(1j * (kx[None] * self.bonds[:, 0, None, None]
                                       + ky[None] * self.bonds[:, 1, None, None])))
        assert np.allclose(recon.real, f, atol=1e-12) and np.allclose(recon.imag, 0, atol=1e-12)
        self._coeff = c
        return c

    def rep_matrix(self, S):
        """C^S with f_m(S k) = sum_mt C^S[m, mt] f_mt(k) (App. C)."""
        n = 16
        k = -np.pi + 2 * np.pi * np.arange(n) / n
        kx, ky = np.meshgrid(k, k, indexing="ij")
        skx = S[0, 0] * kx + S[0, 1] * ky
        sky = S[1, 0] * kx + S[1, 1] * ky
        fs = self.values(skx, sky).reshape(self.nff, -1)
        f = self.values(kx, ky).reshape(self.nff, -1)
        return fs @ f.T / f.shape[1]
