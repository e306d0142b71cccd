"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module holds only workload descriptions and random draws: model
parameters, grid sizes, bond lists (lattice geometry the caller chooses) and
seeded random states.  It contains none of the method's arithmetic (no
dispersion, form factor, loop, projection or flow formula), so that the oracle
and the CUDA path can both take their inputs from here without sharing code.

All inputs are analytic model inputs of the t-t' Hubbard model on the square
lattice (Sec. 4 of the paper); no dataset is involved.
"""
from __future__ import annotations

import numpy as np

# Bond vectors of the square lattice grouped into shells of equal length
# (onsite, 1st NN, 2nd NN, ...).  "Truncation at the n-th nearest neighbour"
# (Sec. 3) keeps shells 0..n.  Within a shell the order is fixed so that both
# implementations enumerate bonds identically.
SHELLS = [
    [(0, 0)],
    [(1, 0), (0, 1), (-1, 0), (0, -1)],
    [(1, 1), (-1, 1), (-1, -1), (1, -1)],
    [(2, 0), (0, 2), (-2, 0), (0, -2)],
    [(2, 1), (1, 2), (-1, 2), (-2, 1), (-2, -1), (-1, -2), (1, -2), (2, -1)],
    [(2, 2), (-2, 2), (-2, -2), (2, -2)],
    [(3, 0), (0, 3), (-3, 0), (0, -3)],
]


def bonds_for_shells(n_shells: int) -> np.ndarray:
    """Bond list (int32 [n][2]) of all shells 0..n_shells (complete shells)."""
    out = []
    for s in range(n_shells + 1):
        out.extend(SHELLS[s])
    return np.asarray(out, dtype=np.int32)


def n_ff_for_shells(n_shells: int) -> int:
    return sum(len(SHELLS[s]) for s in range(n_shells + 1))


# Workloads on which the flow is run (t in units of 1; energies in units of t).
# cfg1: small case the oracle finishes in seconds.
# cfg2: production size (three t' values, van Hove filling mu = 4 t').
# cfg5: large scale.
CONFIGS = {
    "cfg1": dict(t=1.0, tp=-0.25, mu=-1.0, U=3.0, shells=1, nc=8, nf=96,
                 lambda0=10.0, lambda_min=1e-3, threshold=50.0),
    "cfg2": dict(t=1.0, tp=-0.25, mu=-1.0, U=3.0, shells=3, nc=24, nf=480,
                 lambda0=10.0, lambda_min=1e-3, threshold=50.0),
    "cfg5": dict(t=1.0, tp=-0.3, mu=-1.2, U=3.5, shells=5, nc=48, nf=960,
                 lambda0=10.0, lambda_min=1e-3, threshold=50.0),
}
CFG2_TPRIME = (-0.1, -0.25, -0.35)


def config(name: str, **over) -> dict:
    c = dict(CONFIGS[name])
    c.update(over)
    return c


def random_state(seed: int, nl: int, nff: int, scale: float = 1.0) -> np.ndarray:
    """Seeded random coupling state y = (P, C, D) as float64 [3][nl][nff][nff].

    Each matrix is symmetric in (m, n), as exchange propagators are.
    """
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((3, nl, nff, nff)) * scale
    return 0.5 * (a + np.swapaxes(a, -1, -2))


def random_scalars(seed: int, n: int, lo: float, hi: float) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n)


# Batched phase-diagram scan: seeded draws of (t', U, density) and grid sizes.
BATCH_SEED = 1604062960
BATCH_NC = (16, 20, 24, 30, 32)
BATCH_SHELLS = (1, 2, 3, 4)          # Nff = 5, 9, 13, 21
BATCH_NF = (240, 320, 384, 480)


def batch_points(n: int, seed: int = BATCH_SEED) -> list[dict]:
    """n seeded phase-diagram points with uneven grids and form-factor counts.

    t' ~ U[-0.45, 0], U ~ U[2, 4], density ~ U[0.6, 1.0]; (nc, nf) drawn
    uniformly from the pairs with nf % (2 nc) == 0 and nf % 4 == 0, so that
    l/2 +- p stays on the fine grid.
    """
    rng = np.random.default_rng(seed)
    pairs = [(nc, nf) for nc in BATCH_NC for nf in BATCH_NF
             if nf % (2 * nc) == 0 and nf % 4 == 0]
    pts = []
    for _ in range(n):
        tp = float(rng.uniform(-0.45, 0.0))
        U = float(rng.uniform(2.0, 4.0))
        dens = float(rng.uniform(0.6, 1.0))
        nc, nf = pairs[int(rng.integers(len(pairs)))]
        shells = int(BATCH_SHELLS[int(rng.integers(len(BATCH_SHELLS)))])
        pts.append(dict(t=1.0, tp=tp, U=U, density=dens, nc=nc, nf=nf,
                        shells=shells))
    return pts


# Large-scale batch: (t', mu) points around the large single point, all on
# its grids (coarse 48x48, Nff = 25, fine 960x960) and with its U.
LARGE_BATCH_SEED = 1604062961


def large_batch_points(n: int = 16, seed: int = LARGE_BATCH_SEED) -> list[dict]:
    """n seeded (t', mu) points: t' ~ U[-0.4, -0.2], mu = 4 t' + d with
    d ~ U[-0.1, 0.1] (near van Hove filling); the other parameters and the
    grids are those of the large workload."""
    c = CONFIGS["cfg5"]
    rng = np.random.default_rng(seed)
    pts = []
    for _ in range(n):
        tp = float(rng.uniform(-0.4, -0.2))
        mu = 4.0 * tp + float(rng.uniform(-0.1, 0.1))
        pts.append(dict(t=c["t"], tp=tp, mu=mu, U=c["U"], nc=c["nc"], nf=c["nf"],
                        shells=c["shells"]))
    return pts


# Channel-specific bosonic meshes (Sec. 4): nested refinements of the coarse
# grid.  A coarse cell (centre 2 pi i / nc - pi per direction) whose centre lies
# within a channel's radius of one of its centres (periodic distance) is split
# into m x m sub-cells (m odd), each a lattice point j on l = -pi + 2 pi j /
# (nc m) carrying the sub-cell's area as weight; an unsplit cell keeps its
# coarse point with the whole cell's area.  The production-sized meshes below
# hold about as many points as the paper's (992 for P, 6632 for C and D) on the
# production coarse grid: P refined around l = 0 (pairing), C and D around
# l = 0 and (pi, pi) (ferromagnetic and antiferromagnetic peaks).
PRODUCTION_MESH = dict(nc=24, m=5, p=([(0.0, 0.0)], 0.6),
                       cd=([(0.0, 0.0), (-np.pi, -np.pi)], 1.6))


def channel_mesh(nc: int, m: int, p, cd):
    """(points [n][2] int32, w_p [n], w_cd [n]) of the union of mesh_P and
    mesh_CD; p and cd are (centres [(lx, ly)], radius).  Points in
    lexicographic order of (jx, jy)."""
    if m < 1 or m % 2 == 0:
        raise ValueError("m must be odd")
    div, half = nc * m, (m - 1) // 2
    centre = -np.pi + 2.0 * np.pi * np.arange(nc) / nc

    def weights(spec):
        centres, radius = spec
        w = {}
        for ix in range(nc):
            for iy in range(nc):
                split = False
                for cx, cy in centres:
                    d = np.angle(np.exp(1j * (centre[ix] - cx))), \
                        np.angle(np.exp(1j * (centre[iy] - cy)))
                    split = split or np.hypot(*d) <= radius
                if not split:
                    w[(m * ix, m * iy)] = 1.0 / (nc * nc)
                    continue
                for a in range(-half, half + 1):
                    for b in range(-half, half + 1):
                        w[((m * ix + a) % div, (m * iy + b) % div)] = 1.0 / (div * div)
        return w

    wp, wc = weights(p), weights(cd)
    keys = sorted(set(wp) | set(wc))
    return (np.array(keys, dtype=np.int32).reshape(-1, 2),
            np.array([wp.get(k, 0.0) for k in keys]), np.array([wc.get(k, 0.0) for k in keys]))
