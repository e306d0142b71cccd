"""Loop surrogate network (oracle; test infrastructure).

The learned part is not in the paper: a multilayer perceptron stands in for
the loop contraction of Eq. (chis) on the scales where it is accurate enough,
and the exact loops (Eq. chis) judge it.  This module is the plain FP64
statement of that network, its input/target conventions, its loss and the
gradient of the loss, against which the library's GPU training kernels are
checked.

Network (sizes = [25, H, ..., H, n_out]): the five inputs x are first mapped
to 25 fixed features (x itself; cos and sin of k pi x_0 and k pi x_1 for
k = 1..4, since the loops are periodic in l; x_2^2, x_2^3, x_2 x_3, x_2 x_4),
h_0 = embed(x), then
    z_i = W_i h_{i-1} + b_i,   h_i = silu(z_i) = z_i / (1 + exp(-z_i))
for the hidden layers, and the linear output y = W_L h_{L-1} + b_L.
Parameters flattened layer by layer: W_i ([n_i][k_i], row-major), then b_i.

Inputs: x = (l_x / pi, l_y / pi, (ln Lambda - C_LAM) / S_LAM,
             (t' - C_TP) / S_TP, (mu - C_MU) / S_MU)
for a transfer momentum l = (l_x, l_y) of the coarse grid.
Targets: the parity-allowed pairs m <= n of both loops (pp pairs first, then
ph, each in the order of the pair list) as Lambda (1 + Lambda) chi_dot_mn(l):
the scale derivative in the logarithmic variable, which stays of order one
from the start of the flow at Lambda ~ 10 t down to the critical scale.

Loss: L = sum (y - t)^2 / (N n_out) over N samples and n_out outputs;
dL/dtheta by backpropagation written out layer by layer.

Pins (tests/test_oracle_mlp.py): central finite differences of L in every
parameter block; silu' against finite differences; the stationarity of L in
the output bias when the output layer is zero and the bias is the target
mean; a network without hidden layers reduces to linear least squares
(normal equations give zero gradient at the lstsq solution).
"""
from __future__ import annotations

import numpy as np

C_LAM, S_LAM = np.log(0.1), 4.6
C_TP, S_TP = -0.225, 0.225
C_MU, S_MU = -0.9, 0.9


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


N_EMBED = 25


def embed(x):
    """The fixed feature map [N][5] -> [N][25] ahead of the first layer."""
    x = np.asarray(x, dtype=np.float64)
    cols = [x[:, j] for j in range(5)]
    for k in range(1, 5):
        a, b = k * np.pi * x[:, 0], k * np.pi * x[:, 1]
        cols += [np.cos(a), np.sin(a), np.cos(b), np.sin(b)]
    cols += [x[:, 2] ** 2, x[:, 2] ** 3, x[:, 2] * x[:, 3], x[:, 2] * x[:, 4]]
    return np.stack(cols, axis=1)


def n_params(sizes):
    return sum(n * k + n for k, n in zip(sizes[:-1], sizes[1:]))


def unflatten(theta, sizes):
    theta = np.asarray(theta, dtype=np.float64)
    layers, o = [], 0
    for k, n in zip(sizes[:-1], sizes[1:]):
        W = theta[o:o + n * k].reshape(n, k)
        o += n * k
        b = theta[o:o + n]
        o += n
        layers.append((W, b))
    if o != theta.size:
        raise ValueError("parameter vector does not match the sizes")
    return layers


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def forward(theta, sizes, x):
    """Outputs y [N][n_out] and the per-layer (input, pre-activation) cache."""
    layers = unflatten(theta, sizes)
    h = embed(x)
    cache = []
    for i, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = silu(z) if i < len(layers) - 1 else z
    return h, cache


def loss(theta, sizes, x, t):
    y, _ = forward(theta, sizes, x)
    r = y - np.asarray(t, dtype=np.float64)
    return float(np.sum(r * r) / r.size)


def loss_and_grad(theta, sizes, x, t):
    """(L, dL/dtheta) by backpropagation."""
    layers = unflatten(theta, sizes)
    y, cache = forward(theta, sizes, x)
    t = np.asarray(t, dtype=np.float64)
    r = y - t
    L = float(np.sum(r * r) / r.size)
    g = 2.0 * r / r.size                      # dL/dy
    grads = [None] * len(layers)
    for i in range(len(layers) - 1, -1, -1):
        h, z = cache[i]
        if i < len(layers) - 1:
            g = g * dsilu(z)                  # through h_i = silu(z_i)
        grads[i] = (g.T @ h, g.sum(axis=0))   # dL/dW_i, dL/db_i
        g = g @ layers[i][0]                  # dL/dh_{i-1}
    return L, flatten(grads)


def features(lx, ly, lam, tp, mu):
    """Network inputs [N][5] of transfer momenta (lx, ly) at scale lam."""
    lx = np.asarray(lx, dtype=np.float64)
    ly = np.asarray(ly, dtype=np.float64)
    n = lx.size
    return np.stack([lx / np.pi, ly / np.pi,
                     np.full(n, (np.log(lam) - C_LAM) / S_LAM),
                     np.full(n, (tp - C_TP) / S_TP),
                     np.full(n, (mu - C_MU) / S_MU)], axis=1)


def targets(chi_pp, chi_ph, lam, pairs):
    """Targets [Nl][2 npair] from the loops [Nl][Nff][Nff] of both channels."""
    m = np.array([p[0] for p in pairs])
    n = np.array([p[1] for p in pairs])
    s = lam * (1.0 + lam)
    return s * np.concatenate([chi_pp[:, m, n], chi_ph[:, m, n]], axis=1)


def loops_from_outputs(y, lam, pairs, nff):
    """Inverse of targets: the loops [2][Nl][Nff][Nff] (symmetric, zeros at
    the pairs the parity selection forbids)."""
    y = np.asarray(y, dtype=np.float64) / (lam * (1.0 + lam))
    npair = len(pairs)
    out = np.zeros((2, y.shape[0], nff, nff))
    for c in range(2):
        for q, (m, n) in enumerate(pairs):
            out[c, :, m, n] = y[:, c * npair + q]
            out[c, :, n, m] = y[:, c * npair + q]
    return out


def pair_list(parity):
    """Parity-allowed pairs m <= n (pi_m pi_n = +1), row by row."""
    nff = len(parity)
    return [(m, n) for m in range(nff) for n in range(m, nff) if parity[m] * parity[n] > 0]
