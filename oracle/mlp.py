"""FP64 oracle of the warm-start network (TEST INFRASTRUCTURE, like the rest of
``oracle/``): a 3-layer MLP n_in -> h (GELU) -> h (GELU) -> n_out with the
mean-squared-error loss, written as plain matrix algebra (numpy).

Parameters are packed W1 (n_in x h, row-major), b1, W2 (h x h), b2,
W3 (h x n_out), b3 -- the CUDA library's layout -- so the same vector can be
given to both.  GELU(x) = x Phi(x) with the exact normal CDF.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def sizes(n_in, h, n_out):
    return [(n_in, h), (h,), (h, h), (h,), (h, n_out), (n_out,)]


def unpack(p, n_in, h, n_out):
    out, o = [], 0
    for shp in sizes(n_in, h, n_out):
        k = int(np.prod(shp))
        out.append(np.asarray(p[o:o + k], dtype=np.float64).reshape(shp))
        o += k
    return out


def pack(parts):
    return np.concatenate([np.ravel(a) for a in parts])


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p, Xn, n_in, h, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h, n_out)
    Z1 = Xn @ W1 + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2 + b2
    H2 = gelu(Z2)
    Y = H2 @ W3 + b3
    return Y, (Xn, Z1, H1, Z2, H2)


def loss_and_grad(p, Xn, Tn, n_in, h, n_out):
    """Mean over all entries of (Y - T)^2, and its gradient (packed)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h, n_out)
    Y, (X, Z1, H1, Z2, H2) = forward(p, Xn, n_in, h, n_out)
    D = Y - Tn
    loss = float(np.mean(D * D))
    dY = 2.0 * D / D.size
    dW3 = H2.T @ dY
    db3 = dY.sum(0)
    dZ2 = (dY @ W3.T) * gelu_grad(Z2)
    dW2 = H1.T @ dZ2
    db2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2.T) * gelu_grad(Z1)
    dW1 = X.T @ dZ1
    db1 = dZ1.sum(0)
    return loss, pack([dW1, db1, dW2, db2, dW3, db3])


def normalize_inputs(X, lo, hi):
    return 2.0 * (np.asarray(X, np.float64) - lo) / (np.asarray(hi) - lo) - 1.0


def normalize_outputs(Y, mean, sd):
    return (np.asarray(Y, np.float64) - mean) / sd


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, bias-corrected); returns new p, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    return p - lr * (m / (1 - b1**t)) / (np.sqrt(v / (1 - b2**t)) + eps), m, v


def warmstart_nodes(y, n_points, n_cells, periodic, dx, weights, max_per_species=0):
    """Profiles and particle counts of a warm start (the step from the network's
    prediction to the particle loader): `y` = [log10 ne, log10 ni, Te] at
    n_points points spanning [0, L]; each is interpolated linearly to the nodes
    (node i at fraction i / n_cells of the span), densities exponentiated, Te
    clipped at 0; the count of species s is the trapezoid integral of its
    density over the cells divided by its weight, rounded to the nearest
    integer, capped at max_per_species when that is positive.  Returns
    (ne, ni, te, [n_e, n_i]) on the n_cells (periodic) or n_cells + 1 nodes."""
    y = np.asarray(y, dtype=np.float64).ravel()
    n_nodes = n_cells if periodic else n_cells + 1
    s = np.arange(n_nodes) / n_cells * (n_points - 1)
    k = np.minimum(np.floor(s).astype(int), n_points - 2)
    t = s - k

    def at(base):
        return (1 - t) * y[base + k] + t * y[base + k + 1]

    ne, ni = 10.0 ** at(0), 10.0 ** at(n_points)
    te = np.maximum(0.0, at(2 * n_points))
    counts = []
    for d, w in zip((ne, ni), weights):
        right = np.roll(d, -1) if periodic else d[1:]
        total = float(np.sum(0.5 * (d[:n_cells] + right[:n_cells]) * dx))
        n = int(np.floor(total / w + 0.5))
        if max_per_species > 0:
            n = min(n, max_per_species)
        counts.append(n)
    return ne, ni, te, counts
