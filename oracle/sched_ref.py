"""CPU reference for the learned sub-level scheduler -- TEST INFRASTRUCTURE ONLY.

The scheduler is a project addition (the paper schedules with OpenMP's
dynamic loop scheduling, §IV); this module is the plain float64 definition
the device kernels are checked against: an MLP 5 -> 32 -> 32 -> 3 with ReLU
after each hidden layer, inputs normalised as (x - mu) * isd, and the loss
L = sum over samples and outputs of (o - y)^2 / (3 n).  Parameter layout
(flat, as in include/truss.h): mu[5], isd[5], W1[32][5], b1[32], W2[32][32],
b2[32], W3[3][32], b3[3].  The gradient is written out by the chain rule;
tests pin it against central finite differences of the loss.
"""
from __future__ import annotations

import numpy as np

F, H, V = 5, 32, 3
SIZES = [("mu", (F,)), ("isd", (F,)), ("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
         ("W3", (V, H)), ("b3", (V,))]
COUNT = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    p = np.asarray(p, np.float64)
    assert p.shape == (COUNT,)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def forward(p, x):
    """Outputs o [n, 3] and the intermediate values."""
    P = unpack(p)
    xn = (np.asarray(x, np.float64) - P["mu"]) * P["isd"]
    z1 = xn @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ P["W3"].T + P["b3"]
    return o, (xn, z1, h1, z2, h2)


def loss(p, x, y):
    o, _ = forward(p, x)
    n = o.shape[0]
    return float(((o - np.asarray(y, np.float64)) ** 2).sum() / (V * n))


def grad(p, x, y):
    """dL/dp in the flat layout (normalisation entries included)."""
    P = unpack(p)
    o, (xn, z1, h1, z2, h2) = forward(p, x)
    n = o.shape[0]
    do = 2.0 * (o - np.asarray(y, np.float64)) / (V * n)
    g = {"b3": do.sum(0), "W3": do.T @ h2}
    dh2 = do @ P["W3"]
    dz2 = dh2 * (z2 > 0)
    g["b2"] = dz2.sum(0)
    g["W2"] = dz2.T @ h1
    dh1 = dz2 @ P["W2"]
    dz1 = dh1 * (z1 > 0)
    g["b1"] = dz1.sum(0)
    g["W1"] = dz1.T @ xn
    dxn = dz1 @ P["W1"]
    x64 = np.asarray(x, np.float64)
    g["isd"] = (dxn * (x64 - P["mu"])).sum(0)
    g["mu"] = -(dxn * P["isd"]).sum(0)
    return np.concatenate([g[name].ravel() for name, _ in SIZES])


def features(size, dsum, dmax, level, todo):
    """log2(1 + .) of the five sub-level quantities, as the device computes them."""
    return np.log2(1.0 + np.stack([size, dsum, dmax, level, todo], -1).astype(np.float64))
