"""CPU float64 reference of the learned-proposal MLP -- TEST INFRASTRUCTURE
ONLY (imported by tests only).

64 -> 128 (ReLU) -> 128 (ReLU) -> 32, parameters laid out W1[128][64],
b1[128], W2[128][128], b2[128], W3[32][128], b3[32].  The device kernels
run the forward pass on FP16-rounded weights; ``round16`` gives the same
weights here so both sides evaluate the same function.  Loss: mean squared
error over all B x 32 outputs.  Pinned by a finite-difference gradient
check and a closed-form tiny network in tests/test_mlp_oracle.py.
"""
from __future__ import annotations

import numpy as np

D0, D1, D2, D3 = 64, 128, 128, 32
SHAPES = [("W1", (D1, D0)), ("b1", (D1,)), ("W2", (D2, D1)), ("b2", (D2,)), ("W3", (D3, D2)), ("b3", (D3,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = flat[o:o + k].reshape(shp)
        o += k
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def round16(flat):
    return np.asarray(flat, np.float32).astype(np.float16).astype(np.float64)


def forward(flat, X):
    p = unpack(flat)
    X = np.asarray(X, np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    return z, (X, a1, h1, a2, h2)


def loss(flat, X, Y):
    z, _ = forward(flat, X)
    return float(np.mean((z - np.asarray(Y, np.float64)) ** 2))


def gradient(flat, X, Y):
    """Backpropagation of the mean squared error (chain rule, layer by layer)."""
    p = unpack(flat)
    z, (X, a1, h1, a2, h2) = forward(flat, X)
    Y = np.asarray(Y, np.float64)
    dz = 2.0 * (z - Y) / z.size
    g = {"W3": dz.T @ h2, "b3": dz.sum(0)}
    dh2 = dz @ p["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(0)
    return pack(g), float(np.mean((z - Y) ** 2))


def init_params(seed: int) -> np.ndarray:
    """He-style random initialisation (float32 values)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W"):
            parts.append(rng.standard_normal(shp) * np.sqrt(2.0 / shp[1]))
        else:
            parts.append(np.zeros(shp))
    return pack(dict(zip([n for n, _ in SHAPES], parts))).astype(np.float32)
