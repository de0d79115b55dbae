"""Pins for the CPU MLP reference (oracle/mlp.py): a finite-difference
gradient check and a closed-form tiny network."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = mlp.init_params(1).astype(np.float64) * 0.5
    w += rng.standard_normal(w.shape) * 0.01          # break ReLU ties
    X = rng.standard_normal((6, mlp.D0))
    Y = rng.standard_normal((6, mlp.D3))
    g, _ = mlp.gradient(w, X, Y)
    idx = rng.choice(len(w), size=60, replace=False)
    for i in idx:
        e = np.zeros_like(w)
        e[i] = 1e-6
        fd = (mlp.loss(w + e, X, Y) - mlp.loss(w - e, X, Y)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_closed_form_bias_only_network():
    # All weights zero: z = b3 everywhere; the loss gradient reaches b3 only.
    p = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    p["b3"] = np.arange(mlp.D3, dtype=np.float64)
    w = mlp.pack(p)
    X = np.ones((3, mlp.D0))
    Y = np.zeros((3, mlp.D3))
    z, _ = mlp.forward(w, X)
    assert np.array_equal(z, np.tile(np.arange(32.0), (3, 1)))
    g, l = mlp.gradient(w, X, Y)
    gp = mlp.unpack(g)
    assert np.allclose(gp["b3"], 2.0 * np.arange(32.0) / 32.0)
    assert np.all(gp["W1"] == 0) and np.all(gp["W2"] == 0) and np.all(gp["W3"] == 0)
    assert abs(l - np.mean(np.arange(32.0) ** 2)) < 1e-12


def test_relu_passes_positive_identity():
    # W1 = [I; -I] picks up x and -x, W2 = I, W3 sums back x: z = sum of |x| parts.
    p = {name: np.zeros(shp) for name, shp in mlp.SHAPES}
    p["W1"][:64, :] = np.eye(64)
    p["W1"][64:, :] = -np.eye(64)
    p["W2"] = np.eye(128)
    p["W3"][0, :] = 1.0
    x = np.linspace(-1, 1, 64)[None, :]
    z, _ = mlp.forward(mlp.pack(p), x)
    assert abs(z[0, 0] - np.abs(x).sum()) < 1e-12
