"""Training driver of the learned filter proposal.

Data: seeded instances of the three anisotropic families (Gaussian with
axis ratio 1-100 and random rotation, elliptic disk with aspect 1-100,
mixtures of 8 Gaussian clusters).  Features and labels are computed on the
GPU by the library (hull_learned_features / hull_learned_labels: the
discard fraction each direction's extreme adds to the quadrilateral,
counted exactly); the MLP is trained by the library's own forward,
backward and Adam kernels (hull_mlp_train_step).  Everything numeric runs
in the CUDA library; this module only draws inputs and loops.
"""
from __future__ import annotations

import math

import numpy as np

from . import hull as _hull
from . import workloads as W


def init_params(seed: int) -> np.ndarray:
    """He-style random initialisation of the 64-128-128-32 network."""
    rng = np.random.default_rng(seed)
    shapes = [(128, 64), (128,), (128, 128), (128,), (32, 128), (32,)]
    parts = []
    for shp in shapes:
        if len(shp) == 2:
            parts.append(rng.standard_normal(shp) * math.sqrt(2.0 / shp[1]))
        else:
            parts.append(np.zeros(shp))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def instance(family: int, n: int, seed: int) -> np.ndarray:
    return W.anisotropic_family(family, n, seed)


def make_dataset(ctx, count: int, seed0: int, lo: float = 1e5, hi: float = 4e5):
    """Features X (count x 64) and labels Y (count x 32) of `count` seeded
    instances (family k % 3, size log-uniform in [lo, hi])."""
    import torch
    rng = np.random.default_rng(seed0)
    X = np.zeros((count, 64), np.float32)
    Y = np.zeros((count, 32), np.float32)
    for k in range(count):
        n = int(math.exp(rng.uniform(math.log(lo), math.log(hi))))
        pts = torch.as_tensor(instance(k % 3, n, seed0 + k)).cuda(ctx.device)
        X[k] = ctx.learned_features(pts)[0]
        Y[k] = ctx.learned_labels(pts)[0]
    return X, Y


def train(ctx, X, Y, steps: int = 3000, lr: float = 2e-3, batch: int = 64, seed: int = 0):
    """Mini-batch Adam on the device; returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    Xd = torch.as_tensor(X).cuda(ctx.device)
    Yd = torch.as_tensor(Y).cuda(ctx.device)
    ctx.mlp_set_params(init_params(seed))
    losses = []
    for step in range(steps):
        idx = torch.as_tensor(rng.integers(0, len(X), size=min(batch, len(X)))).cuda(ctx.device)
        xb = Xd.index_select(0, idx).contiguous()
        yb = Yd.index_select(0, idx).contiguous()
        losses.append(ctx.mlp_train_step(xb, yb, lr))
    return losses


def discard_fraction(ctx, pts) -> float:
    """Fraction of points discarded by the first-round filter in the last
    hull of `pts` under the context's proposal setting."""
    ctx.compute(pts)
    st = ctx.last_stats()
    return 1.0 - st["s"] / max(st["n"], 1)
