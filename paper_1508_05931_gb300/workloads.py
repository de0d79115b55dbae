"""Seeded synthetic point sets (int32 (x, y) pairs, AoS, shape (n, 2)).

This module only draws inputs.  It holds none of the hull method's
arithmetic (no orientation tests, no filtering, no sorting), so both the
CUDA path and the CPU oracle can take their inputs from it.

The paper measures on point sets drawn uniformly in a square and in a
circle (Section 4, Tables 2-5, generated there with Qhull's ``rbox``); the
generators below stand in for those sets with project-defined seeds and
integer coordinates bounded by 2^29 in absolute value.  The near-circle
set exercises the limitation the paper names in Section 5.3 (every point
an extreme point).  The anisotropic families and the batch of uneven sizes
are the project's own workloads for the learned filter proposal and the
batched mode.
"""
from __future__ import annotations

import math

import numpy as np

COORD_LIMIT = 1 << 29


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _round_clamp(v: np.ndarray, limit: int = COORD_LIMIT) -> np.ndarray:
    # np.rint rounds half to even (IEEE default mode).
    return np.clip(np.rint(v), -limit, limit).astype(np.int32)


def uniform_square(n: int, half: int, seed: int) -> np.ndarray:
    """n points, x and y i.i.d. uniform integers in [-half, half)."""
    r = _rng(seed)
    return r.integers(-half, half, size=(n, 2), dtype=np.int64).astype(np.int32)


def uniform_disk(n: int, radius: float, seed: int, center=(0.0, 0.0)) -> np.ndarray:
    """n points uniform in the disk: r = R sqrt(u), theta = 2 pi v, in float64,
    rounded to the nearest integer (ties to even) and clamped to +-2^29."""
    g = _rng(seed)
    u = g.random(n)
    v = g.random(n)
    rr = radius * np.sqrt(u)
    th = 2.0 * math.pi * v
    out = np.empty((n, 2), dtype=np.int32)
    out[:, 0] = _round_clamp(center[0] + rr * np.cos(th))
    out[:, 1] = _round_clamp(center[1] + rr * np.sin(th))
    return out


def near_circle(n: int, radius: float, seed: int) -> np.ndarray:
    """Half the points on the integer lattice nearest the circle of the given
    radius (uniform angles), half uniform in that disk, shuffled."""
    g = _rng(seed)
    n_ring = n // 2
    th = 2.0 * math.pi * g.random(n_ring)
    ring = np.empty((n_ring, 2), dtype=np.int32)
    ring[:, 0] = _round_clamp(radius * np.cos(th))
    ring[:, 1] = _round_clamp(radius * np.sin(th))
    disk = uniform_disk(n - n_ring, radius, seed + 0x9E3779B9)
    pts = np.concatenate([ring, disk], axis=0)
    perm = g.permutation(n)
    return np.ascontiguousarray(pts[perm])


def gaussian(n: int, sigma: float, seed: int, limit: int = COORD_LIMIT - 1) -> np.ndarray:
    """Isotropic Gaussian (Box-Muller in float64), rounded, clamped."""
    g = _rng(seed)
    u1 = 1.0 - g.random(n)
    u2 = g.random(n)
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty((n, 2), dtype=np.int32)
    out[:, 0] = _round_clamp(sigma * rad * np.cos(2.0 * math.pi * u2), limit)
    out[:, 1] = _round_clamp(sigma * rad * np.sin(2.0 * math.pi * u2), limit)
    return out


def anisotropic_gaussian(n: int, seed: int, sigma_major: float = float(1 << 26)) -> np.ndarray:
    """Gaussian with axis ratio log-uniform in [1, 100], random rotation."""
    g = _rng(seed)
    ratio = math.exp(g.uniform(0.0, math.log(100.0)))
    rot = g.uniform(0.0, 2.0 * math.pi)
    a = g.standard_normal(n) * sigma_major
    b = g.standard_normal(n) * (sigma_major / ratio)
    c, s = math.cos(rot), math.sin(rot)
    out = np.empty((n, 2), dtype=np.int32)
    out[:, 0] = _round_clamp(c * a - s * b)
    out[:, 1] = _round_clamp(s * a + c * b)
    return out


def elliptic_disk(n: int, seed: int, semi_major: float = float(1 << 28)) -> np.ndarray:
    """Uniform elliptic disk, aspect log-uniform in [1, 100], rotated."""
    g = _rng(seed)
    ratio = math.exp(g.uniform(0.0, math.log(100.0)))
    rot = g.uniform(0.0, 2.0 * math.pi)
    rr = np.sqrt(g.random(n))
    th = 2.0 * math.pi * g.random(n)
    a = semi_major * rr * np.cos(th)
    b = (semi_major / ratio) * rr * np.sin(th)
    c, s = math.cos(rot), math.sin(rot)
    out = np.empty((n, 2), dtype=np.int32)
    out[:, 0] = _round_clamp(c * a - s * b)
    out[:, 1] = _round_clamp(s * a + c * b)
    return out


def gaussian_clusters(n: int, seed: int, k: int = 8) -> np.ndarray:
    """Mixture of k equal-weight isotropic Gaussian clusters; centres uniform
    in the disk of radius 2^27, sigma log-uniform in [2^20, 2^25]."""
    g = _rng(seed)
    cr = float(1 << 27) * np.sqrt(g.random(k))
    ct = 2.0 * math.pi * g.random(k)
    cx, cy = cr * np.cos(ct), cr * np.sin(ct)
    sig = np.exp(g.uniform(math.log(2.0 ** 20), math.log(2.0 ** 25), size=k))
    lab = g.integers(0, k, size=n)
    out = np.empty((n, 2), dtype=np.int32)
    out[:, 0] = _round_clamp(cx[lab] + sig[lab] * g.standard_normal(n))
    out[:, 1] = _round_clamp(cy[lab] + sig[lab] * g.standard_normal(n))
    return out


def parabola_lattice(k: int) -> np.ndarray:
    """Lattice points (t, t^2 - k^2/2) for t in [-k, k], shifted to stay in
    range; every point is a strict vertex of the hull."""
    t = np.arange(-k, k + 1, dtype=np.int64)
    y = t * t - (k * k) // 2
    return np.stack([t, y], axis=1).astype(np.int32)


def filled_grid(a: int, b: int, x0: int = 0, y0: int = 0) -> np.ndarray:
    xs, ys = np.meshgrid(np.arange(a) + x0, np.arange(b) + y0, indexing="ij")
    return np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int32)


# --- named workloads ------------------------------------------------------

def small_square(n: int = 100_000, seed: int = 0) -> np.ndarray:
    """100,000 points uniform in [-2^20, 2^20)^2, seed 0."""
    return uniform_square(n, 1 << 20, seed)


def paper_square(n: int = 20_000_000, seed: int = 1) -> np.ndarray:
    """Paper-scale square set: 2e7 points uniform in [-2^29, 2^29)^2."""
    return uniform_square(n, 1 << 29, seed)


def paper_disk(n: int = 20_000_000, seed: int = 2) -> np.ndarray:
    """Paper-scale circle set: 2e7 points uniform in the disk of radius 2^29."""
    return uniform_disk(n, float(1 << 29), seed)


def adversarial_ring(n: int = 4_000_000, seed: int = 3) -> np.ndarray:
    """4e6 points: half on the lattice nearest the circle of radius 2^28,
    half uniform in that disk."""
    return near_circle(n, float(1 << 28), seed)


def batch_sizes(b: int = 4096, seed: int = 4, lo: float = 1e3, hi: float = 1e6,
                cap: float = 2.5e8) -> np.ndarray:
    """Instance sizes floor(exp(U[ln lo, ln hi])); while the total exceeds the
    cap the largest size is redrawn from log-uniform [lo, that size)."""
    g = _rng(seed)
    sizes = np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), size=b))).astype(np.int64)
    total = int(sizes.sum())
    while total > cap:
        j = int(np.argmax(sizes))
        old = int(sizes[j])
        new = int(math.floor(math.exp(g.uniform(math.log(lo), math.log(old)))))
        sizes[j] = new
        total += new - old
    return sizes


def batch(b: int = 4096, seed: int = 4, cap: float = 2.5e8, lo: float = 1e3,
          hi: float = 1e6):
    """Batch of b instances, family chosen with probability 1/3 each from
    square [-2^29, 2^29)^2, disk R = 2^29 and Gaussian sigma = 2^26.
    Returns (points (sum n, 2) int32, offsets (b + 1,) int64, families)."""
    sizes = batch_sizes(b, seed, lo, hi, cap)
    g = _rng(seed + 7919)
    fam = g.integers(0, 3, size=b)
    parts = []
    for i in range(b):
        s = int(sizes[i])
        sd = int(seed) * 1_000_003 + i
        if fam[i] == 0:
            parts.append(uniform_square(s, 1 << 29, sd))
        elif fam[i] == 1:
            parts.append(uniform_disk(s, float(1 << 29), sd))
        else:
            parts.append(gaussian(s, float(1 << 26), sd))
    offs = np.zeros(b + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    pts = np.concatenate(parts, axis=0) if parts else np.zeros((0, 2), np.int32)
    return np.ascontiguousarray(pts), offs, fam


def anisotropic_family(family: int, n: int, seed: int) -> np.ndarray:
    """family 0: anisotropic Gaussian, 1: elliptic disk, 2: 8 clusters."""
    if family == 0:
        return anisotropic_gaussian(n, seed)
    if family == 1:
        return elliptic_disk(n, seed)
    return gaussian_clusters(n, seed)
