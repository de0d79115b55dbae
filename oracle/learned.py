"""CPU restatement of the learned-proposal features and labels -- TEST
INFRASTRUCTURE ONLY.

features: the strided sample i_k = floor(k n / S), S = min(n, 16384); its
centre (float64 mean, then float32); for every sample point the angle of
(p - c) in float32 split into 32 equal bins over (-pi, pi], the point
fraction and the maximum radius per bin (radii normalised by the largest);
and per direction u_j = (cos 2 pi j/32, sin 2 pi j/32) the maximum of
<u_j, p> over the sample.  The angle and the dot products are float32 on
the device, so bins and argmaxes are compared with a tolerance (parity of
an approximate feature); the labels are exact integer counts.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

NB = 32
SAMPLE = 16384


def sample_indices(n: int) -> np.ndarray:
    S = min(n, SAMPLE)
    return (np.arange(S, dtype=np.uint64) * np.uint64(n)) // np.uint64(S)


def features(xy):
    xy = np.asarray(xy, np.int32)
    n = len(xy)
    idx = sample_indices(n).astype(np.int64)
    p = xy[idx]
    S = len(idx)
    cx = np.float32(p[:, 0].astype(np.float64).sum() / S)
    cy = np.float32(p[:, 1].astype(np.float64).sum() / S)
    dx = p[:, 0].astype(np.float32) - cx
    dy = p[:, 1].astype(np.float32) - cy
    ang = np.arctan2(dy, dx).astype(np.float32)
    b = np.floor((ang + np.float32(3.14159265358979)) * np.float32(NB / 6.283185307179586)).astype(np.int64)
    b = np.clip(b, 0, NB - 1)
    r = np.sqrt(dx * dx + dy * dy).astype(np.float32)
    cnt = np.bincount(b, minlength=NB)
    maxr = np.zeros(NB, np.float32)
    np.maximum.at(maxr, b, r)
    mr = maxr.max()
    feat = np.concatenate([cnt / S, maxr / mr if mr > 0 else np.zeros(NB)]).astype(np.float32)
    # exact dot maxima per direction (float64 on the float32 directions)
    ang_j = np.float32(6.283185307179586) * np.arange(NB // 2, dtype=np.float32) / np.float32(NB)
    u = np.stack([np.cos(ang_j.astype(np.float64)), np.sin(ang_j.astype(np.float64))], 1)
    u = np.concatenate([u, -u], 0)
    dots = p.astype(np.float64) @ u.T
    return feat, dots.max(0), idx, dots


def inside_counts(xy, poly):
    """Number of points strictly inside the convex polygon `poly` (CCW, int64)."""
    xy = np.asarray(xy, np.int64)
    k = len(poly)
    if k < 3:
        return 0
    inside = np.ones(len(xy), bool)
    for j in range(k):
        ax, ay = int(poly[j][0]), int(poly[j][1])
        bx, by = int(poly[(j + 1) % k][0]), int(poly[(j + 1) % k][1])
        o = (bx - ax) * (xy[:, 1] - ay) - (by - ay) * (xy[:, 0] - ax)
        inside &= o > 0
    return int(inside.sum())


def labels(xy, ext_xy):
    """Label j = fraction strictly inside hull(quad corners + e_j) minus the
    fraction strictly inside the quadrilateral."""
    xy = np.asarray(xy, np.int32)
    q = oracle.quad(xy)
    base = inside_counts(xy, q)
    out = np.zeros(NB)
    for j in range(NB):
        pts = np.concatenate([q, np.asarray(ext_xy[j], np.int32)[None, :]], 0)
        h = oracle.hull(pts)
        out[j] = (inside_counts(xy, pts[h]) - base) / len(xy)
    return out, base / len(xy)
