"""Learned filter proposal: MLP forward/gradient against the float64 CPU
reference on the same FP16-rounded weights, features and exact labels
against the CPU restatement, exact hulls whatever the weights, training
that lowers the loss, and the gain over the plain quadrilateral."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import learned as OL
from oracle import mlp as OM
from paper_1508_05931_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx(hull_lib):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = hull_lib.Context(0, proposal=1, collect_stats=True)
    yield c
    c.close()


def test_mlp_forward_matches_cpu(ctx):
    w = OM.init_params(3)
    ctx.mlp_set_params(w)
    rng = np.random.default_rng(1)
    X = rng.random((37, 64)).astype(np.float32)
    z = ctx.mlp_forward(X)
    zr, _ = OM.forward(OM.round16(w), X.astype(np.float64))
    assert np.allclose(z, zr, rtol=1e-4, atol=1e-4 * np.abs(zr).max())


def test_mlp_gradient_matches_cpu(ctx):
    w = OM.init_params(4)
    ctx.mlp_set_params(w)
    rng = np.random.default_rng(2)
    X = rng.random((50, 64)).astype(np.float32)
    Y = rng.standard_normal((50, 32)).astype(np.float32) * 0.1
    g, loss = ctx.mlp_gradient(X, Y)
    gr, lr = OM.gradient(OM.round16(w), X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - lr) <= 1e-4 * abs(lr) + 1e-7
    scale = np.abs(gr).max()
    assert np.allclose(g, gr, rtol=1e-3, atol=1e-4 * scale)


@pytest.mark.parametrize("family", [0, 1, 2])
def test_features_match_cpu(ctx, family):
    pts = W.anisotropic_family(family, 300_001, 77 + family)
    f, e, exy = ctx.learned_features(torch.as_tensor(pts).cuda())
    fr, dmax, idx, dots = OL.features(pts)
    # angular bins in float32 on both sides: allow a handful of boundary cases
    assert np.abs(f[:32] - fr[:32]).sum() * len(idx) <= 8
    assert np.allclose(f[32:], fr[32:], atol=2e-3)
    # each chosen extreme attains the maximum dot product (float32 rounding)
    d = np.array([pts[e[j]].astype(np.float64) @ (np.array([math.cos(2 * math.pi * j / 32),
                                                             math.sin(2 * math.pi * j / 32)]))
                  for j in range(32)])
    assert np.all(d >= dmax - 2048.0)
    assert np.array_equal(exy, pts[e])


@pytest.mark.parametrize("family", [0, 1, 2])
def test_labels_exact(ctx, family):
    pts = W.anisotropic_family(family, 200_003, 91 + family)
    t = torch.as_tensor(pts).cuda()
    lab, qf = ctx.learned_labels(t)
    _, _, exy = ctx.learned_features(t)
    lr, qr = OL.labels(pts, exy)
    assert abs(qf - qr) < 1e-6
    assert np.allclose(lab, lr, atol=1e-6)


@pytest.mark.parametrize("weights", ["random", "zero", "huge"])
@pytest.mark.parametrize("gen", ["aniso", "ellipse", "clusters", "square", "ring", "ties"])
def test_learned_hull_is_exact(ctx, weights, gen):
    w = {"random": OM.init_params(5), "zero": np.zeros(OM.N_PARAMS, np.float32),
         "huge": OM.init_params(6) * 1e3}[weights]
    ctx.mlp_set_params(w)
    n = 400_001
    pts = {"aniso": lambda: W.anisotropic_gaussian(n, 3),
           "ellipse": lambda: W.elliptic_disk(n, 4),
           "clusters": lambda: W.gaussian_clusters(n, 5),
           "square": lambda: W.uniform_square(n, 1 << 29, 6),
           "ring": lambda: W.near_circle(n, 2.0 ** 22, 7),
           "ties": lambda: np.random.default_rng(8).integers(-4, 5, size=(n, 2)).astype(np.int32)}[gen]()
    h = ctx.compute(torch.as_tensor(pts).cuda()).cpu().numpy()
    assert h.tolist() == oracle.hull(pts).tolist()


@pytest.mark.parametrize("family", ["aniso", "ellipse", "clusters"])
def test_learned_hull_exact_full_size(ctx, family):
    """The three anisotropic families at their full 20M points, learned
    polygon in use (any weights keep the hull exact)."""
    ctx.mlp_set_params(OM.init_params(9))
    pts = {"aniso": lambda: W.anisotropic_gaussian(20_000_000, 5),
           "ellipse": lambda: W.elliptic_disk(20_000_000, 6),
           "clusters": lambda: W.gaussian_clusters(20_000_000, 7)}[family]()
    h = ctx.compute(torch.as_tensor(pts).cuda()).cpu().numpy()
    assert h.tolist() == oracle.hull(pts).tolist()


def test_checkpoint_roundtrip(ctx, hull_lib, tmp_path):
    w = OM.init_params(7)
    ctx.mlp_set_params(w)
    path = str(tmp_path / "p.gbhl")
    ctx.save_proposal(path)
    ctx.mlp_set_params(np.zeros_like(w))
    ctx.load_proposal(path)
    assert np.array_equal(ctx.mlp_get_params(), w)
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    with pytest.raises(hull_lib.HullError):
        ctx.load_proposal(path)


def test_training_lowers_loss_and_beats_quadrilateral(ctx):
    """A network trained by the library's own kernels on method-measured
    labels must discard more than the plain quadrilateral on held-out
    anisotropic instances, with the hull unchanged."""
    from paper_1508_05931_gb300 import learned as L
    X, Y = L.make_dataset(ctx, 96, seed0=1000, lo=5e4, hi=2e5)
    losses = L.train(ctx, X, Y, steps=1500, lr=2e-3, batch=48)
    assert np.mean(losses[-50:]) < 0.5 * np.mean(losses[:20])
    gain = []
    for k in range(9):
        pts = L.instance(k % 3, 300_000, 5000 + k)
        t = torch.as_tensor(pts).cuda()
        dl = L.discard_fraction(ctx, t)
        assert ctx.last_stats()["learned_used"] in (0, 1)
        h = ctx.compute(t).cpu().numpy()
        assert h.tolist() == oracle.hull(pts).tolist()
        dq = 1.0 - len(oracle.quad_filter(pts)) / len(pts)
        gain.append(dl - dq)
        assert dl >= dq - 1e-9
    assert np.mean(gain) > 0.0
