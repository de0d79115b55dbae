"""hull_compute_noalloc -- the allocation-free entry point for callers that
must not allocate device memory (see include/gbhull.h) -- against the
oracle: mid-size sets, every degenerate input right after a full
65,536-point call (so each runs on the scratch array a large call left
behind), the output-capacity error with its count, and the size limit.
Collected last so that a failure here cannot hide any other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1508_05931_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def noalloc(hull_lib, pts, cap=None):
    """(status, count, indices) of one call on the current stream."""
    t = torch.as_tensor(np.ascontiguousarray(pts, dtype=np.int32).reshape(-1, 2)).cuda()
    cap = len(pts) if cap is None else cap
    out = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(-1)
    rc = hull_lib._lib.hull_compute_noalloc(
        ctypes.c_void_p(t.data_ptr() if len(pts) else 0), len(pts), ctypes.c_void_p(out.data_ptr()), cap,
        ctypes.byref(cnt), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, cnt.value, out.cpu().numpy()


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def test_noalloc_matches_oracle(hull_lib, gpu):
    for pts in (W.uniform_disk(65536, 2.0 ** 29, 101), W.near_circle(50001, 2.0 ** 18, 102),
                W.uniform_square(65536, 1 << 29, 103), W.gaussian_clusters(40000, 104)):
        rc, cnt, out = noalloc(hull_lib, pts)
        assert rc == hull_lib.HULL_OK, hull_lib.hull_status_string(rc)
        assert out[:cnt].tolist() == oracle.hull(pts).tolist()


DEGENERATE = {
    "empty": np.zeros((0, 2), np.int32),
    "one": np.array([[5, 7]], np.int32),
    "two": np.array([[5, 7], [1, 2]], np.int32),
    "three_collinear": np.array([[0, 0], [2, 2], [1, 1]], np.int32),
    "triangle": np.array([[0, 0], [4, 0], [0, 3]], np.int32),
    "identical": np.full((9000, 2), 3, np.int32),
    "collinear": np.array([[i * 2, i * 3] for i in range(-500, 500)], np.int32),
    "grid": W.filled_grid(200, 150, -7, 9),
    "lattice": W.parabola_lattice(1 << 12),
    "max_coords": np.array([[-(1 << 29), -(1 << 29)], [1 << 29, -(1 << 29)], [1 << 29, 1 << 29],
                            [-(1 << 29), 1 << 29], [0, 0]], np.int32),
}


@pytest.mark.parametrize("name", sorted(DEGENERATE))
def test_noalloc_degenerate_after_a_full_call(hull_lib, gpu, name):
    big = W.uniform_disk(hull_lib.NOALLOC_MAX_POINTS, 2.0 ** 29, 7)
    rc, cnt, out = noalloc(hull_lib, big)
    assert rc == hull_lib.HULL_OK and out[:cnt].tolist() == oracle.hull(big).tolist()
    pts = DEGENERATE[name]
    rc, cnt, out = noalloc(hull_lib, pts)
    assert rc == hull_lib.HULL_OK, hull_lib.hull_status_string(rc)
    assert out[:cnt].tolist() == oracle.hull(pts).tolist()


def test_noalloc_capacity_error_reports_the_count(hull_lib, gpu):
    pts = W.near_circle(30000, 2.0 ** 16, 105)
    ref = oracle.hull(pts)
    rc, cnt, out = noalloc(hull_lib, pts, cap=len(ref) - 1)
    assert rc == hull_lib.HULL_ECAPACITY
    assert cnt == len(ref)
    rc, cnt, out = noalloc(hull_lib, pts, cap=len(ref))     # exactly enough
    assert rc == hull_lib.HULL_OK and out[:cnt].tolist() == ref.tolist()


def test_noalloc_rejects_oversized_input(hull_lib, gpu):
    big = torch.zeros((hull_lib.NOALLOC_MAX_POINTS + 1, 2), dtype=torch.int32, device="cuda")
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64()
    rc = hull_lib._lib.hull_compute_noalloc(ctypes.c_void_p(big.data_ptr()), big.shape[0],
                                            ctypes.c_void_p(out.data_ptr()), out.numel(),
                                            ctypes.byref(cnt), None)
    assert rc == hull_lib.HULL_EINVAL
