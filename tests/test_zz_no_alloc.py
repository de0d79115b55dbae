"""hull_compute_noalloc -- the allocation-free entry point for callers that
must not allocate device memory (see include/gbhull.h) -- must give exactly
the hull that hull_compute gives.  Two calls in a row on different inputs,
so the second call runs on the scratch array the first one left behind.
Collected last so that a failure here cannot hide any other test."""
import ctypes

import numpy as np
import pytest

from paper_1508_05931_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_hull_compute_twice(hull_lib):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    inputs = [W.uniform_disk(65536, 2.0 ** 29, 101), W.near_circle(50001, 2.0 ** 18, 102)]
    with hull_lib.Context(0) as ctx:
        for pts in inputs:
            t = torch.as_tensor(pts).cuda()
            ref = ctx.compute(t).cpu().numpy()
            out = torch.full((len(pts),), -1, dtype=torch.int32, device="cuda")
            cnt = ctypes.c_int64()
            rc = hull_lib._lib.hull_compute_noalloc(
                ctypes.c_void_p(t.data_ptr()), len(pts), ctypes.c_void_p(out.data_ptr()), out.numel(),
                ctypes.byref(cnt), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == hull_lib.HULL_OK, hull_lib.hull_status_string(rc)
            got = out[: cnt.value].cpu().numpy()
            assert np.array_equal(got, ref)


def test_noalloc_rejects_oversized_input(hull_lib):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    big = torch.zeros((hull_lib.NOALLOC_MAX_POINTS + 1, 2), dtype=torch.int32, device="cuda")
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64()
    rc = hull_lib._lib.hull_compute_noalloc(ctypes.c_void_p(big.data_ptr()), big.shape[0],
                                            ctypes.c_void_p(out.data_ptr()), out.numel(),
                                            ctypes.byref(cnt), None)
    assert rc == hull_lib.HULL_EINVAL
