"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point that include/gbhull.h declares.  No compute call
is made (there may be no GPU)."""
import ctypes
import os
import re

import pytest

from paper_1508_05931_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hull_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build_library()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert "hull_compute" in syms and "hull_create" in syms and len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_names_match_header():
    build.build_library()
    from paper_1508_05931_gb300 import hull
    assert set(declared_symbols()) <= set(hull.EXPORTED)
    for s in declared_symbols():
        assert callable(getattr(hull, s, None)) or s in ("hull_status_string",)


def test_status_strings():
    build.build_library()
    from paper_1508_05931_gb300 import hull
    assert hull.hull_status_string(0) == "ok"
    assert "range" in hull.hull_status_string(2)


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    build.build_library()
    from paper_1508_05931_gb300 import hull
    h = ctypes.c_void_p()
    rc = hull._lib.hull_create(ctypes.byref(h), 0, None)
    assert rc != 0 and not h.value


def test_null_arguments_rejected_without_gpu():
    build.build_library()
    from paper_1508_05931_gb300 import hull
    cnt = ctypes.c_int64()
    assert hull._lib.hull_compute(None, None, 10, None, 0, ctypes.byref(cnt), None) == hull.HULL_EINVAL
    assert hull._lib.hull_last_stats(None, None) == hull.HULL_EINVAL
    hull._lib.hull_destroy(None)


def test_stage_and_variant_entries_reject_null_context_without_gpu():
    build.build_library()
    from paper_1508_05931_gb300 import hull
    a, b = ctypes.c_int64(), ctypes.c_int64()
    E = hull.HULL_EINVAL
    L = hull._lib
    assert L.hull_stage_angular(None, None, 10, None, None, 0, ctypes.byref(a), ctypes.byref(b), None) == E
    assert L.hull_compute_angular(None, None, 10, None, 0, ctypes.byref(a), None) == E
    assert L.hull_stage_sorted_survivors(None, None, 10, None, None, 0, ctypes.byref(a), None) == E
    assert L.hull_stage_second_round_chunked(None, None, None, 10, 1024, None, ctypes.byref(a), None,
                                             ctypes.byref(b), None) == E
    assert L.hull_compute_multi(None, 1, None, None, None, None, None, None) == E
