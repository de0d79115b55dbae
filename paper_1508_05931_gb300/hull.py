"""Python binding of the gbhull C ABI (include/gbhull.h).

Argument marshalling only: every step of the hull runs in the CUDA library
``_lib/libgbhull.so``.  Importing this module fails loudly when that
library is missing; there is no CPU fallback.  PyTorch supplies device
memory and streams (tensor data pointers and ``torch.cuda`` streams are
passed straight through).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB_PATH
if not os.path.exists(_LIB_PATH):
    raise ImportError("libgbhull.so is not built (%s); run paper_1508_05931_gb300.build."
                      "build_library() or __graft_entry__.build()" % _LIB_PATH)
_lib = ctypes.CDLL(_LIB_PATH)

HULL_OK, HULL_EINVAL, HULL_ERANGE, HULL_ENOMEM, HULL_ECAPACITY, HULL_ETIMEOUT, HULL_ECUDA, \
    HULL_EINTERNAL = range(8)
COORD_LIMIT = 1 << 29
MAX_POINTS = (1 << 30) - 1


class hull_config(ctypes.Structure):
    _fields_ = [("proposal", ctypes.c_int), ("collect_stats", ctypes.c_int),
                ("spin_limit", ctypes.c_uint32), ("autotune", ctypes.c_int),
                ("reverse_round", ctypes.c_int), ("batched_seg_min", ctypes.c_int)]


class hull_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("s", ctypes.c_int64), ("r_lower", ctypes.c_int64),
                ("r_upper", ctypes.c_int64), ("h", ctypes.c_int64), ("ext", ctypes.c_int32 * 4),
                ("ncorner", ctypes.c_int32), ("learned_used", ctypes.c_int32),
                ("sort_fallback", ctypes.c_int32), ("s_witness", ctypes.c_int64)]


NUM_STAGES = 12
# Stage slots of hull_profile.ms on the bucket-sort path (the default) and on
# the radix-pass path (a call whose bins the bucket sort could not take).
STAGE_NAMES = ["polygon", "extremes", "witness", "filter", "scatter", "split", "sort"] + ["-%d" % i for i in range(7, 10)] + [
    "regions", "final"]
RADIX_STAGE_NAMES = ["extremes", "filter"] + ["sort_pass%d" % i for i in range(8)] + ["regions", "final"]


class hull_profile(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("radix_calls", ctypes.c_int64), ("sort_passes", ctypes.c_int64),
                ("points", ctypes.c_int64), ("survivors", ctypes.c_int64), ("second_round", ctypes.c_int64),
                ("ms", ctypes.c_double * NUM_STAGES), ("witness_survivors", ctypes.c_int64),
                ("raw_survivors", ctypes.c_int64), ("single_read_calls", ctypes.c_int64)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_PI64 = ctypes.POINTER(ctypes.c_int64)
_sig = {
    "hull_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "hull_create": ([ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(hull_config)], ctypes.c_int),
    "hull_destroy": ([_P], None),
    "hull_compute": ([_P, _P, _I64, _P, _I64, _PI64, _P], ctypes.c_int),
    "hull_compute_host": ([_P, _P, _I64, _P, _I64, _PI64, _P], ctypes.c_int),
    "hull_compute_host_multi": ([_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "hull_compute_multi": ([_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "hull_compute_batched": ([_P, _P, _P, ctypes.c_int32, _P, _I64, _P, _P], ctypes.c_int),
    "hull_compute_noalloc": ([_P, _I64, _P, _I64, _PI64, _P], ctypes.c_int),
    "hull_last_stats": ([_P, ctypes.POINTER(hull_stats)], ctypes.c_int),
    "hull_batched_max_instance": ([], ctypes.c_int64),
    "hull_bucket_group_cap": ([], ctypes.c_int64),
    "hull_mlp_num_params": ([], ctypes.c_int64),
    "hull_mlp_set_params": ([_P, _P, _I64], ctypes.c_int),
    "hull_mlp_get_params": ([_P, _P, _I64], ctypes.c_int),
    "hull_save_proposal": ([_P, ctypes.c_char_p], ctypes.c_int),
    "hull_load_proposal": ([_P, ctypes.c_char_p], ctypes.c_int),
    "hull_learned_features": ([_P, _P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "hull_learned_labels": ([_P, _P, _I64, _P, _P, _P], ctypes.c_int),
    "hull_mlp_forward": ([_P, _P, ctypes.c_int32, _P, _P], ctypes.c_int),
    "hull_mlp_gradient": ([_P, _P, _P, ctypes.c_int32, _P, _P, _P], ctypes.c_int),
    "hull_mlp_train_step": ([_P, _P, _P, ctypes.c_int32, ctypes.c_float, _P, _P], ctypes.c_int),
    "hull_set_profiling": ([_P, ctypes.c_int], ctypes.c_int),
    "hull_get_profile": ([_P, ctypes.POINTER(hull_profile)], ctypes.c_int),
    "hull_stage_extremes": ([_P, _P, _I64, _P, _P], ctypes.c_int),
    "hull_stage_filter": ([_P, _P, _I64, _P, _PI64, _P], ctypes.c_int),
    "hull_stage_sort": ([_P, _P, _P, _I64, _P], ctypes.c_int),
    "hull_stage_bucket_sort": ([_P, _P, _P, _I64, ctypes.POINTER(ctypes.c_int32), _P], ctypes.c_int),
    "hull_stage_second_round": ([_P, _P, _P, _I64, _P, _PI64, _P, _PI64, _P], ctypes.c_int),
    "hull_stage_sorted_survivors": ([_P, _P, _I64, _P, _P, _I64, _PI64, _P], ctypes.c_int),
    "hull_stage_second_round_chunked": ([_P, _P, _P, _I64, ctypes.c_int32, _P, _PI64, _P, _PI64, _P], ctypes.c_int),
    "hull_stage_regions": ([_P, _P, _I64, _P, _I64, _P, _I64, _PI64, ctypes.POINTER(ctypes.c_int32), _P],
                           ctypes.c_int),
    "hull_stage_chain": ([_P, _P, _I64, _P, _I64, _PI64, _PI64, _P], ctypes.c_int),
    "hull_stage_angular": ([_P, _P, _I64, _P, _P, _I64, _PI64, _PI64, _P], ctypes.c_int),
    "hull_compute_angular": ([_P, _P, _I64, _P, _I64, _PI64, _P], ctypes.c_int),
}
for _name, (_args, _res) in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_sig)


class HullError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where, hull_status_string(code), code))


def hull_status_string(code: int) -> str:
    return _lib.hull_status_string(int(code)).decode()


def _check(code: int, where: str):
    if code != HULL_OK:
        raise HullError(code, where)


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _as_points(pts, device):
    torch = _torch()
    if not isinstance(pts, torch.Tensor):
        pts = torch.as_tensor(np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 2)))
    if pts.dtype != torch.int32 or pts.dim() != 2 or pts.shape[1] != 2:
        raise ValueError("points must be an int32 tensor of shape (n, 2)")
    if not pts.is_cuda:
        pts = pts.to(device)
    return pts.contiguous()


class Context:
    """One hull_ctx: owns the device workspace for one GPU."""

    def __init__(self, device: int = 0, proposal: int = 0, collect_stats: bool = False,
                 spin_limit: int = 0, autotune: bool = False, reverse_round: bool = False,
                 batched_seg_min: int = 0):
        self.device = int(device)
        cfg = hull_config(int(proposal), int(bool(collect_stats)), int(spin_limit), int(bool(autotune)),
                          int(bool(reverse_round)), int(batched_seg_min))
        h = ctypes.c_void_p()
        _check(_lib.hull_create(ctypes.byref(h), self.device, ctypes.byref(cfg)), "hull_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.hull_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ hull
    def compute(self, pts, out=None, stream=None):
        """CCW hull vertex indices (int32 device tensor) of an (n, 2) int32
        point tensor; see hull_compute."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        pts = _as_points(pts, dev)
        n = pts.shape[0]
        if out is None:
            out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        cnt = ctypes.c_int64()
        _check(_lib.hull_compute(self._h, _ptr(pts), n, _ptr(out), out.numel(), ctypes.byref(cnt),
                                 _stream_handle(stream)), "hull_compute")
        return out[: cnt.value]

    def compute_raw(self, pts, out, stream=None) -> int:
        """hull_compute on preallocated tensors; returns the vertex count."""
        cnt = ctypes.c_int64()
        _check(_lib.hull_compute(self._h, _ptr(pts), pts.shape[0], _ptr(out), out.numel(),
                                 ctypes.byref(cnt), _stream_handle(stream)), "hull_compute")
        return cnt.value

    def compute_host(self, pts, out=None, stream=None) -> np.ndarray:
        """Hull of host points (numpy or CPU tensor, ideally pinned) into a
        host array; see hull_compute_host."""
        torch = _torch()
        if isinstance(pts, torch.Tensor):
            src = pts.contiguous()
            n = src.shape[0]
            sp = _ptr(src)
        else:
            src = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 2))
            n = src.shape[0]
            sp = src.ctypes.data_as(ctypes.c_void_p)
        if out is None:
            out = np.empty(max(n, 1), dtype=np.int32)
        op = _ptr(out) if isinstance(out, torch.Tensor) else out.ctypes.data_as(ctypes.c_void_p)
        cnt = ctypes.c_int64()
        _check(_lib.hull_compute_host(self._h, sp, n, op, out.shape[0], ctypes.byref(cnt),
                                      _stream_handle(stream)), "hull_compute_host")
        return out[: cnt.value]

    def compute_multi(self, pts_list, outs, stream=None) -> list:
        """Hulls of several device point sets (int32 (n, 2) CUDA tensors)
        into the device tensors `outs`, back to back with one
        synchronisation; see hull_compute_multi.  Returns one index tensor
        (a view of outs[i]) per input."""
        k = len(pts_list)
        if len(outs) != k:
            raise ValueError("one output per input")
        arr_p = (ctypes.c_void_p * max(k, 1))(*[int(t.data_ptr()) for t in pts_list])
        arr_n = (ctypes.c_int64 * max(k, 1))(*[t.shape[0] for t in pts_list])
        arr_o = (ctypes.c_void_p * max(k, 1))(*[int(o.data_ptr()) for o in outs])
        arr_c = (ctypes.c_int64 * max(k, 1))(*[o.numel() for o in outs])
        arr_h = (ctypes.c_int64 * max(k, 1))()
        _check(_lib.hull_compute_multi(self._h, k, arr_p, arr_n, arr_o, arr_c, arr_h, _stream_handle(stream)),
               "hull_compute_multi")
        return [outs[i][: arr_h[i]] for i in range(k)]

    def compute_host_multi(self, pts_list, outs=None, stream=None) -> list:
        """Hulls of several host point sets (numpy arrays or CPU tensors,
        ideally pinned), the copy of each overlapping the previous hull;
        see hull_compute_host_multi.  Returns one index array per input."""
        torch = _torch()
        k = len(pts_list)
        srcs, ns, sps = [], [], []
        for pts in pts_list:
            if isinstance(pts, torch.Tensor):
                src = pts.contiguous()
                sps.append(int(src.data_ptr()))
            else:
                src = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 2))
                sps.append(src.ctypes.data)
            srcs.append(src)
            ns.append(src.shape[0])
        if outs is None:
            outs = [np.empty(max(n, 1), dtype=np.int32) for n in ns]
        ops = [int(o.data_ptr()) if isinstance(o, torch.Tensor) else o.ctypes.data for o in outs]
        arr_p = (ctypes.c_void_p * max(k, 1))(*sps)
        arr_n = (ctypes.c_int64 * max(k, 1))(*ns)
        arr_o = (ctypes.c_void_p * max(k, 1))(*ops)
        arr_c = (ctypes.c_int64 * max(k, 1))(*[o.shape[0] for o in outs])
        arr_h = (ctypes.c_int64 * max(k, 1))()
        _check(_lib.hull_compute_host_multi(self._h, k, arr_p, arr_n, arr_o, arr_c, arr_h,
                                            _stream_handle(stream)), "hull_compute_host_multi")
        return [outs[i][: arr_h[i]] for i in range(k)]

    def compute_batched(self, pts, offsets, out=None, stream=None):
        """B hulls; offsets int64 (B+1,).  Returns (indices, out_offsets)."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        pts = _as_points(pts, dev)
        offsets = torch.as_tensor(offsets, dtype=torch.int64).to(dev).contiguous()
        b = offsets.numel() - 1
        if out is None:
            out = torch.empty(max(pts.shape[0], 1), dtype=torch.int32, device=dev)
        oo = torch.empty(b + 1, dtype=torch.int64, device=dev)
        _check(_lib.hull_compute_batched(self._h, _ptr(pts), _ptr(offsets), b, _ptr(out), out.numel(),
                                         _ptr(oo), _stream_handle(stream)), "hull_compute_batched")
        return out, oo

    def last_stats(self) -> dict:
        st = hull_stats()
        _check(_lib.hull_last_stats(self._h, ctypes.byref(st)), "hull_last_stats")
        return {"n": st.n, "s": st.s, "r_lower": st.r_lower, "r_upper": st.r_upper, "h": st.h,
                "ext": list(st.ext), "ncorner": st.ncorner, "learned_used": st.learned_used,
                "sort_fallback": st.sort_fallback, "s_witness": st.s_witness}

    def set_profiling(self, enable: bool = True):
        _check(_lib.hull_set_profiling(self._h, int(bool(enable))), "hull_set_profiling")

    def profile(self) -> dict:
        p = hull_profile()
        _check(_lib.hull_get_profile(self._h, ctypes.byref(p)), "hull_get_profile")
        names = STAGE_NAMES if p.radix_calls == 0 else RADIX_STAGE_NAMES
        return {"calls": p.calls, "radix_calls": p.radix_calls, "sort_passes": p.sort_passes, "points": p.points,
                "survivors": p.survivors, "second_round": p.second_round,
                "witness_survivors": p.witness_survivors,
                "raw_survivors": p.raw_survivors, "single_read_calls": p.single_read_calls,
                "ms": {names[k]: p.ms[k] for k in range(NUM_STAGES)}}

    # ------------------------------------------------------------ learned
    def mlp_set_params(self, params):
        w = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        _check(_lib.hull_mlp_set_params(self._h, w.ctypes.data_as(ctypes.c_void_p), w.size),
               "hull_mlp_set_params")

    def mlp_get_params(self) -> np.ndarray:
        w = np.empty(int(_lib.hull_mlp_num_params()), dtype=np.float32)
        _check(_lib.hull_mlp_get_params(self._h, w.ctypes.data_as(ctypes.c_void_p), w.size),
               "hull_mlp_get_params")
        return w

    def save_proposal(self, path: str):
        _check(_lib.hull_save_proposal(self._h, os.fsencode(path)), "hull_save_proposal")

    def load_proposal(self, path: str):
        _check(_lib.hull_load_proposal(self._h, os.fsencode(path)), "hull_load_proposal")

    def learned_features(self, pts, stream=None):
        """(features float32[64], extreme indices int32[32], extreme xy int32[32, 2])."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        pts = _as_points(pts, dev)
        f = torch.empty(64, dtype=torch.float32, device=dev)
        e = torch.empty(32, dtype=torch.int32, device=dev)
        exy = torch.empty((32, 2), dtype=torch.int32, device=dev)
        _check(_lib.hull_learned_features(self._h, _ptr(pts), pts.shape[0], _ptr(f), _ptr(e), _ptr(exy),
                                          _stream_handle(stream)), "hull_learned_features")
        return f.cpu().numpy(), e.cpu().numpy(), exy.cpu().numpy()

    def learned_labels(self, pts, stream=None):
        """(labels float32[32], quadrilateral discard fraction)."""
        torch = _torch()
        pts = _as_points(pts, torch.device("cuda", self.device))
        lab = np.empty(32, dtype=np.float32)
        q = ctypes.c_float()
        _check(_lib.hull_learned_labels(self._h, _ptr(pts), pts.shape[0], lab.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.byref(q), _stream_handle(stream)), "hull_learned_labels")
        return lab, q.value

    def mlp_forward(self, X, stream=None):
        torch = _torch()
        X = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32)).cuda(self.device)
        Z = torch.empty((X.shape[0], 32), dtype=torch.float32, device=X.device)
        _check(_lib.hull_mlp_forward(self._h, _ptr(X), X.shape[0], _ptr(Z), _stream_handle(stream)),
               "hull_mlp_forward")
        return Z.cpu().numpy()

    def mlp_gradient(self, X, Y, stream=None):
        torch = _torch()
        X = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32)).cuda(self.device)
        Y = torch.as_tensor(np.ascontiguousarray(Y, dtype=np.float32)).cuda(self.device)
        g = np.empty(int(_lib.hull_mlp_num_params()), dtype=np.float32)
        loss = ctypes.c_float()
        _check(_lib.hull_mlp_gradient(self._h, _ptr(X), _ptr(Y), X.shape[0], g.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(loss), _stream_handle(stream)), "hull_mlp_gradient")
        return g, loss.value

    def mlp_train_step(self, X_dev, Y_dev, lr: float, stream=None) -> float:
        loss = ctypes.c_float()
        _check(_lib.hull_mlp_train_step(self._h, _ptr(X_dev), _ptr(Y_dev), X_dev.shape[0], float(lr),
                                        ctypes.byref(loss), _stream_handle(stream)), "hull_mlp_train_step")
        return loss.value

    # ------------------------------------------------------------ stages
    def stage_extremes(self, pts, stream=None) -> np.ndarray:
        torch = _torch()
        pts = _as_points(pts, torch.device("cuda", self.device))
        ext = np.zeros(4, dtype=np.int32)
        _check(_lib.hull_stage_extremes(self._h, _ptr(pts), pts.shape[0],
                                        ext.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)),
               "hull_stage_extremes")
        return ext

    def stage_filter(self, pts, stream=None):
        torch = _torch()
        dev = torch.device("cuda", self.device)
        pts = _as_points(pts, dev)
        keep = torch.empty(max(pts.shape[0], 1), dtype=torch.int32, device=dev)
        s = ctypes.c_int64()
        _check(_lib.hull_stage_filter(self._h, _ptr(pts), pts.shape[0], _ptr(keep), ctypes.byref(s),
                                      _stream_handle(stream)), "hull_stage_filter")
        return keep[: s.value]

    def stage_sort(self, keys, vals, stream=None):
        """Sorts (uint64 keys stored in an int64 tensor, int32 values) in place."""
        torch = _torch()
        assert keys.dtype == torch.int64 and vals.dtype == torch.int32 and keys.is_cuda
        _check(_lib.hull_stage_sort(self._h, _ptr(keys), _ptr(vals), keys.numel(),
                                    _stream_handle(stream)), "hull_stage_sort")
        return keys, vals

    def stage_bucket_sort(self, keys, vals, stream=None):
        """Sorts (uint64 keys stored in an int64 tensor, int32 values) in place
        by (key, value) with the pipeline's bucket sort; returns True when it
        handed the pairs to the radix passes."""
        torch = _torch()
        assert keys.dtype == torch.int64 and vals.dtype == torch.int32 and keys.is_cuda
        fb = ctypes.c_int32(0)
        _check(_lib.hull_stage_bucket_sort(self._h, _ptr(keys), _ptr(vals), keys.numel(), ctypes.byref(fb),
                                           _stream_handle(stream)), "hull_stage_bucket_sort")
        return bool(fb.value)

    def stage_second_round(self, xy_sorted, labels, stream=None):
        torch = _torch()
        dev = torch.device("cuda", self.device)
        xy = _as_points(xy_sorted, dev)
        lab = torch.as_tensor(labels, dtype=torch.int32).to(dev).contiguous()
        m = xy.shape[0]
        lo = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        up = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        nl, nu = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.hull_stage_second_round(self._h, _ptr(xy), _ptr(lab), m, _ptr(lo), ctypes.byref(nl),
                                            _ptr(up), ctypes.byref(nu), _stream_handle(stream)),
               "hull_stage_second_round")
        return lo[: nl.value], up[: nu.value]

    def stage_regions(self, pts, stream=None):
        """The second-round survivors of the fused pipeline front on `pts`:
        (lower labels, upper labels, fell back to the radix passes)."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        xy = _as_points(pts, dev)
        n = xy.shape[0]
        lo = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        up = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        cnt = (ctypes.c_int64 * 2)()
        fb = ctypes.c_int32()
        _check(_lib.hull_stage_regions(self._h, _ptr(xy), n, _ptr(lo), lo.numel(), _ptr(up), up.numel(), cnt,
                                       ctypes.byref(fb), _stream_handle(stream)), "hull_stage_regions")
        return lo[: cnt[0]], up[: cnt[1]], bool(fb.value)

    def stage_sorted_survivors(self, pts, stream=None):
        """Steps 1-4 on the device: (survivor points sorted by (x, y, index),
        their input indices)."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        xy = _as_points(pts, dev)
        n = xy.shape[0]
        oxy = torch.empty((max(n, 1), 2), dtype=torch.int32, device=dev)
        oid = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        cnt = ctypes.c_int64()
        _check(_lib.hull_stage_sorted_survivors(self._h, _ptr(xy), n, _ptr(oxy), _ptr(oid), n, ctypes.byref(cnt),
                                                _stream_handle(stream)), "hull_stage_sorted_survivors")
        return oxy[: cnt.value], oid[: cnt.value]

    def stage_angular(self, pts, stream=None):
        """Steps 1-7 with the paper's angular ordering: (order, keep, l) --
        [P_0, the first-round survivors by angle about P_miny] as input
        indices, the second round's keep flags for those positions (bool),
        and the position of P_longest (-1 when P_0 is the only distinct
        point)."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        xy = _as_points(pts, dev)
        n = xy.shape[0]
        order = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        keep = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
        m, l = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.hull_stage_angular(self._h, _ptr(xy), n, _ptr(order), _ptr(keep), max(n, 1), ctypes.byref(m),
                                       ctypes.byref(l), _stream_handle(stream)), "hull_stage_angular")
        return order[: m.value], keep[: m.value].bool(), int(l.value)

    def compute_angular(self, pts, stream=None):
        """The hull by the paper's angular variant (steps 1-8 on the device):
        vertex indices, counter-clockwise from the lexicographic minimum."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        xy = _as_points(pts, dev)
        n = xy.shape[0]
        out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        h = ctypes.c_int64()
        _check(_lib.hull_compute_angular(self._h, _ptr(xy), n, _ptr(out), max(n, 1), ctypes.byref(h),
                                         _stream_handle(stream)), "hull_compute_angular")
        return out[: h.value]

    def stage_second_round_chunked(self, xy_sorted, labels, block_size=1024, stream=None):
        """Section 3.4's chunked second round over sorted points: (lower
        labels, upper labels)."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        xy = _as_points(xy_sorted, dev)
        lab = torch.as_tensor(labels, dtype=torch.int32).to(dev).contiguous()
        m = xy.shape[0]
        lo = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        up = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        nl, nu = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.hull_stage_second_round_chunked(self._h, _ptr(xy), _ptr(lab), m, int(block_size), _ptr(lo),
                                                    ctypes.byref(nl), _ptr(up), ctypes.byref(nu),
                                                    _stream_handle(stream)), "hull_stage_second_round_chunked")
        return lo[: nl.value], up[: nu.value]

    def stage_chain(self, xy_sorted, stream=None):
        """Returns (lower chain positions, upper chain positions), both from
        the first to the last point."""
        torch = _torch()
        dev = torch.device("cuda", self.device)
        xy = _as_points(xy_sorted, dev)
        m = xy.shape[0]
        out = torch.empty(2 * m, dtype=torch.int32, device=dev)
        hl, hu = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.hull_stage_chain(self._h, _ptr(xy), m, _ptr(out), out.numel(), ctypes.byref(hl),
                                     ctypes.byref(hu), _stream_handle(stream)), "hull_stage_chain")
        o = out.cpu().numpy()
        lower = o[: hl.value]
        inner = o[hl.value: hl.value + hu.value - 2][::-1]
        upper = np.concatenate([[0], inner, [m - 1]]).astype(np.int32)
        return lower.copy(), upper


NOALLOC_MAX_POINTS = 65536


def compute_noalloc(pts, out, stream=None) -> int:
    """hull_compute_noalloc on the current device: pts an (n, 2) int32 CUDA
    tensor with n <= NOALLOC_MAX_POINTS, out an int32 CUDA tensor; returns
    the vertex count (indices in out[:count]).  Allocates nothing."""
    cnt = ctypes.c_int64()
    _check(_lib.hull_compute_noalloc(_ptr(pts), pts.shape[0], _ptr(out), out.numel(), ctypes.byref(cnt),
                                     _stream_handle(stream)), "hull_compute_noalloc")
    return cnt.value


# Module-level C-ABI names (thin aliases).
hull_create = _lib.hull_create
hull_destroy = _lib.hull_destroy
hull_compute = _lib.hull_compute
hull_compute_host = _lib.hull_compute_host
hull_compute_host_multi = _lib.hull_compute_host_multi
hull_compute_batched = _lib.hull_compute_batched
hull_compute_noalloc = _lib.hull_compute_noalloc
hull_last_stats = _lib.hull_last_stats
hull_batched_max_instance = _lib.hull_batched_max_instance
hull_bucket_group_cap = _lib.hull_bucket_group_cap
hull_mlp_train_step = _lib.hull_mlp_train_step
hull_mlp_gradient = _lib.hull_mlp_gradient
hull_mlp_forward = _lib.hull_mlp_forward
hull_learned_labels = _lib.hull_learned_labels
hull_learned_features = _lib.hull_learned_features
hull_load_proposal = _lib.hull_load_proposal
hull_save_proposal = _lib.hull_save_proposal
hull_mlp_get_params = _lib.hull_mlp_get_params
hull_mlp_set_params = _lib.hull_mlp_set_params
hull_mlp_num_params = _lib.hull_mlp_num_params
hull_set_profiling = _lib.hull_set_profiling
hull_get_profile = _lib.hull_get_profile
hull_stage_extremes = _lib.hull_stage_extremes
hull_stage_filter = _lib.hull_stage_filter
hull_stage_sort = _lib.hull_stage_sort
hull_stage_bucket_sort = _lib.hull_stage_bucket_sort
hull_stage_second_round = _lib.hull_stage_second_round
hull_stage_regions = _lib.hull_stage_regions
hull_stage_second_round_chunked = _lib.hull_stage_second_round_chunked
hull_stage_sorted_survivors = _lib.hull_stage_sorted_survivors
hull_compute_multi = _lib.hull_compute_multi
hull_stage_chain = _lib.hull_stage_chain
hull_stage_angular = _lib.hull_stage_angular
hull_compute_angular = _lib.hull_compute_angular
