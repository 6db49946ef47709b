"""Thin ctypes binding over libseg.so (include/seg.h). Argument marshalling only.

torch supplies device memory and the current CUDA stream; every step of the computation runs in
libseg's kernels. There is no CPU fallback: if libseg.so is missing or the device is not sm_103a
the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libseg.so")

SEG_OK = 0
STATUS_NAMES = {0: "SEG_OK", 1: "SEG_ERR_INVALID_ARG", 2: "SEG_ERR_CUDA", 3: "SEG_ERR_OOM",
                4: "SEG_ERR_UNSUPPORTED", 5: "SEG_ERR_TIMEOUT", 6: "SEG_ERR_OVERFLOW"}
MODES = {"plain": 0, "gemm_bf16": 1, "gemm_tf32": 2, "gemm_inv_bf16": 3, "gemm_inv_tf32": 4,
         "plain_culled": 5, "culled_fused": 6}
NPTS = 21

# Every entry point the header declares: (name, restype, argtypes).
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
SIGNATURES = [
    ("seg_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("seg_last_error", ctypes.c_char_p, []),
    ("seg_create_atlas", ctypes.c_int, [_P, _P, _P, _I32, _I32, _I32, _P, ctypes.POINTER(_P)]),
    ("seg_destroy_atlas", ctypes.c_int, [_P]),
    ("seg_atlas_info", ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    ("seg_label", ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _P, _P, _P, _P]),
    ("seg_label_host", ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _P, _P]),
    ("seg_set_gemm_record_cap", ctypes.c_int, [_P, _I64]),
    ("seg_label_batch", ctypes.c_int, [_P, _I32, _P, _P, ctypes.c_int, _P, _P, _P]),
    ("seg_apply_affine", ctypes.c_int, [_P, _I64, _P, _P, _P]),
    ("seg_grad", ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    ("seg_grad_noalloc", ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P]),
    ("seg_sync_status", ctypes.c_int, [_P, _P]),
    ("seg_num_configs", ctypes.c_int32, [ctypes.c_int]),
    ("seg_set_config", ctypes.c_int, [_P, ctypes.c_int, _I32]),
    ("seg_get_config", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_I32)]),
    ("seg_gemm_stats", ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I64)]),
    ("seg_refine_affine", ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _I32,
                                         ctypes.c_double, _P, ctypes.POINTER(_I32), _P]),
    ("seg_label_multi", ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _I64, _P, _P, _P]),
    ("seg_resample", ctypes.c_int, [_P, _P, _I64, _P, _P]),
    ("seg_label_streamlines", ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_int, _P, _P, _P, _P,
                                             _P]),
    ("seg_set_classification", ctypes.c_int, [_P, ctypes.c_int]),
    ("seg_set_wait_limit", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("seg_set_scratch_limit", ctypes.c_int, [_P, _I64]),
    ("seg_get_classification", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("seg_gemm_screen_bits", ctypes.c_int, [_P, _P, _I64, ctypes.c_int, _P, _I64, _P]),
    ("seg_profile_enable", ctypes.c_int, [_P, _I32]),
    ("seg_profile_read", ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(_I64),
                                        ctypes.POINTER(ctypes.c_double)]),
]

_lib = None


class SegError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libseg.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libseg.so not found at {LIB_PATH}; build it with "
                               "`python -m paper_1912_11494_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != SEG_OK:
        raise SegError(status, lib().seg_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t, dtype, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype):
        raise ValueError(f"{name} must be a CUDA {dtype} tensor")
    return t


class Atlas:
    """Owning wrapper of a seg_atlas handle."""

    def __init__(self, centroids, bundle_of, thresholds, stream=None):
        cen = _dev(centroids, torch.float32, "centroids").contiguous()
        bo = _dev(bundle_of, torch.int32, "bundle_of").contiguous()
        thr = _dev(thresholds, torch.float32, "thresholds").contiguous()
        if cen.dim() != 3 or cen.shape[1:] != (NPTS, 3):
            raise ValueError("centroids must be [M,21,3]")
        h = ctypes.c_void_p()
        _check(lib().seg_create_atlas(_ptr(cen), _ptr(bo), _ptr(thr), cen.shape[0],
                                      thr.shape[0], NPTS, _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.M = int(cen.shape[0])
        self.B = int(thr.shape[0])
        self.device = cen.device

    def close(self):
        if getattr(self, "handle", None):
            lib().seg_destroy_atlas(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def seg_create_atlas(centroids, bundle_of, thresholds, stream=None) -> Atlas:
    return Atlas(centroids, bundle_of, thresholds, stream)


def seg_label(atlas: Atlas, fibers, mode, labels, dist=None, cidx=None, orient=None,
              stream=None, n=None):
    """Enqueue labelling of fibers [n,21,3] into caller-provided outputs."""
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    if n is None:
        n = 0 if fibers is None else int(fibers.shape[0])
    _check(lib().seg_label(atlas.handle, _ptr(fibers), n, m, _ptr(labels), _ptr(dist),
                           _ptr(cidx), _ptr(orient), _stream(stream)))


def label(atlas: Atlas, fibers, mode="plain", stream=None, want_cidx=True):
    """Allocate outputs with torch and label; returns (labels, dist, cidx, orient)."""
    fib = _dev(fibers, torch.float32, "fibers").contiguous()
    n = fib.shape[0]
    dev = fib.device
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    dist = torch.empty(n, dtype=torch.float32, device=dev)
    cidx = torch.empty(n, dtype=torch.int32, device=dev) if want_cidx else None
    orient = torch.empty(n, dtype=torch.uint8, device=dev) if want_cidx else None
    seg_label(atlas, fib, mode, labels, dist, cidx, orient, stream)
    return labels, dist, cidx, orient


def seg_label_host(atlas: Atlas, fibers, mode, labels, dist=None, stream=None):
    """Enqueue labelling of host (CPU, ideally pinned) tensors: fibers [n,21,3] float32 into
    labels [n] int32 and dist [n] float32 (or None); read them after the stream completes."""
    for name, t in (("fibers", fibers), ("labels", labels), ("dist", dist)):
        if t is not None and (t.device.type != "cpu" or not t.is_contiguous()):
            raise SegError(1, f"seg_label_host: {name} must be a contiguous CPU tensor")
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    _check(lib().seg_label_host(atlas.handle, _ptr(fibers), int(fibers.shape[0]), m,
                                _ptr(labels), _ptr(dist), _stream(stream)))


def seg_label_batch(atlas: Atlas, fibers_list, mode, labels_list, dist_list=None, stream=None):
    k = len(fibers_list)
    P = ctypes.c_void_p * max(k, 1)
    fp = P(*[_ptr(f) if f is not None else None for f in fibers_list])
    cnt = (ctypes.c_int64 * max(k, 1))(*[int(f.shape[0]) if f is not None else 0
                                         for f in fibers_list])
    lp = P(*[_ptr(x) for x in labels_list])
    dp = P(*[_ptr(x) for x in dist_list]) if dist_list is not None else None
    _check(lib().seg_label_batch(atlas.handle, k, ctypes.cast(fp, ctypes.c_void_p),
                                 ctypes.cast(cnt, ctypes.c_void_p), MODES[mode] if isinstance(
                                     mode, str) else int(mode), ctypes.cast(lp, ctypes.c_void_p),
                                 ctypes.cast(dp, ctypes.c_void_p) if dp is not None else None,
                                 _stream(stream)))


def _affine_buf(affine12):
    a = [float(x) for x in (affine12.tolist() if hasattr(affine12, "tolist") else affine12)]
    if len(a) != 12:
        raise ValueError("affine must have 12 values")
    return (ctypes.c_double * 12)(*a)


def seg_apply_affine(fibers, affine12, out=None, stream=None):
    fib = _dev(fibers, torch.float32, "fibers").contiguous()
    if out is None:
        out = torch.empty_like(fib)
    buf = _affine_buf(affine12)
    _check(lib().seg_apply_affine(_ptr(fib), int(fib.shape[0]), ctypes.cast(buf, ctypes.c_void_p),
                                  _ptr(out), _stream(stream)))
    return out


def seg_grad(atlas: Atlas, fibers, affine12, cidx, orient, grad_affine, grad_centroids=None,
             cost=None, stream=None):
    buf = _affine_buf(affine12)
    _check(lib().seg_grad(atlas.handle, _ptr(fibers), int(fibers.shape[0]),
                          ctypes.cast(buf, ctypes.c_void_p), _ptr(cidx), _ptr(orient),
                          _ptr(grad_affine), _ptr(grad_centroids), _ptr(cost), _stream(stream)))


def _mode(mode):
    return MODES[mode] if isinstance(mode, str) else int(mode)


def seg_num_configs(mode) -> int:
    return int(lib().seg_num_configs(_mode(mode)))


def seg_set_config(atlas: Atlas, mode, config: int):
    _check(lib().seg_set_config(atlas.handle, _mode(mode), int(config)))


def seg_get_config(atlas: Atlas, mode) -> int:
    v = ctypes.c_int32()
    _check(lib().seg_get_config(atlas.handle, _mode(mode), ctypes.byref(v)))
    return v.value


def seg_grad_noalloc(atlas: Atlas, fibers, affine12, cidx, orient, grad_affine,
                     grad_centroids=None, cost=None, stream=None):
    """seg_grad for callers that cannot allocate device memory (fixed in-library scratch;
    at most 4,194,304 fibers per call; overlapping calls race)."""
    buf = _affine_buf(affine12)
    n = 0 if fibers is None else int(fibers.shape[0])
    _check(lib().seg_grad_noalloc(atlas.handle, _ptr(fibers), n,
                                  ctypes.cast(buf, ctypes.c_void_p), _ptr(cidx), _ptr(orient),
                                  _ptr(grad_affine), _ptr(grad_centroids), _ptr(cost),
                                  _stream(stream)))


def seg_gemm_screen_bits(atlas: Atlas, fibers, mode, stream=None):
    """Pairs the tensor-core screen of a GEMM mode keeps, as uint32 [n, words] bit rows (bit
    2c+o for directional modes, c for orientation-free ones, caller's centroid numbering)."""
    fib = _dev(fibers, torch.float32, "fibers").contiguous()
    m = _mode(mode)
    cols = atlas.M if m in (MODES["gemm_inv_bf16"], MODES["gemm_inv_tf32"],
                            MODES["plain_culled"]) else 2 * atlas.M
    words = (cols + 31) // 32
    bits = torch.empty((fib.shape[0], words), dtype=torch.int32, device=fib.device)
    _check(lib().seg_gemm_screen_bits(atlas.handle, _ptr(fib), int(fib.shape[0]), m,
                                      _ptr(bits), words, _stream(stream)))
    return bits


def seg_refine_affine(atlas: Atlas, fibers, affine12, mode="plain", iters=50, step_mm=0.5,
                      stream=None):
    """Refine a subject-to-atlas affine: returns (best affine float64 [12], cost history [k+1])."""
    fib = _dev(fibers, torch.float32, "fibers").contiguous()
    aff = (ctypes.c_double * 12)(*[float(x) for x in affine12])
    cost = (ctypes.c_double * (int(iters) + 1))()
    done = ctypes.c_int32()
    _check(lib().seg_refine_affine(atlas.handle, _ptr(fib), int(fib.shape[0]), _mode(mode),
                                   ctypes.cast(aff, ctypes.c_void_p), int(iters), float(step_mm),
                                   ctypes.cast(cost, ctypes.c_void_p), ctypes.byref(done),
                                   _stream(stream)))
    import numpy as np
    return np.array(aff[:]), np.array(cost[: done.value + 1])


def label_multi(atlas: Atlas, fibers, mode="plain", stream=None):
    """Every bundle each fiber passes: (bits int32 [n, ceil(B/32)] bit rows, labels, dist)."""
    fib = _dev(fibers, torch.float32, "fibers").contiguous()
    n = int(fib.shape[0])
    words = (atlas.B + 31) // 32
    bits = torch.empty((n, words), dtype=torch.int32, device=fib.device)
    labels = torch.empty(n, dtype=torch.int32, device=fib.device)
    dist = torch.empty(n, dtype=torch.float32, device=fib.device)
    _check(lib().seg_label_multi(atlas.handle, _ptr(fib), n, _mode(mode), _ptr(bits), words,
                                 _ptr(labels), _ptr(dist), _stream(stream)))
    return bits, labels, dist


def seg_resample(points, offsets, out=None, stream=None):
    """21 arc-length-equidistant points per raw streamline: points CUDA float32 [P, 3], offsets
    CUDA int64 [n + 1]; returns (or fills) float32 [n, 21, 3]."""
    pts = _dev(points, torch.float32, "points").contiguous()
    off = _dev(offsets, torch.int64, "offsets").contiguous()
    n = int(off.shape[0]) - 1
    if out is None:
        out = torch.empty((n, NPTS, 3), dtype=torch.float32, device=pts.device)
    _check(lib().seg_resample(_ptr(pts), _ptr(off), n, _ptr(out), _stream(stream)))
    return out


def label_streamlines(atlas: Atlas, points, offsets, mode="plain", stream=None):
    """Resample raw streamlines and label them: returns (labels, dist, cidx, orient)."""
    pts = _dev(points, torch.float32, "points").contiguous()
    off = _dev(offsets, torch.int64, "offsets").contiguous()
    n = int(off.shape[0]) - 1
    dev = pts.device
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    dist = torch.empty(n, dtype=torch.float32, device=dev)
    cidx = torch.empty(n, dtype=torch.int32, device=dev)
    orient = torch.empty(n, dtype=torch.uint8, device=dev)
    _check(lib().seg_label_streamlines(atlas.handle, _ptr(pts), _ptr(off), n, _mode(mode),
                                       _ptr(labels), _ptr(dist), _ptr(cidx), _ptr(orient),
                                       _stream(stream)))
    return labels, dist, cidx, orient


CLASSIFICATIONS = {"eq2": 0, "eq2_tn": 1, "paper": 2}


def seg_set_classification(atlas: Atlas, cls):
    """Classification of later labelling calls: "eq2" (default), "eq2_tn" (Eq. 2 + TN) or
    "paper" (direction inferred from the end points, + TN)."""
    _check(lib().seg_set_classification(atlas.handle, CLASSIFICATIONS[cls] if isinstance(cls, str)
                                        else int(cls)))


def seg_get_classification(atlas: Atlas) -> str:
    v = ctypes.c_int()
    _check(lib().seg_get_classification(atlas.handle, ctypes.byref(v)))
    return {i: k for k, i in CLASSIFICATIONS.items()}[v.value]


def seg_set_wait_limit(atlas: Atlas, ns: int):
    _check(lib().seg_set_wait_limit(atlas.handle, int(ns)))


def seg_set_scratch_limit(atlas: Atlas, nbytes: int):
    _check(lib().seg_set_scratch_limit(atlas.handle, int(nbytes)))


def seg_sync_status(atlas: Atlas, stream=None):
    _check(lib().seg_sync_status(atlas.handle, _stream(stream)))


def seg_set_gemm_record_cap(atlas: Atlas, records: int):
    _check(lib().seg_set_gemm_record_cap(atlas.handle, int(records)))


def seg_gemm_stats(atlas: Atlas):
    p, s, o, c, d = (ctypes.c_int64() for _ in range(5))
    _check(lib().seg_gemm_stats(atlas.handle, ctypes.byref(p), ctypes.byref(s), ctypes.byref(o),
                                ctypes.byref(c), ctypes.byref(d)))
    return dict(pairs=p.value, survivors=s.value, overflow_fibers=o.value, screened=c.value,
                point_distances=d.value)


PROFILED_KERNELS = ("plain", "batch", "gemm_sort", "gemm_prep", "gemm_screen", "cull_screen",
                    "gemm_exact", "gemm_finalize", "grad", "culled_fused")


def seg_profile_enable(atlas: Atlas, enable: bool = True):
    _check(lib().seg_profile_enable(atlas.handle, 1 if enable else 0))


def seg_profile_read(atlas: Atlas, kernel: str):
    """(launches, total milliseconds) of one kernel since profiling was enabled."""
    c = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(lib().seg_profile_read(atlas.handle, kernel.encode(), ctypes.byref(c),
                                  ctypes.byref(ms)))
    return c.value, ms.value
