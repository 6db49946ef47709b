"""FP64 CPU oracle for atlas-based fiber segmentation (arXiv:1912.11494, Section 2.3-2.4).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg use it; the product path never imports it. The arithmetic lives in
``seg_oracle.c`` (plain C, double precision, OpenMP over fibers); this module compiles it with
gcc on first use and marshals numpy arrays through ctypes.

Every function follows the paper directly: Eq. 1 (point distance), Eq. 2 (d_ME, minimum over
the direct and reversed orientation of the maximum point distance), Algorithm 1 (visit order,
strict-decrease update, closest passing bundle), Section 2.3 (progressive discarding, test1 to
test4). See ``seg_oracle.c`` for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seg_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libsegoracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction) and return the .so path."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _bind(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I32 = ctypes.c_int32
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_dme_matrix.argtypes = [P, I64, P, I64, P, P, P, ctypes.c_int]
    lib.oracle_label_brute.argtypes = [P, I64, P, P, I64, P, I32, P, P, P, P, P, ctypes.c_int]
    lib.oracle_label_cascade.argtypes = [P, I64, P, P, I64, P, I32, P, P, P, P, P, P,
                                         ctypes.c_int]
    lib.oracle_near_tie.argtypes = [P, I64, P, P, I64, P, I32, P, P, ctypes.c_double, P,
                                    ctypes.c_int]
    lib.oracle_near_tie_pruned.argtypes = lib.oracle_near_tie.argtypes
    lib.oracle_dme_pairs.argtypes = [P, I64, P, I64, P, P, P, P, ctypes.c_int]
    lib.oracle_label_cls.argtypes = [P, I64, P, P, I64, P, I32, ctypes.c_int, P, P, P, P,
                                     ctypes.c_int]
    lib.oracle_near_tie_cls.argtypes = [P, I64, P, P, I64, P, I32, ctypes.c_int, P, P,
                                        ctypes.c_double, P, ctypes.c_int]
    lib.oracle_lengths.argtypes = [P, I64, P]
    lib.oracle_resample.argtypes = [P, P, I64, P, ctypes.c_int]
    lib.oracle_label_multi.argtypes = [P, I64, P, P, I64, P, I32, ctypes.c_int, I64, P, P,
                                       ctypes.c_double, ctypes.c_int]
    lib.oracle_grad.argtypes = [P, I64, P, P, P, I64, P, I32, P, P, P, P, P, P, P, P, P, P, P,
                                ctypes.c_int]
    for f in (lib.oracle_dme_matrix, lib.oracle_label_brute, lib.oracle_label_cascade,
              lib.oracle_near_tie, lib.oracle_near_tie_pruned, lib.oracle_dme_pairs,
              lib.oracle_label_cls, lib.oracle_near_tie_cls, lib.oracle_lengths,
              lib.oracle_resample, lib.oracle_label_multi,
              lib.oracle_grad):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _ptr(x):
    return None if x is None else x.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle call failed with code {rc}")


def dme_matrix(fibers, centroids, nthreads: int = 0):
    """(d_ME, direct max, reversed max), each float64 [n, M] (Eq. 1, Eq. 2)."""
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    n, M = fib.shape[0], cen.shape[0]
    dme = np.empty((n, M))
    dd = np.empty((n, M))
    dr = np.empty((n, M))
    _check(_load().oracle_dme_matrix(_ptr(fib), n, _ptr(cen), M, _ptr(dme), _ptr(dd), _ptr(dr),
                                     nthreads))
    return dme, dd, dr


def label(fibers, centroids, bundle_of, thresholds, mode: str = "brute", nthreads: int = 0):
    """Closest passing bundle per fiber (Algorithm 1): dict of labels int32 (-1 none), dist
    float64 (+inf none, NaN for non-finite input), cidx int32, orient uint8, argmax int32 and,
    for the cascade, per-stage counts [point distances test1..4, pairs reaching test1..4]."""
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    bo = np.ascontiguousarray(bundle_of, dtype=np.int32)
    thr = _f32(thresholds)
    n, M, B = fib.shape[0], cen.shape[0], thr.shape[0]
    out = dict(labels=np.empty(n, np.int32), dist=np.empty(n), cidx=np.empty(n, np.int32),
               orient=np.empty(n, np.uint8), argmax=np.empty(n, np.int32))
    lib = _load()
    if mode == "brute":
        rc = lib.oracle_label_brute(_ptr(fib), n, _ptr(cen), _ptr(bo), M, _ptr(thr), B,
                                    _ptr(out["labels"]), _ptr(out["dist"]), _ptr(out["cidx"]),
                                    _ptr(out["orient"]), _ptr(out["argmax"]), nthreads)
    elif mode == "cascade":
        counts = np.zeros(8, np.int64)
        rc = lib.oracle_label_cascade(_ptr(fib), n, _ptr(cen), _ptr(bo), M, _ptr(thr), B,
                                      _ptr(out["labels"]), _ptr(out["dist"]), _ptr(out["cidx"]),
                                      _ptr(out["orient"]), _ptr(out["argmax"]), _ptr(counts),
                                      nthreads)
        out["counts"] = counts
    else:
        raise ValueError(mode)
    _check(rc)
    return out


def dme_pairs(fibers, centroids, idx, nthreads: int = 0):
    """(d_ME, direct max, reversed max) of fiber f against centroid idx[f], float64 [n] each
    (Eq. 1, Eq. 2); NaN where idx[f] < 0."""
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    n = fib.shape[0]
    dme, dd, dr = np.empty(n), np.empty(n), np.empty(n)
    _check(_load().oracle_dme_pairs(_ptr(fib), n, _ptr(cen), cen.shape[0], _ptr(ix), _ptr(dme),
                                    _ptr(dd), _ptr(dr), nthreads))
    return dme, dd, dr


def near_tie(fibers, centroids, bundle_of, thresholds, labels, dist, tol: float = 2e-3,
             nthreads: int = 0, pruned: bool = False):
    """uint8 [n]: 1 where the label is not decidable at tolerance tol (mm). pruned=True skips
    the centroids farther than their threshold + tol (same flags, far less work)."""
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    bo = np.ascontiguousarray(bundle_of, dtype=np.int32)
    thr = _f32(thresholds)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.float64)
    n = fib.shape[0]
    flag = np.empty(n, np.uint8)
    fn = _load().oracle_near_tie_pruned if pruned else _load().oracle_near_tie
    _check(fn(_ptr(fib), n, _ptr(cen), _ptr(bo), cen.shape[0], _ptr(thr), thr.shape[0],
              _ptr(lab), _ptr(dist), tol, _ptr(flag), nthreads))
    return flag


CLASSIFICATIONS = {"eq2": 0, "eq2_tn": 1, "paper": 2}


def label_cls(fibers, centroids, bundle_of, thresholds, cls: str, nthreads: int = 0):
    """Labelling with the length term TN of Eq. 3 (lazy, Section 2.4): cls "eq2_tn" adds TN to
    Eq. 2's d_ME; cls "paper" is the paper's new algorithm (direction inferred from test2's end
    points, tests 3-4 in that orientation only, then TN). dict of labels, dist (= D, the
    classification distance), cidx, orient. cls "eq2" is label(..., "brute")."""
    if cls == "eq2":
        r = label(fibers, centroids, bundle_of, thresholds, "brute", nthreads)
        return {k: r[k] for k in ("labels", "dist", "cidx", "orient")}
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    bo = np.ascontiguousarray(bundle_of, dtype=np.int32)
    thr = _f32(thresholds)
    n = fib.shape[0]
    out = dict(labels=np.empty(n, np.int32), dist=np.empty(n), cidx=np.empty(n, np.int32),
               orient=np.empty(n, np.uint8))
    _check(_load().oracle_label_cls(_ptr(fib), n, _ptr(cen), _ptr(bo), cen.shape[0], _ptr(thr),
                                    thr.shape[0], CLASSIFICATIONS[cls], _ptr(out["labels"]),
                                    _ptr(out["dist"]), _ptr(out["cidx"]), _ptr(out["orient"]),
                                    nthreads))
    return out


def near_tie_cls(fibers, centroids, bundle_of, thresholds, cls: str, labels, dist,
                 tol: float = 2e-3, nthreads: int = 0):
    """uint8 [n]: 1 where label_cls's result is not decidable at tolerance tol (mm)."""
    if cls == "eq2":
        return near_tie(fibers, centroids, bundle_of, thresholds, labels, dist, tol, nthreads,
                        pruned=True)
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    bo = np.ascontiguousarray(bundle_of, dtype=np.int32)
    thr = _f32(thresholds)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.float64)
    n = fib.shape[0]
    flag = np.empty(n, np.uint8)
    _check(_load().oracle_near_tie_cls(_ptr(fib), n, _ptr(cen), _ptr(bo), cen.shape[0],
                                       _ptr(thr), thr.shape[0], CLASSIFICATIONS[cls], _ptr(lab),
                                       _ptr(dist), tol, _ptr(flag), nthreads))
    return flag


def resample(points, offsets, nthreads: int = 0):
    """21 arc-length-equidistant points of each raw streamline (CSR: points float32 [P, 3],
    offsets int64 [n+1]), float64 [n, 21, 3] (Section 2.3)."""
    pts = _f32(points).reshape(-1, 3)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    n = off.shape[0] - 1
    out = np.empty((n, 21, 3))
    _check(_load().oracle_resample(_ptr(pts), _ptr(off), n, _ptr(out), nthreads))
    return out


def label_multi(fibers, centroids, bundle_of, thresholds, cls: str = "eq2",
                tol: float = 2e-3, nthreads: int = 0):
    """Every bundle each fiber passes (Section 2.4): (bits, ambiguous), uint32 [n, ceil(B/32)]
    bit rows; ambiguous marks bundles whose best centroid lies within tol of its threshold."""
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    bo = np.ascontiguousarray(bundle_of, dtype=np.int32)
    thr = _f32(thresholds)
    n, B = fib.shape[0], thr.shape[0]
    words = (B + 31) // 32
    bits = np.empty((n, words), np.uint32)
    amb = np.empty((n, words), np.uint32)
    _check(_load().oracle_label_multi(_ptr(fib), n, _ptr(cen), _ptr(bo), cen.shape[0], _ptr(thr),
                                      B, CLASSIFICATIONS[cls], words, _ptr(bits), _ptr(amb), tol,
                                      nthreads))
    return bits, amb


def lengths(fibers):
    """Polyline arc length of each 21-point fiber, float64 [n]."""
    fib = _f32(fibers).reshape(-1, 63)
    out = np.empty(fib.shape[0])
    _check(_load().oracle_lengths(_ptr(fib), fib.shape[0], _ptr(out)))
    return out


def grad(fibers, affine12, centroids, bundle_of, thresholds, mask=None, frozen=None,
         want_cen: bool = True, nthreads: int = 0):
    """Cost sum of d_ME(T f, assigned centroid) and its gradient w.r.t. the 12 affine values
    (M row-major, then t) and the centroid coordinates [M,21,3]. frozen = (cidx, orient,
    argmax) fixes the structure; otherwise the oracle labels the transformed fibers itself."""
    fib = _f32(fibers).reshape(-1, 63)
    cen = _f32(centroids).reshape(-1, 63)
    bo = np.ascontiguousarray(bundle_of, dtype=np.int32)
    thr = _f32(thresholds)
    aff = np.ascontiguousarray(affine12, dtype=np.float64)
    n, M = fib.shape[0], cen.shape[0]
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    if frozen is not None:
        fc, fo, fa = (np.ascontiguousarray(frozen[0], np.int32),
                      np.ascontiguousarray(frozen[1], np.uint8),
                      np.ascontiguousarray(frozen[2], np.int32))
    else:
        fc = fo = fa = None
    cost = np.zeros(1)
    ga = np.zeros(12)
    gc = np.zeros((M, 21, 3)) if want_cen else None
    out = dict(cidx=np.empty(n, np.int32), orient=np.empty(n, np.uint8),
               argmax=np.empty(n, np.int32), gap=np.empty(n))
    _check(_load().oracle_grad(_ptr(fib), n, _ptr(aff), _ptr(cen), _ptr(bo), M, _ptr(thr),
                               thr.shape[0], _ptr(m), _ptr(fc), _ptr(fo), _ptr(fa), _ptr(cost),
                               _ptr(ga), _ptr(gc), _ptr(out["cidx"]), _ptr(out["orient"]),
                               _ptr(out["argmax"]), _ptr(out["gap"]), nthreads))
    out.update(cost=float(cost[0]), grad_affine=ga, grad_centroids=gc)
    return out
