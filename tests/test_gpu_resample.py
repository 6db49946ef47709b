"""GPU resampling of raw streamlines to 21 arc-length-equidistant points (seg_resample,
seg_label_streamlines; Section 2.3) against the FP64 oracle resampler.

Tolerance: the GPU keeps cumulative arc lengths in FP32 with a compensated running total, so a
target's arc length (k L / 20, itself an FP32 value) is off by a few FP32 ulps of the
streamline's length L, and each coordinate by about one ulp of its magnitude: every resampled
coordinate must be within max(1e-4 mm, 4 ulp(L)) of the oracle's (1e-4 mm for any streamline
shorter than about 500 mm; brain streamlines are at most a few hundred mm)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_11494_gb300 import binding, synth
from tests import parity

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    return torch.device("cuda:0")


def tolerance(pts, off):
    """Per streamline: max(TOL, 4 FP32 ulps of its length)."""
    seg = np.linalg.norm(np.diff(pts.astype(np.float64), axis=0), axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    L = cum[np.maximum(off[1:] - 1, off[:-1])] - cum[off[:-1]]
    return np.maximum(TOL, 4 * np.spacing(L.astype(np.float32)).astype(np.float64))


def gpu_resample(pts, off, dev):
    out = binding.seg_resample(torch.as_tensor(pts, device=dev), torch.as_tensor(off, device=dev))
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_resample_subject_streamlines(dev):
    """20,000 raw streamlines of the subject recipe (about 0.2 mm steps, uneven arc spacing,
    half of them reversed) against the oracle."""
    a = synth.make_atlas(50, seed=1001)
    pts, off = synth.make_streamlines(a, 20_000, 0.7, seed=3)
    got = gpu_resample(pts.numpy(), off.numpy(), dev)
    ref = oracle.resample(pts.numpy(), off.numpy())
    err = np.abs(got - ref).max()
    assert np.all(np.abs(got - ref).max(axis=(1, 2)) <= tolerance(pts.numpy(), off.numpy()))
    assert err <= TOL, err
    print(f"\n20,000 streamlines ({pts.shape[0]} points): max coordinate error {err:.2e} mm")


def test_resample_edge_cases(dev):
    """The oracle's pinned cases on the GPU (uneven straight line with a repeated vertex, 201
    equal chords of a circle, a single point, an empty streamline), plus a two-point streamline,
    streamlines of 5,000 and 20,000 points, all points equal, and an already equidistant fiber."""
    line = np.array([[0, 0, 0], [1, 0, 0], [5, 0, 0], [5, 0, 0], [20, 0, 0]], np.float32)
    ang = np.linspace(0.0, 1.5 * np.pi, 201)
    circ = np.stack([9 * np.cos(ang), 9 * np.sin(ang), 0 * ang], axis=1).astype(np.float32)
    single = np.array([[3, -2, 7]], np.float32)
    two = np.array([[1, 2, 3], [4, 6, 3]], np.float32)
    rng = np.random.default_rng(0)
    walk5k = np.cumsum(rng.normal(0, 0.2, size=(5000, 3)), axis=0).astype(np.float32) + 50
    walk20k = np.cumsum(rng.normal(0, 0.2, size=(20000, 3)), axis=0).astype(np.float32) - 60
    same = np.repeat(np.array([[7, 7, 7]], np.float32), 9, axis=0)
    t = np.arange(21, dtype=np.float32)
    eq = np.stack([2 * t, 0 * t, 0 * t], axis=1)
    parts = [line, circ, single, np.zeros((0, 3), np.float32), two, walk5k, walk20k, same, eq]
    off = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
    pts = np.concatenate(parts)
    got = gpu_resample(pts, off, dev)
    ref = oracle.resample(pts, off)
    assert np.isnan(got[3]).all() and np.isnan(ref[3]).all()
    keep = [0, 1, 2, 4, 5, 6, 7, 8]
    err = np.abs(got[keep] - ref[keep]).max(axis=(1, 2))
    tol = tolerance(pts, off)[keep]
    assert np.all(err <= tol), (err, tol)
    assert err[[0, 1, 2, 3, 6, 7]].max() <= TOL  # the streamlines shorter than 500 mm
    np.testing.assert_array_equal(got[2], np.repeat(single, 21, axis=0))
    np.testing.assert_array_equal(got[7], np.repeat(same[:1], 21, axis=0))
    np.testing.assert_allclose(got[8], eq, atol=1e-5)
    assert got[0, 20, 0] == 20.0 and got[0, 0, 0] == 0.0


@pytest.mark.parametrize("mode", ["plain", "gemm_bf16", "plain_culled", "culled_fused"])
def test_label_streamlines(dev, mode):
    """seg_label_streamlines equals seg_resample followed by seg_label, and its labels match the
    oracle's labelling of the same resampled fibers."""
    a = synth.make_atlas(50, seed=1001)
    pts, off = synth.make_streamlines(a, 10_000, 0.7, seed=1)
    at = binding.Atlas(torch.as_tensor(a.centroids, device=dev),
                       torch.as_tensor(a.bundle_of, device=dev),
                       torch.as_tensor(a.thresholds, device=dev))
    p, o = torch.as_tensor(pts, device=dev), torch.as_tensor(off, device=dev)
    got = [x.cpu().numpy() for x in binding.label_streamlines(at, p, o, mode)]
    binding.seg_sync_status(at)
    fib = binding.seg_resample(p, o)
    ref = [x.cpu().numpy() for x in binding.label(at, fib, mode)]
    binding.seg_sync_status(at)
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x, y)
    res = parity.compare_all(fib.cpu().numpy(), a.centroids, a.bundle_of, a.thresholds, *got)
    assert res["labelled"] > 0.5 * res["n"]
