"""Affine refinement driven by seg_grad (seg_refine_affine): a subject moved by a random affine
(<= 5 degrees, <= 4 mm, scale 0.95-1.05) is brought back onto the atlas from the identity. The
cost J (sum of d_ME over labelled fibers + the largest threshold per unlabelled fiber) must
fall, the recovered affine composed with the misalignment must move points by well under the
misalignment, and the J the library reports at its answer must equal the FP64 oracle's J
there (labels from the oracle's cascade on the transformed fibers)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_11494_gb300 import binding, synth

pytestmark = pytest.mark.gpu

IDENTITY = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float64)


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    return torch.device("cuda:0")


def affine_np(x, aff):
    A = np.asarray(aff[:9], np.float64).reshape(3, 3)
    return x.astype(np.float64) @ A.T + np.asarray(aff[9:], np.float64)


def oracle_cost(atlas, fib, aff):
    y = affine_np(fib, aff).astype(np.float32)
    r = oracle.label(y, atlas.centroids, atlas.bundle_of, atlas.thresholds, "cascade")
    lab = r["labels"] >= 0
    return r["dist"][lab].sum() + float(atlas.thresholds.max()) * (~lab).sum(), int(lab.sum())


@pytest.mark.parametrize("mode", ["plain", "gemm_bf16"])
def test_refine_recovers_misalignment(dev, mode):
    atlas, fib = synth.workload("affine1m_atlas5k", n=100_000)
    mis = synth.random_affine(5)
    moved = affine_np(fib, mis).astype(np.float32)
    at = binding.Atlas(torch.as_tensor(atlas.centroids, device=dev),
                       torch.as_tensor(atlas.bundle_of, device=dev),
                       torch.as_tensor(atlas.thresholds, device=dev))
    f = torch.as_tensor(moved, device=dev)
    aff, cost = binding.seg_refine_affine(at, f, IDENTITY, mode, iters=80, step_mm=0.5)
    j0, lab0 = oracle_cost(atlas, moved, IDENTITY)
    j1, lab1 = oracle_cost(atlas, moved, aff)
    j_al, lab_al = oracle_cost(atlas, fib, IDENTITY)  # the subject before the misalignment
    # residual motion of the composition (refined after misalignment) on the subject's points
    pts = fib.reshape(-1, 3)
    comp = affine_np(affine_np(pts, mis), aff)
    rms = float(np.sqrt(((comp - pts) ** 2).sum(axis=1).mean()))
    rms0 = float(np.sqrt(((affine_np(pts, mis) - pts) ** 2).sum(axis=1).mean()))
    print(f"\n{mode}: J {cost[0]:.4g} -> {cost.min():.4g} (aligned {j_al:.4g}); labelled "
          f"{lab0} -> {lab1} (aligned {lab_al}); residual RMS motion {rms0:.3f} -> {rms:.3f} mm")
    assert cost[0] == pytest.approx(j0, rel=1e-4)
    assert cost.min() == pytest.approx(j1, rel=1e-4)   # the returned affine is the best one
    # back to (within 1% of) the cost and labels of the subject before it was moved
    assert j1 <= 1.01 * j_al and lab1 >= 0.99 * lab_al and j1 < j0
    assert rms < 0.25 * rms0
