"""GPU parity of seg_apply_affine / seg_grad and the autograd wrapper against the FP64 oracle.

Both sides differentiate the same branch of the piecewise-smooth cost: the structure (centroid,
orientation) comes from the GPU forward pass, the oracle supplies the FP64 argmax point, and
fibers whose structure is not decidable in FP64 (a label that differs from the oracle's, which
must then be a near-tie; an argmax or orientation margin below 1e-3 mm) are left out of both
sums.

Tolerances, derived from the FP32 arithmetic of the per-fiber terms (seg_grad_terms.cuh): the
residual r at the argmax point is recovered to within half an FP32 ulp by error-free
transformations, |r| has at most 1.5 ulp of relative error (a fused sum of three squares and a
correctly rounded square root), u = r / |r| at most 2.5 ulp, and the product u_r x_c 3 ulp. With
a factor 2 of headroom every term is within EPS_TERM = 8 * 2^-24 of its own magnitude, and the
FP64 sum over fibers adds nothing at that scale. So
    |dC/dA_rc - oracle| <= EPS_TERM * sum_f |x_f,c|     (x at the argmax point),
    |dC/dt_r  - oracle| <= EPS_TERM * n_used,
    |C - oracle|        <= EPS_TERM * C,
each on top of rtol 1e-4. The centroid gradient is summed in 64-bit fixed point (2^-36 per
term) and rounded to FP32 once: per coordinate it is within EPS_TERM * (terms) + 2^-37 *
(terms) + 2^-24 |value|, and within 1e-4 absolute everywhere.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_11494_gb300 import autograd, binding, synth

pytestmark = pytest.mark.gpu

EPS_TERM = 8.0 * 2.0 ** -24


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    return torch.device("cuda:0")


def affine_np(fib, aff):
    A = np.asarray(aff[:9], np.float64).reshape(3, 3)
    t = np.asarray(aff[9:], np.float64)
    return (fib.astype(np.float64) @ A.T + t).astype(np.float32)


def make_at(a, dev, thr=None):
    return binding.Atlas(torch.as_tensor(a.centroids, device=dev),
                         torch.as_tensor(a.bundle_of, device=dev),
                         torch.as_tensor(a.thresholds if thr is None else thr, device=dev))


def gpu_forward(at, f, aff, mode="plain"):
    """seg_apply_affine + seg_label on the device: (cidx, orient) tensors."""
    y = binding.seg_apply_affine(f, aff)
    n = f.shape[0]
    lab = torch.empty(n, dtype=torch.int32, device=f.device)
    cidx = torch.empty(n, dtype=torch.int32, device=f.device)
    orient = torch.empty(n, dtype=torch.uint8, device=f.device)
    binding.seg_label(at, y, mode, lab, None, cidx, orient)
    binding.seg_sync_status(at)
    return cidx, orient


def gpu_grad(at, f, aff, cidx, orient, M):
    dev = f.device
    ga = torch.full((12,), np.nan, dtype=torch.float64, device=dev)
    gc = torch.full((M, 21, 3), np.nan, dtype=torch.float32, device=dev)
    cost = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    binding.seg_grad(at, f, aff, cidx, orient, ga, gc, cost)
    binding.seg_sync_status(at)
    return ga.cpu().numpy(), gc.cpu().numpy(), float(cost.item())


def decidable_structure(a, fib, aff, cidx, orient, min_gap=1e-3):
    """Fibers whose GPU structure equals the FP64 one with margins above min_gap, and the FP64
    argmax. Fibers labelled differently from the oracle must be near-ties."""
    y = affine_np(fib, aff)
    ref = oracle.label(y, a.centroids, a.bundle_of, a.thresholds, "cascade")
    diff = np.nonzero(ref["cidx"] != cidx)[0]
    if diff.size:
        tie = oracle.near_tie(y[diff], a.centroids, a.bundle_of, a.thresholds,
                              ref["labels"][diff], ref["dist"][diff])
        assert tie.all(), f"{int((tie == 0).sum())} decidable structure mismatches"
    same = (ref["cidx"] == cidx) & ((cidx < 0) | (ref["orient"] == orient))
    og = oracle.grad(fib, aff, a.centroids, a.bundle_of, a.thresholds,
                     frozen=(np.where(same, cidx, -1), orient, ref["argmax"]), want_cen=False)
    keep = same & (cidx >= 0) & (og["gap"] > min_gap)
    return keep, ref["argmax"], int(diff.size)


def check_against_oracle(a, fib, aff, ga, gc, cost, cidx, orient, argmax, keep):
    og = oracle.grad(fib, aff, a.centroids, a.bundle_of, a.thresholds, mask=keep,
                     frozen=(np.where(keep, cidx, -1), orient, argmax))
    idx = np.nonzero(keep)[0]
    xs = fib[idx, argmax[idx]].astype(np.float64)            # [n_used, 3]
    sx = np.abs(xs).sum(axis=0)                               # sum_f |x_f,c|
    atol_a = np.concatenate([np.tile(EPS_TERM * sx, 3), np.full(3, EPS_TERM * idx.size)])
    assert cost == pytest.approx(og["cost"], rel=max(1e-6, EPS_TERM))
    err = np.abs(ga - og["grad_affine"])
    # the derived bound alone (tighter than rtol 1e-4 on every entry of these workloads)
    assert np.all(err <= atol_a), (err, atol_a)
    assert np.all(err <= atol_a + 1e-4 * np.abs(og["grad_affine"]))
    # centroid gradient: count the terms of every coordinate
    pi = np.where(orient[idx] == 1, 20 - argmax[idx], argmax[idx])
    cnt = np.zeros((a.M, 21), np.int64)
    np.add.at(cnt, (cidx[idx], pi), 1)
    cnt = np.repeat(cnt[:, :, None], 3, axis=2)
    gref = og["grad_centroids"]
    bound = cnt * (EPS_TERM + 2.0 ** -37) + 2.0 ** -24 * np.abs(gref) + 1e-12
    gerr = np.abs(gc.astype(np.float64) - gref)
    assert np.all(gerr <= bound), float((gerr - bound).max())
    assert gerr.max() <= 1e-4
    return og


@pytest.fixture(scope="module")
def c5(dev):
    """1,000,000 fibers (bundle fraction 0.7) moved by a random affine (<= 5 deg, <= 4 mm,
    scale 0.95-1.05) against a 250-bundle x 20-centroid atlas."""
    atlas, fib = synth.workload("affine1m_atlas5k", device=dev)
    mis = synth.random_affine(5)
    return atlas, affine_np(fib, mis)


@pytest.mark.parametrize("aff_seed", [None, 21])
def test_grad_vs_oracle_full_size(dev, c5, aff_seed):
    """seg_grad at 1,000,000 fibers x 5,000 centroids against the FP64 analytic gradient."""
    a, fib = c5
    aff = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float64) if aff_seed is None \
        else synth.random_affine(aff_seed, max_deg=2.0, max_t=1.0, s_lo=0.99, s_hi=1.01)
    at = make_at(a, dev)
    f = torch.as_tensor(fib, device=dev)
    cidx_t, orient_t = gpu_forward(at, f, aff)
    cidx, orient = cidx_t.cpu().numpy(), orient_t.cpu().numpy()
    keep, argmax, ndiff = decidable_structure(a, fib, aff, cidx, orient)
    assert keep.sum() > 0.5 * len(fib)
    cidx_t[torch.as_tensor(~keep, device=dev)] = -1    # the same fibers on both sides
    ga, gc, cost = gpu_grad(at, f, aff, cidx_t, orient_t, a.M)
    check_against_oracle(a, fib, aff, ga, gc, cost, cidx, orient, argmax, keep)
    print(f"\nC5 gradient: {int(keep.sum())} of {len(fib)} fibers used, {ndiff} near-tie labels")


def test_grad_vs_central_differences_full_size(dev, c5):
    """The adjoint against central differences of the GPU's own cost (seg_grad's C) with the
    structure held, h = 1e-3 on each of the 12 affine entries, Richardson-extrapolated with
    h / 2 (so the O(h^2) truncation of the A entries, whose points sit ~100 mm from the origin,
    drops to O(h^4)). Fibers whose argmax and orientation margins exceed 0.5 mm are used: a step
    of 1e-3 moves a point by at most ~0.1 mm, so no argmax or orientation switches."""
    a, fib = c5
    aff = synth.random_affine(23, max_deg=2.0, max_t=1.0, s_lo=0.99, s_hi=1.01)
    at = make_at(a, dev)
    f = torch.as_tensor(fib, device=dev)
    cidx_t, orient_t = gpu_forward(at, f, aff)
    cidx, orient = cidx_t.cpu().numpy(), orient_t.cpu().numpy()
    keep, _, _ = decidable_structure(a, fib, aff, cidx, orient, min_gap=0.5)
    cidx_t[torch.as_tensor(~keep, device=dev)] = -1
    ga, _, _ = gpu_grad(at, f, aff, cidx_t, orient_t, a.M)

    def fd(k, h):
        e = np.zeros(12)
        e[k] = h
        _, _, cp = gpu_grad(at, f, aff + e, cidx_t, orient_t, a.M)
        _, _, cm = gpu_grad(at, f, aff - e, cidx_t, orient_t, a.M)
        return (cp - cm) / (2 * h)

    h = 1e-3
    rich = np.array([(4 * fd(k, h / 2) - fd(k, h)) / 3 for k in range(12)])
    # each fiber's distance carries <= 1.5 FP32 ulp of rounding, independent across fibers:
    # 6 sigma of that random walk over the used fibers, through the extrapolation (x 3)
    nu = int(keep.sum())
    noise = 3 * 6 * np.sqrt(2 * nu) * 1.5 * 2.0 ** -24 * 8.0 / (2 * (h / 2))
    err = np.abs(ga - rich)
    assert np.all(err <= 1e-4 * np.abs(ga) + noise), (err, noise, ga)


def test_apply_affine_matches_fp64(dev):
    a = synth.make_atlas(40, seed=1005)
    fib = synth.make_subject(a, 4000, 0.7, seed=5)
    aff = synth.random_affine(11)
    y = binding.seg_apply_affine(torch.as_tensor(fib, device=dev), aff).cpu().numpy()
    ref = fib.astype(np.float64) @ aff[:9].reshape(3, 3).T + aff[9:]
    assert np.abs(y - ref).max() < 1e-4
    # in place
    f = torch.as_tensor(fib, device=dev)
    binding.seg_apply_affine(f, aff, out=f)
    assert np.array_equal(f.cpu().numpy(), y)


@pytest.fixture(scope="module")
def case():
    a = synth.make_atlas(40, seed=1005)
    fib = synth.make_subject(a, 4000, 0.7, seed=5)
    mis = synth.random_affine(5)
    return a, affine_np(fib, mis)


def test_grad_small_case_vs_oracle(dev, case):
    """4,000 fibers x 800 centroids, the same bounds as the full-size case."""
    a, fib = case
    aff = synth.random_affine(21, max_deg=2.0, max_t=1.0, s_lo=0.99, s_hi=1.01)
    at = make_at(a, dev)
    f = torch.as_tensor(fib, device=dev)
    cidx_t, orient_t = gpu_forward(at, f, aff)
    cidx, orient = cidx_t.cpu().numpy(), orient_t.cpu().numpy()
    keep, argmax, _ = decidable_structure(a, fib, aff, cidx, orient)
    assert keep.sum() > 1000
    cidx_t[torch.as_tensor(~keep, device=dev)] = -1
    ga, gc, cost = gpu_grad(at, f, aff, cidx_t, orient_t, a.M)
    check_against_oracle(a, fib, aff, ga, gc, cost, cidx, orient, argmax, keep)


def test_grad_translation_closed_form(dev):
    t = np.arange(21, dtype=np.float32)
    fib = np.stack([t, 0 * t, 0 * t], axis=1)[None]
    cen = fib.copy()
    cen[0, 13] += np.array([1.0, -2.0, 2.0], np.float32)
    at = binding.Atlas(torch.as_tensor(cen, device=dev), torch.zeros(1, dtype=torch.int32,
                                                                     device=dev),
                       torch.full((1,), 10.0, device=dev))
    aff = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float64)
    f = torch.as_tensor(fib, device=dev)
    cidx, orient = gpu_forward(at, f, aff)
    ga, gc, cost = gpu_grad(at, f, aff, cidx, orient, 1)
    u = -np.array([1.0, -2.0, 2.0]) / 3.0
    assert cost == pytest.approx(3.0, abs=1e-6)
    np.testing.assert_allclose(ga[9:], u, atol=1e-6)
    np.testing.assert_allclose(ga[:9].reshape(3, 3), np.outer(u, fib[0, 13]), atol=1e-5)
    ref = np.zeros((1, 21, 3))
    ref[0, 13] = -u
    np.testing.assert_allclose(gc, ref, atol=1e-6)


def test_grad_deterministic_and_unlabelled(dev, case):
    a, fib = case
    aff = synth.random_affine(3, max_deg=1.0, max_t=0.5, s_lo=0.995, s_hi=1.005)
    at = make_at(a, dev)
    f = torch.as_tensor(fib, device=dev)
    cidx, orient = gpu_forward(at, f, aff)
    r1 = gpu_grad(at, f, aff, cidx, orient, a.M)
    r2 = gpu_grad(at, f, aff, cidx, orient, a.M)
    # FP64 sums in a fixed order and the centroid gradient in integer fixed point: bit-identical
    assert np.array_equal(r1[0], r2[0]) and r1[2] == r2[2] and np.array_equal(r1[1], r2[1])
    # nothing passes: zero cost and gradient
    at0 = make_at(a, dev, thr=np.full(a.B, 1e-6, np.float32))
    cidx, orient = gpu_forward(at0, f, aff)
    ga, gc, cost = gpu_grad(at0, f, aff, cidx, orient, a.M)
    assert np.all(cidx.cpu().numpy() == -1) and cost == 0.0 and not ga.any() and not gc.any()


def test_autograd_function(dev, case):
    """SegDME: forward = seg_apply_affine + seg_label + seg_grad's cost, backward = the saved
    gradient times the incoming one; compared with the oracle on the fibers whose structure is
    decidable (the others are dropped before the call)."""
    a, fib = case
    aff0 = synth.random_affine(4, max_deg=1.0, max_t=0.5, s_lo=0.995, s_hi=1.005)
    at = make_at(a, dev)
    f = torch.as_tensor(fib, device=dev)
    cidx_t, orient_t = gpu_forward(at, f, aff0)
    cidx, orient = cidx_t.cpu().numpy(), orient_t.cpu().numpy()
    keep, argmax, _ = decidable_structure(a, fib, aff0, cidx, orient)
    sub = torch.as_tensor(np.ascontiguousarray(fib[keep]), device=dev)
    cen = torch.as_tensor(a.centroids, device=dev).requires_grad_(True)
    aff = torch.tensor(aff0, dtype=torch.float64, requires_grad=True)
    cost = autograd.seg_cost(sub, aff, cen, at)
    (2.0 * cost).backward()
    ones = np.ones(int(keep.sum()), bool)
    og = oracle.grad(sub.cpu().numpy(), aff0, a.centroids, a.bundle_of, a.thresholds,
                     mask=ones, frozen=(cidx[keep], orient[keep], argmax[keep]))
    assert float(cost.detach()) == pytest.approx(og["cost"], rel=1e-6)
    xs = fib[keep][np.arange(keep.sum()), argmax[keep]].astype(np.float64)
    atol = 2 * np.concatenate([np.tile(EPS_TERM * np.abs(xs).sum(axis=0), 3),
                               np.full(3, EPS_TERM * keep.sum())])
    err = np.abs(aff.grad.numpy() - 2 * og["grad_affine"])
    assert np.all(err <= atol + 2e-4 * np.abs(og["grad_affine"])), (err, atol)
    g = cen.grad.cpu().numpy()
    assert np.abs(g - 2 * og["grad_centroids"]).max() <= 2e-4
