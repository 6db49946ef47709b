"""Soundness of the tensor-core prune on the GPU's own output (seg_gemm_screen_bits).

The GEMM modes keep a (fiber, centroid, orientation) pair for the exact test when the
BF16/TF32 lower bound with its rounding margin does not exceed the threshold, and skip whole
blocks whose centre-point boxes are out of reach (SEG_MODE_PLAIN_CULLED keeps the pairs that
pass test1 in dot-product form, with its rounding slack, in the blocks it does not cull).
Labels only stay exact if no pair the FP32 exact test would accept is ever dropped. This test
reads the pairs the screen kept, straight from the kernel, and checks them against FP64 d_ME
from the oracle (Eq. 2): every pair whose FP64 distance in an orientation is within
theta (1 + 4e-6) must be kept (the FP32 exact test accepts d^2 <= theta^2 computed in FP32,
i.e. FP64 distances up to about theta (1 + 1e-6)).

Inputs: the 10,000 x 1,000 workload's atlas with 2,048 of its fibers, plus adversarial fibers
built to sit on the bound: a centroid moved rigidly by a vector of length theta (1 - 1e-6), so
that all 21 point distances are equal, the mean over points equals the maximum and the lower
bound is tight, in both orientations and placed across the whole atlas (large coordinates give
the largest operand rounding).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_11494_gb300 import binding, synth

pytestmark = pytest.mark.gpu

GEMM_MODES = ["gemm_bf16", "gemm_tf32", "gemm_inv_bf16", "gemm_inv_tf32", "plain_culled"]


@pytest.fixture(scope="module")
def case():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    atlas, fib = synth.workload("subject10k_atlas1k")
    rng = np.random.default_rng(2024)
    pick = rng.choice(len(fib), size=2048, replace=False)
    base = fib[pick]
    # adversarial: rigid shifts of centroids by theta (1 - 1e-6), direct and reversed
    k = 1536
    ci = rng.integers(0, atlas.M, size=k)
    u = rng.normal(size=(k, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    th = atlas.thresholds[atlas.bundle_of[ci]].astype(np.float64)
    adv = atlas.centroids[ci].astype(np.float64) + (u * (th * (1 - 1e-6))[:, None])[:, None, :]
    adv[1::2] = adv[1::2, ::-1]
    fibers = np.ascontiguousarray(np.concatenate([base, adv.astype(np.float32)]))
    d, dd, dr = oracle.dme_matrix(fibers, atlas.centroids)
    thr = atlas.thresholds[atlas.bundle_of].astype(np.float64)[None, :] * (1 + 4e-6)
    at = binding.Atlas(torch.as_tensor(atlas.centroids, device=dev),
                       torch.as_tensor(atlas.bundle_of, device=dev),
                       torch.as_tensor(atlas.thresholds, device=dev))
    return dev, atlas, at, fibers, dd <= thr, dr <= thr


def unpack(bits, cols):
    b = bits.cpu().numpy().view(np.uint32)
    out = np.unpackbits(b.view(np.uint8), axis=1, bitorder="little")
    return out[:, :cols].astype(bool)


@pytest.mark.parametrize("mode", GEMM_MODES)
def test_screen_keeps_every_passing_pair(case, mode):
    dev, atlas, at, fib, pass_d, pass_r = case
    bits = binding.seg_gemm_screen_bits(at, torch.as_tensor(fib, device=dev), mode)
    binding.seg_sync_status(at)
    st = binding.seg_gemm_stats(at)
    assert st["overflow_fibers"] == 0
    M = atlas.M
    if "inv" in mode or mode == "plain_culled":
        kept = unpack(bits, M)
        need = pass_d | pass_r
    else:
        kb = unpack(bits, 2 * M)
        kept_d, kept_r = kb[:, 0::2], kb[:, 1::2]
        need = None
        miss_d = pass_d & ~kept_d
        miss_r = pass_r & ~kept_r
        assert not miss_d.any() and not miss_r.any(), (
            f"{int(miss_d.sum())} direct and {int(miss_r.sum())} reversed passing pairs dropped")
        kept = kept_d | kept_r
        need = pass_d | pass_r
    missing = need & ~kept
    assert not missing.any(), f"{int(missing.sum())} passing pairs dropped by the screen"
    # the adversarial fibers really test the bound: each passes its own centroid
    assert need[2048:].any(axis=1).mean() > 0.9
    # and the screen still prunes: most kept pairs are not passing ones
    frac = kept.sum() / kept.size
    assert frac < (0.2 if mode == "plain_culled" else 0.05)
    print(f"\n{mode}: {int(need.sum())} passing pairs all kept; {int(kept.sum())} kept of "
          f"{kept.size} ({100 * frac:.2f}%)")


def test_screen_bits_rejects_bad_arguments(case):
    dev, atlas, at, fib, _, _ = case
    f = torch.as_tensor(fib[:10], device=dev)
    with pytest.raises(binding.SegError):
        binding.seg_gemm_screen_bits(at, f, "plain")
    with pytest.raises(binding.SegError):  # one kernel: no separate screen to read
        binding.seg_gemm_screen_bits(at, f, "culled_fused")
    bits = torch.empty((10, 1), dtype=torch.int32, device=dev)
    rc = binding.lib().seg_gemm_screen_bits(at.handle, f.data_ptr(), 10, 1, bits.data_ptr(), 1,
                                            None)
    assert rc == 1 and b"words_per_fiber" in binding.lib().seg_last_error()
