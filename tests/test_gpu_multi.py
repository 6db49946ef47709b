"""GPU multi-label output (seg_label_multi; Section 2.4, on classifying fibers): every
bundle a fiber passes, against the FP64 oracle. Bits are compared wherever the oracle calls
them decidable (the bundle's best centroid is not within 2e-3 mm of its threshold); the
closest-bundle labels equal seg_label's bit for bit, and every mode gives identical bits."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_11494_gb300 import binding, synth

pytestmark = pytest.mark.gpu

MODES = ["plain", "gemm_bf16", "gemm_tf32", "gemm_inv_bf16", "gemm_inv_tf32", "plain_culled",
         "culled_fused"]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    return torch.device("cuda:0")


def make_atlas(a, dev):
    return binding.Atlas(torch.as_tensor(a.centroids, device=dev),
                         torch.as_tensor(a.bundle_of, device=dev),
                         torch.as_tensor(a.thresholds, device=dev))


def multi(at, fib, dev, mode):
    bits, lab, dist = binding.label_multi(at, torch.as_tensor(fib, device=dev), mode)
    binding.seg_sync_status(at)
    return bits.cpu().numpy().view(np.uint32), lab.cpu().numpy(), dist.cpu().numpy()


def check(fib, a, bits, lab, cls):
    ref, amb = oracle.label_multi(fib, a.centroids, a.bundle_of, a.thresholds, cls)
    diff = (bits ^ ref) & ~amb
    assert not diff.any(), f"{int(np.unpackbits(diff.view(np.uint8)).sum())} bundle bits differ"
    # the closest bundle is always among the passing ones
    sel = np.nonzero(lab >= 0)[0]
    assert np.all((bits[sel, lab[sel] // 32] >> (lab[sel] % 32).astype(np.uint32)) & 1)
    return ref, amb


@pytest.fixture(scope="module")
def small():
    """10,000 fibers of the 500-bundle x 20-centroid workload with the thresholds doubled
    (10-16 mm), so that neighbouring bundles overlap and many fibers pass several of them."""
    a, fib = synth.workload("subject4145k_atlas10k", n=10_000)
    a = synth.Atlas(a.centroids, a.bundle_of, (a.thresholds * 2.0).astype(np.float32),
                    a.base_ctrl)
    return a, fib


@pytest.mark.parametrize("cls", ["eq2", "eq2_tn"])
@pytest.mark.parametrize("mode", MODES)
def test_multi_label_parity(dev, small, mode, cls):
    a, fib = small
    at = make_atlas(a, dev)
    binding.seg_set_classification(at, cls)
    bits, lab, dist = multi(at, fib, dev, mode)
    l1, d1, _, _ = binding.label(at, torch.as_tensor(fib, device=dev), mode)
    np.testing.assert_array_equal(lab, l1.cpu().numpy())
    np.testing.assert_array_equal(dist, d1.cpu().numpy())
    if mode == "plain":
        ref, amb = check(fib, a, bits, lab, cls)
        per = np.unpackbits(ref.view(np.uint8), axis=1).sum(axis=1)
        print(f"\n{cls}: bundles passed per fiber: mean {per.mean():.2f}, max {per.max()}, "
              f"{int((per > 1).sum())} of {len(fib)} fibers pass more than one")
        assert (per > 1).sum() > 300
    else:
        ref_bits, _, _ = multi(at, fib, dev, "plain")
        np.testing.assert_array_equal(bits, ref_bits)


def test_multi_label_hand_case(dev):
    """The oracle's pinned parallel-offset case on every mode."""
    t = np.arange(21, dtype=np.float64)
    line = np.stack([t, 0 * t, 0 * t], axis=1)
    offs = [(0, 0, 3.0), (0, 4.5, 0), (0, 0, -1.0), (0, -6.0, 0), (5.0, 0, 0)]
    cen = np.stack([line + np.array(o) for o in offs]).astype(np.float32)
    a = synth.Atlas(cen, np.arange(5, dtype=np.int32),
                    np.array([5.0, 4.0, 5.0, 7.0, 5.0], np.float32), None)
    fib = np.stack([line, line + [0, 0, 100.0]]).astype(np.float32)
    at = make_atlas(a, dev)
    for mode in MODES:
        bits, lab, _ = multi(at, fib, dev, mode)
        assert bits[0, 0] == (1 << 0) | (1 << 2) | (1 << 3) | (1 << 4), mode
        assert bits[1, 0] == 0 and lab[0] == 2 and lab[1] == -1


def test_multi_label_full_size(dev):
    """4,145,000 fibers: the tensor-core and culled modes give the plain kernel's bits on every
    fiber; 20,000 sampled fibers against the oracle."""
    a, fib = synth.workload("subject4145k_atlas10k", device="cuda")
    at = make_atlas(a, dev)
    ref = multi(at, fib, dev, "plain")
    for mode in ("gemm_bf16", "plain_culled", "culled_fused"):
        got = multi(at, fib, dev, mode)
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)
    idx = np.sort(np.random.default_rng(9).choice(len(fib), size=20_000, replace=False))
    check(fib[idx], a, ref[0][idx], ref[1][idx], "eq2")
