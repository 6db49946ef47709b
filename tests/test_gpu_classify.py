"""GPU parity of the paper-faithful classifications (seg_set_classification) against the FP64
oracle: Eq. 2 + the length term TN (Eq. 3, lazy), and the paper's new algorithm (direction
inferred from test2's end points, tests 3-4 in that orientation, + TN; Section 2.4).

The bars are those of the Eq. 2 path on the classification distance D: labels identical for
every fiber the oracle's near-tie flag (on D, including fibers whose inferred direction is
ambiguous) leaves decidable, D within 1e-3 mm, the chosen centroid's own FP64 D within 1e-3 mm,
every mode bit-identical to the plain kernel. The tests also count how many labels the
classification changes against exact Eq. 2.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_11494_gb300 import binding, synth

pytestmark = pytest.mark.gpu

MODES = ["plain", "gemm_bf16", "gemm_tf32", "gemm_inv_bf16", "gemm_inv_tf32", "plain_culled",
         "culled_fused"]
DIST_TOL = 1e-3


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    return torch.device("cuda:0")


def make_atlas(a, dev):
    return binding.Atlas(torch.as_tensor(np.ascontiguousarray(a.centroids, np.float32),
                                         device=dev),
                         torch.as_tensor(np.ascontiguousarray(a.bundle_of, np.int32), device=dev),
                         torch.as_tensor(np.ascontiguousarray(a.thresholds, np.float32),
                                         device=dev))


def run(at, fib, dev, mode):
    lab, dist, cidx, orient = binding.label(at, torch.as_tensor(fib, device=dev), mode)
    binding.seg_sync_status(at)
    return lab.cpu().numpy(), dist.cpu().numpy(), cidx.cpu().numpy(), orient.cpu().numpy()


def compare_cls(cls, fib, a, lab, dist, cidx, orient):
    ref = oracle.label_cls(fib, a.centroids, a.bundle_of, a.thresholds, cls)
    flag = oracle.near_tie_cls(fib, a.centroids, a.bundle_of, a.thresholds, cls,
                               ref["labels"], ref["dist"])
    bad = np.nonzero((flag == 0) & (lab != ref["labels"]))[0]
    assert bad.size == 0, f"{bad.size} decidable label mismatches, first {bad[:5]}"
    both = (lab >= 0) & (ref["labels"] >= 0) & (flag == 0)
    if both.any():
        assert np.abs(dist[both] - ref["dist"][both]).max() <= DIST_TOL
    assert np.all(np.isinf(dist[lab < 0]))
    # the chosen centroid's own D in FP64, in the reported orientation
    sel = np.nonzero((lab >= 0) & (flag == 0))[0]
    if sel.size:
        own = own_d(fib[sel], a, cidx[sel], cls, orient[sel])
        assert np.abs(own - dist[sel]).max() <= DIST_TOL
    return ref, flag


def own_d(fib, a, cidx, cls, orient):
    """FP64 D of each fiber against its own chosen centroid: d_ME (or, for the paper's
    algorithm, the reported orientation's maximum) plus TN from the FP64 lengths."""
    d, dd, dr = oracle.dme_pairs(fib, a.centroids, cidx)
    lf = oracle.lengths(fib)
    lc = oracle.lengths(a.centroids)[cidx]
    m = np.maximum(lf, lc)
    r = np.abs(lf - lc) / np.where(m > 0, m, 1.0)
    base = np.where(orient == 0, dd, dr) if cls == "paper" else d
    return base + (r + 1.0) ** 2 - 1.0


@pytest.fixture(scope="module")
def small():
    return synth.workload("subject10k_atlas1k")


@pytest.mark.parametrize("cls", ["eq2_tn", "paper"])
@pytest.mark.parametrize("mode", MODES)
def test_classification_parity(dev, small, cls, mode):
    a, fib = small
    at = make_atlas(a, dev)
    binding.seg_set_classification(at, cls)
    assert binding.seg_get_classification(at) == cls
    got = run(at, fib, dev, mode)
    if mode != "plain":
        ref = run(at, fib, dev, "plain")
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)
    else:
        ref_cls, flag = compare_cls(cls, fib, a, *got)
        eq2 = oracle.label(fib, a.centroids, a.bundle_of, a.thresholds)
        changed = int((ref_cls["labels"] != eq2["labels"]).sum())
        print(f"\n{cls}: {changed} of {len(fib)} labels differ from exact Eq. 2 "
              f"({int(flag.sum())} near-ties)")


def test_classification_hand_cases(dev):
    """The oracle's pinned worked examples on the GPU: TN decides a fiber that Eq. 2 accepts,
    and direction inference loses a fiber whose end points favour the wrong orientation."""
    t = np.arange(21, dtype=np.float64)
    line = np.stack([t, 0 * t, 0 * t], axis=1)
    fib = line[None].astype(np.float32)
    cen = (line * [1.1, 1.0, 1.0])[None].astype(np.float32)
    a = synth.Atlas(cen, np.zeros(1, np.int32), np.array([2.1], np.float32), None)
    at = make_atlas(a, dev)
    for cls, want in (("eq2", 0), ("eq2_tn", -1), ("paper", -1)):
        binding.seg_set_classification(at, cls)
        for mode in MODES:
            assert run(at, fib, dev, mode)[0][0] == want, (cls, mode)
    R = 5.0
    ang = 2 * np.pi * 0.95 * t / 20
    loop = np.stack([R * np.cos(ang), R * np.sin(ang), 0 * ang], axis=1)
    b = loop[::-1].copy()
    b[0] = loop[0] + [0, 0, 0.5]
    b[20] = loop[20] + [0, 0, 0.5]
    a = synth.Atlas(b[None].astype(np.float32), np.zeros(1, np.int32),
                    np.array([3.0], np.float32), None)
    at = make_atlas(a, dev)
    f = loop[None].astype(np.float32)
    for cls, want in (("eq2", 0), ("eq2_tn", 0), ("paper", -1)):
        binding.seg_set_classification(at, cls)
        for mode in MODES:
            lab, dist, cidx, orient = run(at, f, dev, mode)
            assert lab[0] == want, (cls, mode)
            if want == 0:
                assert orient[0] == 1


@pytest.fixture(scope="module")
def full_size():
    return synth.workload("subject4145k_atlas10k", device="cuda")


@pytest.mark.parametrize("cls", ["eq2_tn", "paper"])
def test_classification_full_size(dev, full_size, cls):
    """4,145,000 fibers: every mode bit-identical to the plain kernel under the classification,
    20,000 sampled fibers against the oracle, and the count of labels that differ from exact
    Eq. 2 over all fibers."""
    a, fib = full_size
    at = make_atlas(a, dev)
    eq2 = run(at, fib, dev, "plain")
    binding.seg_set_classification(at, cls)
    ref = run(at, fib, dev, "plain")
    for mode in ("gemm_bf16", "plain_culled", "culled_fused"):
        got = run(at, fib, dev, mode)
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)
    idx = np.sort(np.random.default_rng(7).choice(len(fib), size=20_000, replace=False))
    compare_cls(cls, fib[idx], a, *(x[idx] for x in ref))
    changed = int((ref[0] != eq2[0]).sum())
    print(f"\n{cls} at 4,145,000 fibers: {changed} labels differ from exact Eq. 2 "
          f"({100 * changed / len(fib):.3f}%)")
