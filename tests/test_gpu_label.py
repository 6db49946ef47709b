"""GPU parity of seg_label (C ABI through the ctypes binding) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from paper_1912_11494_gb300 import binding, synth
import oracle
from tests import parity

pytestmark = pytest.mark.gpu

MODES = ["plain", "gemm_bf16", "gemm_tf32", "gemm_inv_bf16", "gemm_inv_tf32", "plain_culled",
         "culled_fused"]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1912_11494_gb300 import build
    build.build()
    return torch.device("cuda:0")


def make_atlas(cen, bo, thr, dev):
    return binding.Atlas(torch.as_tensor(np.ascontiguousarray(cen, np.float32), device=dev),
                         torch.as_tensor(np.ascontiguousarray(bo, np.int32), device=dev),
                         torch.as_tensor(np.ascontiguousarray(thr, np.float32), device=dev))


def run(atlas, fib, dev, mode):
    f = torch.as_tensor(np.ascontiguousarray(fib, np.float32), device=dev)
    lab, dist, cidx, orient = binding.label(atlas, f, mode)
    binding.seg_sync_status(atlas)
    return lab.cpu().numpy(), dist.cpu().numpy(), cidx.cpu().numpy(), orient.cpu().numpy()


@pytest.mark.parametrize("mode", MODES)
def test_small_workload_parity(dev, small_workload, mode):
    atlas_np, fib = small_workload
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    lab, dist, cidx, orient = run(at, fib, dev, mode)
    res = parity.compare(fib, atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, lab,
                         dist, cidx, orient)
    assert res["labelled"] > 0.5 * len(fib)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,M", [(1, 1), (31, 20), (32, 257), (33, 20), (1000, 257),
                                 (129, 1), (300, 513)])
def test_ragged_shapes(dev, n, M, mode):
    rng = np.random.default_rng(n * 1000 + M)
    nb = max(1, M // 20)
    cen = synth.make_atlas(nb, per_bundle=M // nb + 1, seed=6000 + M).centroids[:M]
    bo = (np.arange(M) % nb).astype(np.int32)
    rng.shuffle(bo)  # bundles interleaved in the caller's order
    thr = rng.uniform(5, 8, size=nb).astype(np.float32)
    src = cen[rng.integers(0, M, size=n)] + rng.normal(0, 1.5, size=(n, 21, 3))
    src[::2] = src[::2, ::-1]
    fib = src.astype(np.float32)
    at = make_atlas(cen, bo, thr, dev)
    lab, dist, cidx, orient = run(at, fib, dev, mode)
    parity.compare(fib, cen, bo, thr, lab, dist, cidx, orient)


@pytest.mark.parametrize("mode", MODES)
def test_degenerate_cases(dev, mode):
    a = synth.make_atlas(10, per_bundle=5, seed=77)
    cen, bo = a.centroids, a.bundle_of
    # fibers exactly on centroids, reversed copies, a non-finite fiber, a far fiber
    fib = np.concatenate([cen[:7], cen[7:14, ::-1], cen[:2] + 500.0]).astype(np.float32)
    fib[3, 5, 1] = np.nan
    fib[4, 0, 0] = np.inf
    for thr in (a.thresholds, np.full(10, 1e-3, np.float32), np.full(10, 1e4, np.float32)):
        at = make_atlas(cen, bo, thr, dev)
        lab, dist, cidx, orient = run(at, fib, dev, mode)
        parity.compare(fib, cen, bo, thr, lab, dist, cidx, orient)
        assert lab[3] == -1 and np.isnan(dist[3]) and lab[4] == -1
        assert dist[0] == 0.0 and dist[8] == 0.0 and orient[8] == 1
    # every fiber far from everything: all unlabelled
    at = make_atlas(cen, bo, a.thresholds, dev)
    lab, dist, _, _ = run(at, fib[-2:], dev, mode)
    assert np.all(lab == -1) and np.all(np.isinf(dist))


@pytest.mark.parametrize("mode", MODES)
def test_exact_ties_lowest_bundle_then_centroid(dev, mode):
    t = np.arange(21, dtype=np.float32)
    base = np.stack([t, 0 * t, 0 * t], axis=1)
    offs = [(0, 0, 2), (0, 2, 0), (0, -2, 0), (0, 0, -2), (2, 0, 0)]  # all exactly 2
    cen = np.stack([base + np.array(o, np.float32) for o in offs])
    bo = np.array([3, 1, 1, 2, 0], np.int32)  # every centroid at distance 2
    thr = np.full(4, 5.0, np.float32)
    at = make_atlas(cen, bo, thr, dev)
    lab, dist, cidx, orient = run(at, base[None].repeat(40, 0), dev, mode)
    assert np.all(lab == 0) and np.all(cidx == 4) and np.all(dist == 2.0)
    bo2 = np.array([3, 1, 1, 2, 3], np.int32)
    at = make_atlas(cen, bo2, thr, dev)
    lab, dist, cidx, orient = run(at, base[None].repeat(40, 0), dev, mode)
    assert np.all(lab == 1) and np.all(cidx == 1)


def test_empty_input(dev):
    a = synth.make_atlas(3, per_bundle=2, seed=1)
    at = make_atlas(a.centroids, a.bundle_of, a.thresholds, dev)
    binding.seg_label(at, None, "plain", None, n=0)
    binding.seg_sync_status(at)


def test_invalid_atlas_rejected(dev):
    a = synth.make_atlas(3, per_bundle=2, seed=1)
    bad = a.bundle_of.copy()
    bad[0] = 7
    with pytest.raises(binding.SegError):
        make_atlas(a.centroids, bad, a.thresholds, dev)
    thr = a.thresholds.copy()
    thr[1] = -1
    with pytest.raises(binding.SegError):
        make_atlas(a.centroids, a.bundle_of, thr, dev)
    cen = a.centroids.copy()
    cen[2, 3, 1] = np.nan
    with pytest.raises(binding.SegError):
        make_atlas(cen, a.bundle_of, a.thresholds, dev)


@pytest.fixture(scope="module")
def full_size():
    return synth.workload("subject4145k_atlas10k", device="cuda")


@pytest.fixture(scope="module")
def full_size_ref(full_size):
    """The oracle's cascade over all 4,145,000 fibers (about 7 s on 16 host cores)."""
    atlas_np, fib = full_size
    return oracle.label(fib, atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds,
                        "cascade")


@pytest.mark.parametrize("mode", MODES)
def test_full_size_parity_every_fiber(dev, mode, full_size, full_size_ref):
    """4,145,000 fibers x 10,000 centroids labelled in one call (the benchmark's launch), every
    fiber compared with the FP64 oracle: labels identical wherever decidable, distances within
    1e-3 mm, the chosen centroid's own distance and orientation checked; near-ties counted."""
    atlas_np, fib = full_size
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    lab, dist, cidx, orient = run(at, fib, dev, mode)
    res = parity.compare_all(fib, atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds,
                             lab, dist, cidx, orient, ref=full_size_ref,
                             count_ties=(mode == "plain"))
    frac = res["labelled"] / res["n"]
    assert 0.6 < frac < 0.9
    print(f"\n{mode}: {res['n']} fibers, {res['labelled']} labelled, {res['mismatches']} label "
          f"differences from the oracle (all near-ties)"
          + (f", {res['near_ties']} near-ties in all" if res["near_ties"] is not None else ""))


@pytest.mark.parametrize("mode", ["gemm_bf16", "gemm_tf32", "gemm_inv_bf16", "gemm_inv_tf32",
                                  "plain_culled", "culled_fused"])
def test_gemm_equals_plain_everywhere(dev, mode, small_workload, full_size):
    """The prune is conservative and survivors go through the same FP32 exact test, so the GEMM
    modes reproduce the plain kernel bit for bit on every fiber, not only the decidable ones."""
    for atlas_np, fib in (small_workload, full_size):
        at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
        ref = run(at, fib, dev, "plain")
        got = run(at, fib, dev, mode)
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)
        st = binding.seg_gemm_stats(at)
        cols = atlas_np.M if ("inv" in mode or "culled" in mode) else 2 * atlas_np.M
        assert st["pairs"] == len(fib) * cols
        # own bundle alone is 2% at M=1,000; test1 alone keeps more than the GEMM bounds
        assert 0 < st["survivors"] < (0.2 if "culled" in mode else 0.05) * st["pairs"]
        assert st["overflow_fibers"] == 0
        # every listed pair runs test1 at least; the culled blocks are never computed
        assert st["point_distances"] >= st["survivors"]
        assert 0 < st["screened"] <= st["pairs"] + 128 * 256 * (len(fib) // 128 + 1)


@pytest.mark.parametrize("n", [20_000, 300_000, 1_000_000, 2_500_000])
def test_no_survivor_overflow_at_any_size(dev, full_size, n):
    """The default survivor list holds every record at any fiber count (a fiber whose records
    do not fit is still labelled exactly, by a slow rescan, so only the statistic shows it)."""
    atlas_np, fib = full_size
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    for mode in ("plain_culled", "gemm_bf16", "gemm_inv_tf32"):
        run(at, fib[:n], dev, mode)
        assert binding.seg_gemm_stats(at)["overflow_fibers"] == 0, mode


@pytest.mark.parametrize("mode", ["gemm_bf16", "gemm_inv_bf16", "gemm_inv_tf32", "plain_culled",
                                  "culled_fused"])
def test_gemm_locality_order_extremes(dev, mode):
    """The GEMM modes visit fibers in the order of their centre point's 2 mm cell. Centres far
    outside the cell grid (clamped to its border), thousands of fibers in one cell, and a NaN
    centre (sorted to cell 0) still give the plain kernel's results in the caller's order."""
    a = synth.make_atlas(30, per_bundle=20, seed=41)
    base = synth.make_subject(a, 3000, 0.8, seed=42)
    same = np.repeat(base[:1], 2500, axis=0) + np.random.default_rng(43).normal(
        0, 0.3, size=(2500, 21, 3)).astype(np.float32)           # one hot cell
    far = base[:700] + np.array([900.0, -1200.0, 3000.0], np.float32)  # outside the grid
    fib = np.concatenate([base, same, far]).astype(np.float32)
    fib[5, 10, 0] = np.nan                                        # NaN centre point
    fib = fib[np.random.default_rng(44).permutation(len(fib))]
    at = make_atlas(a.centroids, a.bundle_of, a.thresholds, dev)
    ref = run(at, fib, dev, "plain")
    got = run(at, fib, dev, mode)
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x, y)
    parity.compare(fib, a.centroids, a.bundle_of, a.thresholds, *got)


@pytest.mark.parametrize("mode", ["plain", "gemm_bf16", "gemm_inv_tf32"])
def test_fibers_at_any_4_byte_offset(dev, mode):
    """A fiber array starting 0, 4, 8 or 12 bytes past a 16-byte boundary (a view into a larger
    buffer) gives the same results, its first and last fibers included; a pointer off the
    4-byte grid is refused before any work."""
    import ctypes
    a = synth.make_atlas(25, per_bundle=20, seed=61)
    fib = synth.make_subject(a, 1537, 0.9, seed=62)
    fib[0] = a.centroids[3] + 0.5      # first and last fibers next to a centroid, so their
    fib[-1] = a.centroids[17][::-1]    # pairs reach the exact re-check
    at = make_atlas(a.centroids, a.bundle_of, a.thresholds, dev)
    ref = run(at, fib, dev, "plain")
    assert ref[0][0] >= 0 and ref[0][-1] >= 0
    n = len(fib)
    for off in range(4):
        buf = torch.zeros(n * 63 + 8, dtype=torch.float32, device=dev)
        buf[off:off + n * 63] = torch.as_tensor(fib.reshape(-1), device=dev)
        f = buf[off:off + n * 63].view(n, 21, 3)
        assert f.data_ptr() % 16 == 4 * off
        lab, dist, cidx, orient = binding.label(at, f, mode)
        binding.seg_sync_status(at)
        for x, y in zip(ref, (lab.cpu().numpy(), dist.cpu().numpy(), cidx.cpu().numpy(),
                              orient.cpu().numpy())):
            np.testing.assert_array_equal(x, y)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    rc = binding.lib().seg_label(at.handle, ctypes.c_void_p(buf.data_ptr() + 2), n,
                                 binding.MODES[mode], ctypes.c_void_p(lab.data_ptr()), None,
                                 None, None, None)
    assert rc == 1 and b"aligned" in binding.lib().seg_last_error()


@pytest.mark.parametrize("mode", ["plain", "gemm_bf16", "gemm_inv_tf32"])
def test_host_buffers_equal_device_call(dev, mode, full_size):
    """seg_label_host (chunked upload overlapping the labelling) returns seg_label's results,
    for 4 chunks (the full subject, pinned buffers), 2 chunks and 1 chunk (pageable buffers),
    and again on the same atlas after a smaller call (buffer reuse)."""
    atlas_np, fib = full_size
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    for n, pinned in ((len(fib), True), (700_000, False), (100_003, False), (len(fib), False)):
        f = fib[:n]
        ref_lab, ref_dist, _, _ = run(at, f, dev, mode)
        h_fib = torch.as_tensor(np.ascontiguousarray(f))
        h_lab = torch.full((n,), -7, dtype=torch.int32)
        h_dst = torch.full((n,), -7.0)
        if pinned:
            h_fib, h_lab, h_dst = h_fib.pin_memory(), h_lab.pin_memory(), h_dst.pin_memory()
        binding.seg_label_host(at, h_fib, mode, h_lab, h_dst)
        torch.cuda.synchronize()
        binding.seg_sync_status(at)
        np.testing.assert_array_equal(h_lab.numpy(), ref_lab)
        np.testing.assert_array_equal(h_dst.numpy(), ref_dist)


def test_host_calls_back_to_back(dev, full_size):
    """Consecutive seg_label_host calls with no synchronisation in between (each call's upload
    overlaps the previous call's labelling, on alternating device buffers) all return
    seg_label's results."""
    atlas_np, fib = full_size
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    parts = [fib[:1_500_000], fib[1_500_000:3_000_000], fib[3_000_000:], fib[:900_001]]
    outs = []
    for f in parts:
        h_fib = torch.as_tensor(np.ascontiguousarray(f)).pin_memory()
        h_lab = torch.full((len(f),), -7, dtype=torch.int32).pin_memory()
        h_dst = torch.full((len(f),), -7.0).pin_memory()
        binding.seg_label_host(at, h_fib, "gemm_bf16", h_lab, h_dst)
        outs.append((h_fib, h_lab, h_dst))
    torch.cuda.synchronize()
    binding.seg_sync_status(at)
    for f, (_, h_lab, h_dst) in zip(parts, outs):
        ref_lab, ref_dist, _, _ = run(at, f, dev, "gemm_bf16")
        np.testing.assert_array_equal(h_lab.numpy(), ref_lab)
        np.testing.assert_array_equal(h_dst.numpy(), ref_dist)


@pytest.mark.parametrize("mode", ["gemm_bf16", "gemm_inv_tf32", "plain_culled"])
def test_survivor_list_overflow_rescans_exactly(dev, mode):
    """A survivor list capped at a few records overflows on almost every fiber; those fibers are
    rescanned exactly against the whole atlas, and the results do not change."""
    a = synth.make_atlas(20, per_bundle=20, seed=51)
    fib = synth.make_subject(a, 3000, 0.8, seed=52)
    at = make_atlas(a.centroids, a.bundle_of, a.thresholds, dev)
    ref = run(at, fib, dev, "plain")
    for cap in (1, 7, 100):
        binding.seg_set_gemm_record_cap(at, cap)
        got = run(at, fib, dev, mode)
        st = binding.seg_gemm_stats(at)
        assert st["overflow_fibers"] > 0
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)
    binding.seg_set_gemm_record_cap(at, 0)
    run(at, fib, dev, mode)
    assert binding.seg_gemm_stats(at)["overflow_fibers"] == 0
    with pytest.raises(binding.SegError):
        binding.seg_set_gemm_record_cap(at, -1)


def test_gemm_column_limit(dev):
    """The GEMM modes take at most 131,072 operand columns: 66,000 centroids exceed it in the
    directional layout (2M columns) but not in the orientation-free one (M columns)."""
    a = synth.make_atlas(3300, per_bundle=20, seed=53)
    fib = synth.make_subject(a, 500, 0.8, seed=54)
    at = make_atlas(a.centroids, a.bundle_of, a.thresholds, dev)
    with pytest.raises(binding.SegError):
        run(at, fib, dev, "gemm_bf16")
    ref = run(at, fib, dev, "plain")
    for mode in ("gemm_inv_bf16", "plain_culled", "culled_fused"):
        got = run(at, fib, dev, mode)
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)


@pytest.fixture(scope="module")
def whole_brain():
    """A subject of 40,000 fibers against the atlas shaped like the paper's 62-bundle
    whole-brain atlas (44,345 centroids: 88,690 directional columns)."""
    return synth.workload("subject4145k_atlas44k", n=40_000)


@pytest.mark.parametrize("mode", MODES)
def test_whole_brain_atlas_parity(dev, mode, whole_brain):
    """Every mode on the 44,345-centroid atlas: bit-identical to the plain kernel, and every
    fiber against the oracle."""
    atlas_np, fib = whole_brain
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    got = run(at, fib, dev, mode)
    if mode != "plain":
        ref = run(at, fib, dev, "plain")
        for x, y in zip(ref, got):
            np.testing.assert_array_equal(x, y)
        st = binding.seg_gemm_stats(at)
        assert st["overflow_fibers"] == 0
    else:
        res = parity.compare_all(fib, atlas_np.centroids, atlas_np.bundle_of,
                                 atlas_np.thresholds, *got)
        assert res["labelled"] > 0.5 * len(fib)
        print(f"\nwhole-brain atlas: {res['labelled']} of {res['n']} labelled, "
              f"{res['mismatches']} near-tie label differences, {res['near_ties']} near-ties")


def test_every_tile_shape_identical(dev, small_workload):
    """All tile-shape configurations of a mode compute the same labels, distances, centroids."""
    atlas_np, fib = small_workload
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    for mode in MODES:
        outs = []
        for cfg in range(binding.seg_num_configs(mode)):
            binding.seg_set_config(at, mode, cfg)
            assert binding.seg_get_config(at, mode) == cfg
            outs.append(run(at, fib, dev, mode))
        for o in outs[1:]:
            for x, y in zip(outs[0], o):
                np.testing.assert_array_equal(x, y)
    with pytest.raises(binding.SegError):
        binding.seg_set_config(at, "plain", binding.seg_num_configs("plain"))


@pytest.mark.parametrize("mode", MODES)
def test_every_pair_passes_overflowing_queues(dev, mode):
    """Thresholds so large that every (fiber, centroid) pair passes: the per-warp queues of
    test1 survivors overflow many times and must resume without losing or repeating work."""
    a = synth.make_atlas(20, per_bundle=20, seed=31)
    fib = synth.make_subject(a, 200, 0.5, seed=32)
    thr = np.full(20, 1e4, np.float32)
    at = make_atlas(a.centroids, a.bundle_of, thr, dev)
    for cfg in range(binding.seg_num_configs(mode)):
        binding.seg_set_config(at, mode, cfg)
        lab, dist, cidx, orient = run(at, fib, dev, mode)
        parity.compare(fib, a.centroids, a.bundle_of, thr, lab, dist, cidx, orient)
        assert np.all(lab >= 0)


def test_profile_and_tune(dev, small_workload, tmp_path):
    from paper_1912_11494_gb300 import tune
    atlas_np, fib = small_workload
    at = make_atlas(atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds, dev)
    f = torch.as_tensor(fib, device=dev)
    binding.seg_profile_enable(at, True)
    run(at, fib, dev, "plain")
    run(at, fib, dev, "gemm_bf16")
    assert binding.seg_profile_read(at, "plain")[0] == 1
    for k in ("gemm_sort", "gemm_prep", "gemm_screen", "gemm_exact", "gemm_finalize"):
        c, ms = binding.seg_profile_read(at, k)
        assert c == 1 and ms > 0
    binding.seg_profile_enable(at, False)
    assert binding.seg_profile_read(at, "plain") == (0, 0.0)
    with pytest.raises(binding.SegError):
        binding.seg_profile_read(at, "nope")
    path = str(tmp_path / "tune.json")
    r1 = tune.tune(at, f, "plain", path=path)
    assert not r1["cached"] and 0 <= r1["config"] < binding.seg_num_configs("plain")
    r2 = tune.tune(at, f, "plain", path=path)
    assert r2["cached"] and r2["config"] == r1["config"]
    assert binding.seg_get_config(at, "plain") == r1["config"]
