"""GPU tests of seg_label_batch: many subjects of uneven size in one captured launch sequence
(a CUDA graph captured once per batch shape and replayed with a new work table, copied from
one of two pinned host buffers used by alternate calls)."""
import numpy as np
import pytest
import torch

from paper_1912_11494_gb300 import binding, synth
import oracle
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    a = synth.make_atlas(60, seed=1002)
    at = binding.Atlas(torch.as_tensor(a.centroids, device=dev),
                       torch.as_tensor(a.bundle_of, device=dev),
                       torch.as_tensor(a.thresholds, device=dev))
    return dev, a, at


def subjects(a, counts, seed0, dev):
    return [torch.as_tensor(synth.make_subject(a, max(n, 1), 0.75, seed0 + i)[:n], device=dev)
            for i, n in enumerate(counts)]


def single(at, f, mode):
    lab, dist, _, _ = binding.label(at, f, mode) if f.shape[0] else (
        torch.empty(0, dtype=torch.int32), torch.empty(0), None, None)
    return lab.cpu().numpy(), dist.cpu().numpy()


def batch(at, fibs, mode, with_dist=True):
    dev = fibs[0].device
    labs = [torch.full((f.shape[0],), -7, dtype=torch.int32, device=dev) for f in fibs]
    dists = [torch.full((f.shape[0],), -7.0, device=dev) for f in fibs] if with_dist else None
    binding.seg_label_batch(at, fibs, mode, labs, dists)
    binding.seg_sync_status(at)
    return ([l.cpu().numpy() for l in labs],
            [d.cpu().numpy() for d in dists] if with_dist else None)


@pytest.mark.parametrize("mode", ["plain", "gemm_bf16", "gemm_tf32", "gemm_inv_bf16",
                                  "plain_culled", "culled_fused"])
def test_batch_equals_single_calls(env, mode):
    dev, a, at = env
    fibs = subjects(a, [0, 1, 33, 1000, 5000, 257, 31], 100, dev)
    labs, dists = batch(at, fibs, mode)
    for f, l, d in zip(fibs, labs, dists):
        rl, rd = single(at, f, "plain")
        np.testing.assert_array_equal(l, rl)
        np.testing.assert_array_equal(d, rd)
    # oracle parity on one subject
    f = fibs[4].cpu().numpy()
    parity.compare(f, a.centroids, a.bundle_of, a.thresholds, labs[4], dists[4])


def test_graph_replay_and_recapture(env):
    dev, a, at = env
    for counts, seed in (([500, 2000, 17], 7), ([3000, 5, 999], 8), ([64, 64, 64, 64, 0], 9),
                         ([1200], 10)):
        fibs = subjects(a, counts, seed * 100, dev)
        labs, dists = batch(at, fibs, "plain")
        for f, l, d in zip(fibs, labs, dists):
            rl, rd = single(at, f, "plain")
            np.testing.assert_array_equal(l, rl)
            np.testing.assert_array_equal(d, rd)
    # labels only (no distance buffers)
    fibs = subjects(a, [700, 300], 77, dev)
    labs, _ = batch(at, fibs, "plain", with_dist=False)
    for f, l in zip(fibs, labs):
        np.testing.assert_array_equal(l, single(at, f, "plain")[0])


def test_every_tile_shape_in_batch(env):
    dev, a, at = env
    fibs = subjects(a, [900, 40, 2100], 500, dev)
    ref = [single(at, f, "plain") for f in fibs]
    for cfg in range(binding.seg_num_configs("plain")):
        binding.seg_set_config(at, "plain", cfg)
        labs, dists = batch(at, fibs, "plain")
        for (rl, rd), l, d in zip(ref, labs, dists):
            np.testing.assert_array_equal(l, rl)
            np.testing.assert_array_equal(d, rd)
    binding.seg_set_config(at, "plain", 0)


@pytest.mark.parametrize("mode", ["gemm_bf16", "plain_culled", "gemm_inv_tf32",
                                  "culled_fused"])
def test_graph_replay_recapture_and_back_to_back(env, mode):
    """GEMM and culled modes: replays with the same shape, recaptures when the total or the
    subject count changes, and back-to-back calls with no synchronisation in between (the two
    pinned tables alternate)."""
    dev, a, at = env
    sets = [subjects(a, c, seed * 100, dev) for c, seed in
            (([500, 2000, 17], 7), ([500, 2000, 17], 8), ([3000, 5, 999, 0], 9), ([1200], 10))]
    outs = []
    for fibs in sets:  # no synchronisation between the calls
        labs = [torch.full((f.shape[0],), -7, dtype=torch.int32, device=dev) for f in fibs]
        dists = [torch.full((f.shape[0],), -7.0, device=dev) for f in fibs]
        binding.seg_label_batch(at, fibs, mode, labs, dists)
        outs.append((labs, dists))
    binding.seg_sync_status(at)
    for fibs, (labs, dists) in zip(sets, outs):
        for f, l, d in zip(fibs, labs, dists):
            rl, rd = single(at, f, "plain")
            np.testing.assert_array_equal(l.cpu().numpy(), rl)
            np.testing.assert_array_equal(d.cpu().numpy(), rd)


@pytest.fixture(scope="module")
def c4(env):
    """The 16-subject batch: counts log-uniform in [0.3M, 4.2M] (seeds 0-15, 28.6M fibers in
    all) against the 500-bundle x 20-centroid atlas."""
    dev = env[0]
    atlas = synth.make_atlas(500, seed=1002, device=dev)
    fibs = [torch.as_tensor(synth.make_batch_subject(atlas, s, device=dev), device=dev)
            for s in range(16)]
    at = binding.Atlas(torch.as_tensor(atlas.centroids, device=dev),
                       torch.as_tensor(atlas.bundle_of, device=dev),
                       torch.as_tensor(atlas.thresholds, device=dev))
    return atlas, at, fibs


@pytest.mark.parametrize("mode", ["plain", "gemm_bf16", "plain_culled", "culled_fused"])
def test_full_size_batch(env, c4, mode):
    """The full 16-subject batch in one call: every fiber of every subject equal to a single
    seg_label call on that subject (whose full-size parity is checked fiber by fiber in
    test_gpu_label.py), and 20,000 random fibers per subject against the oracle."""
    dev = env[0]
    atlas, at, fibs = c4
    assert 28_000_000 < sum(int(f.shape[0]) for f in fibs) < 29_500_000
    labs = [torch.full((f.shape[0],), -7, dtype=torch.int32, device=dev) for f in fibs]
    dists = [torch.full((f.shape[0],), -7.0, device=dev) for f in fibs]
    binding.seg_label_batch(at, fibs, mode, labs, dists)
    binding.seg_sync_status(at)
    rng = np.random.default_rng(4)
    ties = 0
    for s, f in enumerate(fibs):
        lab = labs[s].cpu().numpy()
        dst = dists[s].cpu().numpy()
        rl, rd, _, _ = binding.label(at, f, "plain")
        binding.seg_sync_status(at)
        np.testing.assert_array_equal(lab, rl.cpu().numpy())
        np.testing.assert_array_equal(dst, rd.cpu().numpy())
        idx = np.sort(rng.choice(f.shape[0], size=20_000, replace=False))
        fn = f[torch.as_tensor(idx, device=dev)].cpu().numpy()
        res = parity.compare_all(fn, atlas.centroids, atlas.bundle_of, atlas.thresholds,
                                 lab[idx], dst[idx])
        ties += res["near_ties"]
    print(f"\n{mode}: 16 subjects equal to single calls; 320,000 sampled fibers against the "
          f"oracle, {ties} near-ties")
