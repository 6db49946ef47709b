"""Failure paths without a GPU fault: a bounded device wait that runs out (the test makes the
tensor-core screen's first wait give up at once) is reported as SEG_ERR_TIMEOUT through
seg_sync_status and leaves the atlas usable; a scratch request above the caller's limit returns
SEG_ERR_OOM before any device work."""
import numpy as np
import pytest
import torch

from paper_1912_11494_gb300 import binding, synth

pytestmark = pytest.mark.gpu

SEG_ERR_OOM, SEG_ERR_TIMEOUT = 3, 5


@pytest.fixture(scope="module")
def env():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    a = synth.make_atlas(100, seed=1003)
    fib = torch.as_tensor(synth.make_subject(a, 50_000, 0.75, seed=3), device=dev)
    at = binding.Atlas(torch.as_tensor(a.centroids, device=dev),
                       torch.as_tensor(a.bundle_of, device=dev),
                       torch.as_tensor(a.thresholds, device=dev))
    ref = [x.cpu().numpy() for x in binding.label(at, fib, "plain")]
    binding.seg_sync_status(at)
    return dev, at, fib, ref


@pytest.mark.parametrize("mode", ["gemm_bf16", "gemm_inv_tf32"])
def test_screen_wait_timeout_is_reported_and_recovered(env, mode):
    dev, at, fib, ref = env
    binding.seg_set_wait_limit(at, 0)
    binding.label(at, fib, mode)
    with pytest.raises(binding.SegError) as err:
        binding.seg_sync_status(at)
    assert err.value.status == SEG_ERR_TIMEOUT
    binding.seg_set_wait_limit(at, 2_000_000_000)
    got = [x.cpu().numpy() for x in binding.label(at, fib, mode)]
    binding.seg_sync_status(at)  # the status word was cleared: no stale timeout
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x, y)


def test_scratch_limit_gives_oom_before_any_work(env):
    dev, at, fib, ref = env
    binding.seg_set_scratch_limit(at, 1 << 20)
    lab = torch.full((fib.shape[0],), -7, dtype=torch.int32, device=dev)
    with pytest.raises(binding.SegError) as err:
        binding.seg_label(at, fib, "gemm_bf16", lab)
    assert err.value.status == SEG_ERR_OOM and b"limit" in binding.lib().seg_last_error()
    torch.cuda.synchronize()
    assert bool((lab == -7).all())  # nothing was enqueued
    binding.seg_sync_status(at)
    # the plain kernel needs no scratch and still runs under the limit
    got = [x.cpu().numpy() for x in binding.label(at, fib, "plain")]
    np.testing.assert_array_equal(got[0], ref[0])
    binding.seg_set_scratch_limit(at, 0)
    got = [x.cpu().numpy() for x in binding.label(at, fib, "gemm_bf16")]
    binding.seg_sync_status(at)
    for x, y in zip(ref, got):
        np.testing.assert_array_equal(x, y)
