"""seg_grad_noalloc: the allocation-free gradient entry point.

Some callers cannot allocate device memory: code inside a host allocator callback, a plugin
whose host framework owns every device allocation, or a process that reserved all device memory
up front. seg_grad may grow a scratch buffer with cudaMalloc; seg_grad_noalloc uses a fixed
array compiled into the library instead. This test calls it through the C ABI twice in a row
and checks each result against seg_grad's, and checks that an oversized call is refused.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_1912_11494_gb300 import binding, synth

pytestmark = pytest.mark.gpu

MAX_FIBERS = 4_194_304


@pytest.fixture(scope="module")
def setup():
    assert torch.cuda.is_available()
    from paper_1912_11494_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    a = synth.make_atlas(40, seed=1005)
    fib = torch.as_tensor(synth.make_subject(a, 5000, 0.7, seed=5), device=dev)
    at = binding.Atlas(torch.as_tensor(a.centroids, device=dev),
                       torch.as_tensor(a.bundle_of, device=dev),
                       torch.as_tensor(a.thresholds, device=dev))
    aff = synth.random_affine(7, max_deg=2.0, max_t=1.0, s_lo=0.99, s_hi=1.01)
    y = binding.seg_apply_affine(fib, aff)
    n = fib.shape[0]
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    cidx = torch.empty(n, dtype=torch.int32, device=dev)
    orient = torch.empty(n, dtype=torch.uint8, device=dev)
    binding.seg_label(at, y, "plain", lab, None, cidx, orient)
    binding.seg_sync_status(at)
    return dev, a, at, fib, aff, cidx, orient


def grads(fn, setup):
    dev, a, at, fib, aff, cidx, orient = setup
    ga = torch.full((12,), np.nan, dtype=torch.float64, device=dev)
    gc = torch.full((a.M, 21, 3), np.nan, dtype=torch.float32, device=dev)
    cost = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
    fn(at, fib, aff, cidx, orient, ga, gc, cost)
    binding.seg_sync_status(at)
    return ga.cpu().numpy(), gc.cpu().numpy(), float(cost.item())


def test_noalloc_matches_seg_grad_twice(setup):
    ref_a, ref_c, ref_cost = grads(binding.seg_grad, setup)
    assert ref_cost > 0 and np.isfinite(ref_a).all()
    prev = None
    for _ in range(2):
        ga, gc, cost = grads(binding.seg_grad_noalloc, setup)
        # same FP32 per-fiber terms; only the FP64 summation order and the order of the FP32
        # atomic adds into the centroid gradient differ
        assert cost == pytest.approx(ref_cost, rel=1e-9)
        np.testing.assert_allclose(ga, ref_a, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(gc, ref_c, rtol=0, atol=1e-4)
        if prev is not None:
            assert np.array_equal(ga, prev[0]) and cost == prev[2]
        prev = (ga, gc, cost)


def test_noalloc_rejects_oversized_call(setup):
    dev, a, at, fib, aff, cidx, orient = setup
    ga = torch.zeros(12, dtype=torch.float64, device=dev)
    buf = binding._affine_buf(aff)
    st = binding.lib().seg_grad_noalloc(at.handle, fib.data_ptr(), MAX_FIBERS + 1,
                                        binding.ctypes.cast(buf, binding.ctypes.c_void_p),
                                        cidx.data_ptr(), orient.data_ptr(), ga.data_ptr(), None,
                                        None, torch.cuda.current_stream().cuda_stream)
    assert st == 1  # SEG_ERR_INVALID_ARG, refused before any device work
    assert b"4194304" in binding.lib().seg_last_error()
