"""seg_grad_noalloc: the allocation-free gradient entry point.

Some callers cannot allocate device memory: code inside a host allocator callback, a plugin
whose host framework owns every device allocation, or a process that reserved all device memory
up front. seg_grad may grow a scratch buffer with cudaMalloc; seg_grad_noalloc uses a fixed
array compiled into the library instead. This test calls it through the C ABI twice in a row
on an atlas whose scratch has never been grown, checks that the device's free memory does not
change across those calls, checks each result against seg_grad's, and checks that an oversized
call is refused.

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
    """A freshly created atlas on which seg_grad has never run, so its scratch arena is still
    empty, and the forward pass's structure for 5,000 transformed fibers."""
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


def outputs(setup):
    dev, a = setup[0], setup[1]
    return (torch.full((12,), np.nan, dtype=torch.float64, device=dev),
            torch.full((a.M, 21, 3), np.nan, dtype=torch.float32, device=dev),
            torch.full((1,), np.nan, dtype=torch.float64, device=dev))


def run(fn, setup, out):
    dev, a, at, fib, aff, cidx, orient = setup
    ga, gc, cost = out
    fn(at, fib, aff, cidx, orient, ga, gc, cost)
    binding.seg_sync_status(at)
    return ga.cpu().numpy(), gc.cpu().numpy(), float(cost.item())


def test_noalloc_matches_seg_grad_twice(setup):
    # the allocation-free calls come first on this atlas: nothing may have grown its scratch
    outs = [outputs(setup) for _ in range(3)]
    run(binding.seg_grad_noalloc, setup, outs[0])      # first call on the device: module load
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = [run(binding.seg_grad_noalloc, setup, outs[k]) for k in (1, 2)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "seg_grad_noalloc allocated device memory"
    ref_a, ref_c, ref_cost = run(binding.seg_grad, setup, outputs(setup))
    assert ref_cost > 0 and np.isfinite(ref_a).all()
    for ga, gc, cost in got:
        # the same FP32 per-fiber terms; the FP64 sums run in another fixed order, and the
        # centroid gradient is an FP32 atomic sum here (seg_grad's is exact fixed point)
        assert cost == pytest.approx(ref_cost, rel=1e-9)
        np.testing.assert_allclose(ga, ref_a, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(gc, ref_c, rtol=0, atol=1e-4)
    assert np.array_equal(got[0][0], got[1][0]) and got[0][2] == got[1][2]


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
