"""torch.autograd wrapper of the segmentation cost for subject-to-atlas affine refinement.

C(T, c) = sum over labelled fibers f of d_ME(T f, c_sigma(f)), T f = A f + t on every point;
sigma(f) is the closest passing centroid (Algorithm 1; Eq. 2 for d_ME). The forward pass runs
seg_apply_affine, seg_label and seg_grad (which also returns C); the backward pass scales the
saved gradient (subgradient through the argmax point) by the incoming gradient. Every step runs
in libseg's kernels; torch only holds the tensors.
"""
from __future__ import annotations

import torch

from . import binding


class SegDME(torch.autograd.Function):
    """cost = SegDME.apply(fibers, affine12, centroids, atlas, mode)

    fibers: CUDA float32 [n,21,3] (untransformed); affine12: float64 [12] (A row-major then t,
    any device); centroids: CUDA float32 [M,21,3], the tensor the atlas was built from (its
    gradient is returned); atlas: binding.Atlas. Returns a float64 scalar on the fibers' device.
    """

    @staticmethod
    def forward(ctx, fibers, affine12, centroids, atlas, mode="plain"):
        dev = fibers.device
        aff = affine12.detach().to("cpu", torch.float64)
        y = binding.seg_apply_affine(fibers, aff)
        n = fibers.shape[0]
        labels = torch.empty(n, dtype=torch.int32, device=dev)
        cidx = torch.empty(n, dtype=torch.int32, device=dev)
        orient = torch.empty(n, dtype=torch.uint8, device=dev)
        binding.seg_label(atlas, y, mode, labels, None, cidx, orient)
        g_aff = torch.empty(12, dtype=torch.float64, device=dev)
        g_cen = torch.empty_like(centroids) if ctx.needs_input_grad[2] else None
        cost = torch.empty(1, dtype=torch.float64, device=dev)
        binding.seg_grad(atlas, fibers, aff, cidx, orient, g_aff, g_cen, cost)
        ctx.save_for_backward(g_aff, g_cen if g_cen is not None else torch.empty(0, device=dev))
        ctx.aff_device = affine12.device
        ctx.has_cen = g_cen is not None
        ctx.structure = (labels, cidx, orient)
        return cost[0]

    @staticmethod
    def backward(ctx, grad_out):
        g_aff, g_cen = ctx.saved_tensors
        ga = (g_aff * grad_out).to(ctx.aff_device) if ctx.needs_input_grad[1] else None
        gc = (g_cen * grad_out.to(g_cen.dtype)) if ctx.has_cen and ctx.needs_input_grad[2] \
            else None
        return None, ga, gc, None, None


def seg_cost(fibers, affine12, centroids, atlas, mode="plain"):
    return SegDME.apply(fibers, affine12, centroids, atlas, mode)
