"""Seeded synthetic tractography inputs shaped like the paper's workloads (Section 2.1-2.3).

This module only makes inputs: Bezier curves, arc-length resampling to 21 points, thresholds
and affines. It holds none of the segmentation arithmetic (no d_E, no d_ME, no labelling), so
both the CUDA path and the FP64 oracle can consume what it produces.

Random numbers come from numpy's PCG64 with fixed seeds; the deterministic geometry (Bezier
evaluation and resampling) runs in float64 torch ops on the requested device, so large
subjects can be generated on the GPU in seconds. Coordinates are millimetres inside the box
[-70,70] x [-100,70] x [-50,80].

Recipe (the paper's atlases have 21-point centroids and per-bundle thresholds, Section 2.2 and
2.3; subjects are 21-point resampled fibers):
  * bundle curve: length L ~ U[20,80]; P0 uniform in the box shrunk by 10 mm; P3 = P0 + 0.8 L d
    with d uniform on the sphere; P1, P2 = the 1/3 and 2/3 chord points + N(0, 0.15 L) per
    coordinate; scaled about the chord midpoint so the dense arc length is L; redrawn if any
    dense point leaves the box;
  * centroids: per bundle, control points + N(0, 1.5) per coordinate, resampled to 21
    arc-length-equidistant points; thresholds U[5, 8] mm per bundle;
  * subject: a fraction of fibers are perturbed bundle curves (control points + N(0, 2)), the
    rest fresh random curves; every fiber's point order is reversed with probability 0.5; the
    fiber order is shuffled.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

NPTS = 21
BOX_LO = np.array([-70.0, -100.0, -50.0])
BOX_HI = np.array([70.0, 70.0, 80.0])
DENSE = 257  # dense Bezier samples used for arc length


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _bernstein(device) -> torch.Tensor:
    t = torch.linspace(0.0, 1.0, DENSE, dtype=torch.float64, device=device)
    s = 1.0 - t
    return torch.stack([s * s * s, 3 * s * s * t, 3 * s * t * t, t * t * t], dim=1)  # [D,4]


def _dense(ctrl: torch.Tensor) -> torch.Tensor:
    """ctrl [n,4,3] float64 -> dense points [n,D,3]."""
    return torch.einsum("dk,nkc->ndc", _bernstein(ctrl.device), ctrl)


def _arc_length(dense: torch.Tensor) -> torch.Tensor:
    return (dense[:, 1:] - dense[:, :-1]).norm(dim=2).sum(dim=1)


def resample(dense: torch.Tensor, npts: int = NPTS) -> torch.Tensor:
    """Resample polylines [n,D,3] to npts arc-length-equidistant points (linear interpolation)."""
    seg = (dense[:, 1:] - dense[:, :-1]).norm(dim=2)  # [n,D-1]
    cum = torch.cat([torch.zeros_like(seg[:, :1]), seg.cumsum(dim=1)], dim=1)  # [n,D]
    total = cum[:, -1:]
    frac = torch.linspace(0.0, 1.0, npts, dtype=dense.dtype, device=dense.device)
    target = total * frac[None, :]  # [n,npts]
    idx = torch.searchsorted(cum.contiguous(), target.contiguous(), right=True) - 1
    idx = idx.clamp(0, dense.shape[1] - 2)
    c0 = torch.gather(cum, 1, idx)
    c1 = torch.gather(cum, 1, idx + 1)
    w = ((target - c0) / (c1 - c0).clamp_min(1e-300)).clamp(0.0, 1.0)
    p0 = torch.gather(dense, 1, idx[..., None].expand(-1, -1, 3))
    p1 = torch.gather(dense, 1, (idx + 1)[..., None].expand(-1, -1, 3))
    return p0 + w[..., None] * (p1 - p0)


def _random_curves(rng: np.random.Generator, count: int, device) -> np.ndarray:
    """Control points [count,4,3] of random bundle-like curves that stay inside the box."""
    out = []
    have = 0
    lo = BOX_LO + 10.0
    hi = BOX_HI - 10.0
    while have < count:
        k = int((count - have) * 1.25) + 16
        L = rng.uniform(20.0, 80.0, size=k)
        p0 = rng.uniform(lo, hi, size=(k, 3))
        d = rng.normal(size=(k, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        p3 = p0 + 0.8 * L[:, None] * d
        p1 = p0 + (p3 - p0) / 3.0 + rng.normal(0.0, 1.0, size=(k, 3)) * (0.15 * L)[:, None]
        p2 = p0 + 2.0 * (p3 - p0) / 3.0 + rng.normal(0.0, 1.0, size=(k, 3)) * (0.15 * L)[:, None]
        ctrl = np.stack([p0, p1, p2, p3], axis=1)
        c = torch.from_numpy(ctrl).to(device)
        l0 = _arc_length(_dense(c)).cpu().numpy()
        mid = 0.5 * (p0 + p3)
        ctrl = mid[:, None, :] + (ctrl - mid[:, None, :]) * (L / l0)[:, None, None]
        dense = _dense(torch.from_numpy(ctrl).to(device))
        lo_t = torch.as_tensor(BOX_LO, device=device)
        hi_t = torch.as_tensor(BOX_HI, device=device)
        inside = ((dense >= lo_t) & (dense <= hi_t)).all(dim=2).all(dim=1).cpu().numpy()
        acc = ctrl[inside]
        take = min(len(acc), count - have)
        out.append(acc[:take])
        have += take
    return np.concatenate(out, axis=0)


def _resample_ctrl(ctrl: np.ndarray, device, chunk: int = 1 << 18) -> np.ndarray:
    """Bezier control points [n,4,3] -> float32 [n,21,3] arc-length-equidistant points."""
    n = ctrl.shape[0]
    res = np.empty((n, NPTS, 3), dtype=np.float32)
    for s in range(0, n, chunk):
        c = torch.from_numpy(np.ascontiguousarray(ctrl[s:s + chunk])).to(device)
        res[s:s + chunk] = resample(_dense(c)).to(torch.float32).cpu().numpy()
    return res


@dataclass
class Atlas:
    centroids: np.ndarray  # float32 [M,21,3]
    bundle_of: np.ndarray  # int32 [M]
    thresholds: np.ndarray  # float32 [B], mm
    base_ctrl: np.ndarray  # float64 [B,4,3], the bundle curves subjects are drawn around

    @property
    def M(self) -> int:
        return int(self.centroids.shape[0])

    @property
    def B(self) -> int:
        return int(self.thresholds.shape[0])


def make_atlas(n_bundles: int, per_bundle=20, seed: int = 1000, thr_lo: float = 5.0,
               thr_hi: float = 8.0, sigma: float = 1.5, device="cpu") -> Atlas:
    """Atlas of n_bundles bundles, bundle-major, thresholds U[thr_lo, thr_hi]; per_bundle is a
    centroid count for every bundle or a sequence of n_bundles counts."""
    rng = _rng(seed)
    base = _random_curves(rng, n_bundles, device)
    thr = rng.uniform(thr_lo, thr_hi, size=n_bundles).astype(np.float32)
    counts = np.broadcast_to(np.asarray(per_bundle, dtype=np.int64), (n_bundles,))
    if np.all(counts == counts[0]):
        pert = rng.normal(0.0, sigma, size=(n_bundles, int(counts[0]), 4, 3))
        ctrl = (base[:, None] + pert).reshape(-1, 4, 3)
    else:
        pert = rng.normal(0.0, sigma, size=(int(counts.sum()), 4, 3))
        ctrl = np.repeat(base, counts, axis=0) + pert
    cen = _resample_ctrl(ctrl, device)
    bundle_of = np.repeat(np.arange(n_bundles, dtype=np.int32), counts)
    return Atlas(cen, bundle_of, thr, base)


def whole_brain_counts(n_bundles: int = 62, total: int = 44_345) -> list[int]:
    """Centroids per bundle of the whole-brain stress atlas: `total` centroids spread as evenly
    as possible over `n_bundles` bundles (the paper's 62-bundle atlas has 44,345 centroids)."""
    q, r = divmod(total, n_bundles)
    return [q + 1] * r + [q] * (n_bundles - r)


def make_subject(atlas: Atlas, n: int, bundle_frac: float, seed: int, sigma: float = 2.0,
                 device="cpu") -> np.ndarray:
    """n fibers float32 [n,21,3]: bundle_frac perturbed bundle curves, the rest random curves."""
    rng = _rng(seed)
    return _subject_from_rng(rng, atlas, n, bundle_frac, sigma, device)


def _subject_ctrl(rng, atlas: Atlas, n: int, bundle_frac: float, sigma: float, device):
    """Control points of a subject's curves, which are reversed, and the shuffle."""
    nb = int(round(bundle_frac * n))
    nn = n - nb
    bid = rng.integers(0, atlas.B, size=nb)
    ctrl_b = atlas.base_ctrl[bid] + rng.normal(0.0, sigma, size=(nb, 4, 3))
    ctrl_n = _random_curves(rng, nn, device) if nn > 0 else np.zeros((0, 4, 3))
    ctrl = np.concatenate([ctrl_b, ctrl_n], axis=0)
    rev = rng.random(n) < 0.5
    perm = rng.permutation(n)
    return ctrl, rev, perm


def _subject_from_rng(rng, atlas: Atlas, n: int, bundle_frac: float, sigma: float, device):
    ctrl, rev, perm = _subject_ctrl(rng, atlas, n, bundle_frac, sigma, device)
    fib = _resample_ctrl(ctrl, device)
    fib[rev] = fib[rev, ::-1]
    return np.ascontiguousarray(fib[perm])


STEP_MM = 0.2  # tractography step of the paper's data (Section 2.1)


def make_streamlines(atlas: Atlas, n: int, bundle_frac: float, seed: int, sigma: float = 2.0,
                     step: float = STEP_MM, device="cpu", chunk: int = 1 << 17):
    """Raw (not resampled) streamlines of the subject recipe, as CSR arrays on `device`:
    points float32 [P, 3] and offsets int64 [n + 1]. Each curve (the same control points,
    reversals and shuffle as make_subject with this seed) is evaluated at K = round(L / step) + 1
    Bezier parameters spaced uniformly in [0, 1], so consecutive points are about `step` mm apart
    on average but unevenly spaced in arc length."""
    ctrl, rev, perm = _subject_ctrl(_rng(seed), atlas, n, bundle_frac, sigma, device)
    ctrl = ctrl[perm]
    rev = rev[perm]
    pts_out, counts = [], []
    for s0 in range(0, n, chunk):
        c = torch.from_numpy(np.ascontiguousarray(ctrl[s0:s0 + chunk])).to(device)
        L = _arc_length(_dense(c))
        k = torch.clamp(torch.round(L / step).to(torch.int64) + 1, min=2)
        fid = torch.repeat_interleave(torch.arange(c.shape[0], device=device), k)
        start = torch.cumsum(k, 0) - k
        idx = torch.arange(fid.shape[0], device=device) - start[fid]
        t = idx.to(torch.float64) / (k[fid] - 1).to(torch.float64)
        r = torch.from_numpy(rev[s0:s0 + chunk]).to(device)[fid]
        t = torch.where(r, 1.0 - t, t)
        u = 1.0 - t
        bern = torch.stack([u * u * u, 3 * u * u * t, 3 * u * t * t, t * t * t], dim=1)
        pts_out.append(torch.einsum("pk,pkc->pc", bern, c[fid]).to(torch.float32))
        counts.append(k)
    counts = torch.cat(counts)
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=device)
    offsets[1:] = torch.cumsum(counts, 0)
    return torch.cat(pts_out).contiguous(), offsets


def batch_counts(nsubj: int = 16, lo: float = 3e5, hi: float = 4.2e6) -> list[int]:
    """Per-subject fiber counts of the batched workload: subject s draws first from seed s."""
    return [int(round(math.exp(_rng(s).uniform(math.log(lo), math.log(hi))))) for s in range(nsubj)]


def make_batch_subject(atlas: Atlas, s: int, bundle_frac: float = 0.75, device="cpu",
                       lo: float = 3e5, hi: float = 4.2e6, scale: float = 1.0) -> np.ndarray:
    """Subject s of the batched workload; scale < 1 shrinks its count (for small tests)."""
    rng = _rng(s)
    n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    n = max(1, int(round(n * scale)))
    return _subject_from_rng(rng, atlas, n, bundle_frac, 2.0, device)


def random_affine(seed: int, max_deg: float = 5.0, max_t: float = 4.0, s_lo: float = 0.95,
                  s_hi: float = 1.05) -> np.ndarray:
    """12 float64 values: M = s R (row-major, 9) then t (3); R axis-angle, angle <= max_deg."""
    rng = _rng(seed)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = math.radians(rng.uniform(0.0, max_deg))
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
    s = rng.uniform(s_lo, s_hi)
    t = rng.normal(size=3)
    t *= rng.uniform(0.0, max_t) / np.linalg.norm(t)
    return np.concatenate([(s * R).reshape(-1), t]).astype(np.float64)


# Named workloads (sizes from the paper's experiments: 21-point fibers, subjects of millions of
# fibers, atlases of thousands of centroids, Section 2.2 and Section 3).
WORKLOADS = {
    # 10,000 fibers, 50 bundles x 20 centroids, 70% bundle fibers.
    "subject10k_atlas1k": dict(n=10_000, bundles=50, bundle_frac=0.70, atlas_seed=1001, seed=1),
    # 4,145,000 fibers (the paper's headline subject size), 500 x 20 centroids, 75% bundle.
    "subject4145k_atlas10k": dict(n=4_145_000, bundles=500, bundle_frac=0.75, atlas_seed=1002,
                                  seed=2),
    # 1,000,000 fibers, 250 x 20 centroids, 70% bundle, after a random affine (seed 5).
    "affine1m_atlas5k": dict(n=1_000_000, bundles=250, bundle_frac=0.70, atlas_seed=1005, seed=5),
    # The paper's headline subject size against an atlas shaped like its 62-bundle whole-brain
    # atlas (44,345 centroids, Section 2.2), 75% bundle fibers.
    "subject4145k_atlas44k": dict(n=4_145_000, bundles=62, per_bundle=whole_brain_counts(),
                                  bundle_frac=0.75, atlas_seed=1006, seed=6),
}


def workload(name: str, n: int | None = None, device="cpu"):
    """(atlas, fibers) for a named workload; n overrides the fiber count (same seeds)."""
    w = WORKLOADS[name]
    atlas = make_atlas(w["bundles"], per_bundle=w.get("per_bundle", 20), seed=w["atlas_seed"],
                       device=device)
    fib = make_subject(atlas, w["n"] if n is None else n, w["bundle_frac"], w["seed"],
                       device=device)
    return atlas, fib
