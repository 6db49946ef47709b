"""Soundness of the tensor-core prune's margin, checked on the CPU.

The GEMM modes keep a (fiber, centroid-orientation) pair when p~.q~ + pad >= alpha, where p~, q~
are the centred coordinates rounded to BF16 (or TF32), pad is the centroid operand's 64th
column and alpha a per-fiber constant (see k_gemm.cu). This test re-derives those operands in
numpy with the same rounding rules, takes the worst case of the FP32 accumulation, and checks on
every pair of the 10,000 x 1,000 workload that each pair the exact test accepts (FP64 d_ME of
that orientation within the threshold) survives. It also reports the prune rate. The bound
itself (max over points >= mean over points) is the plain inequality max >= mean. The kernel
evaluates alpha from an FP32 norm with downward rounding, so its alpha never exceeds the FP64
value used here and it keeps at least every pair this test keeps.
"""
import numpy as np
import pytest

import oracle

U = {"bf16": 2.0 ** -9, "tf32": 2.0 ** -11}
GAMMA = 64.0 / 2 ** 23
RHO = 1e-5


def kappa(fmt):
    u = U[fmt]
    return 1.05 * (2 * u + u * u) + 2 * GAMMA


def bf16_rn(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def bf16_ru(x):
    x = np.asarray(x, np.float32)
    u = x.view(np.uint32)
    low = (u & 0xFFFF) != 0
    hi = (u >> 16).astype(np.uint32)
    up = np.where((x > 0) & low, hi + 1, hi)
    return (up << 16).astype(np.uint32).view(np.float32)


def tf32_rn(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)


def tf32_up(x):
    x = np.asarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    low = (u & 0x1FFF) != 0
    r = np.where((x > 0) & low, (u + 0x2000) & 0xFFFFE000, u & 0xFFFFE000)
    return r.astype(np.uint32).view(np.float32)


def f32_round(x, direction):
    f = np.asarray(x, np.float64).astype(np.float32)
    if direction == "down":
        f = np.where(f.astype(np.float64) > x, np.nextafter(f, np.float32(-np.inf)), f)
    else:
        f = np.where(f.astype(np.float64) < x, np.nextafter(f, np.float32(np.inf)), f)
    return f.astype(np.float32)


def operands(fib, cen, bundle_of, thr, fmt):
    order = np.argsort(bundle_of, kind="stable")
    cs = cen[order]
    th = thr[bundle_of[order]].astype(np.float32)
    t2 = (th * th).astype(np.float32)
    c0 = np.round(cs[:, 10].astype(np.float64).mean(0)).astype(np.float32)
    P = (fib - c0).astype(np.float32).reshape(len(fib), 63)
    qd = (cs - c0).astype(np.float32).reshape(len(cs), 63)
    qr = (cs[:, ::-1] - c0).astype(np.float32).reshape(len(cs), 63)
    Q = np.empty((2 * len(cs), 63), np.float32)
    Q[0::2], Q[1::2] = qd, qr
    tcol = np.repeat(t2, 2).astype(np.float64)
    k = kappa(fmt)
    pn = (P.astype(np.float64) ** 2).sum(1)
    qn = (Q.astype(np.float64) ** 2).sum(1)
    alpha = f32_round(0.5 * (1 - k) * pn - (1e-5 * pn + 0.005), "down")
    G = 0.5 * (qn - 21 * tcol * (1 + RHO)) - 0.5 * k * qn - (1e-5 * (qn + 21 * tcol) + 0.005)
    pad32 = f32_round(-G, "up")
    rn, up = (bf16_rn, bf16_ru) if fmt == "bf16" else (tf32_rn, tf32_up)
    return rn(P), rn(Q), up(pad32), alpha, order, t2


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
def test_prune_never_drops_an_accepted_pair(small_workload, fmt):
    atlas, fib = small_workload
    Pt, Qt, pad, alpha, order, t2 = operands(fib, atlas.centroids, atlas.bundle_of,
                                             atlas.thresholds, fmt)
    P64, Q64 = Pt.astype(np.float64), Qt.astype(np.float64)
    dot = P64 @ Q64.T + pad.astype(np.float64)[None, :]
    mag = np.abs(P64) @ np.abs(Q64).T + np.abs(pad.astype(np.float64))[None, :]
    x_lo = dot - GAMMA * mag          # the smallest value the FP32 accumulation can return
    keep_worst = x_lo >= alpha.astype(np.float64)[:, None]
    # pairs the exact FP32 test accepts: FP64 d_ME^2 of that orientation within theta^2
    _, dd, dr = oracle.dme_matrix(fib, atlas.centroids[order])
    d2 = np.empty((len(fib), 2 * len(order)))
    d2[:, 0::2], d2[:, 1::2] = dd ** 2, dr ** 2
    accepted = d2 <= np.repeat(t2, 2).astype(np.float64)[None, :] * (1 + 1e-6)
    assert accepted.sum() > 1000
    assert not (accepted & ~keep_worst).any(), "a pair the exact test accepts was pruned"
    kept = (dot + GAMMA * mag >= alpha.astype(np.float64)[:, None]).mean()
    assert kept < 0.02  # the prune discards more than 98% of the pairs


def test_margin_constants():
    # BF16's margin is four times TF32's; both exceed the plain 2u bound of two roundings
    assert kappa("bf16") > 2 * U["bf16"] and kappa("tf32") > 2 * U["tf32"]
    assert kappa("bf16") / kappa("tf32") == pytest.approx(4, rel=0.02)


def inv_features(x):
    """30 orientation-free features per fiber: g = c / sqrt(2) + s_9, then sqrt(2) s_i for
    i = 0..8, with c the centre point and s_i the midpoint of points i and 20 - i."""
    x = np.asarray(x, np.float32)
    r2 = np.float32(0.70710678118654752)
    g = (x[:, 10] * r2 + (x[:, 9] + x[:, 11]) * np.float32(0.5)).astype(np.float32)
    m = ((x[:, :9] + x[:, 20:11:-1]) * r2).astype(np.float32)
    return np.concatenate([g, m.reshape(len(x), 27)], axis=1).astype(np.float32)


@pytest.mark.parametrize("fmt", ["bf16", "tf32"])
def test_orientation_free_prune_never_drops_an_accepted_centroid(small_workload, fmt):
    """I'(a,b) = |dg|^2 + 2 sum_(i<9) |ds_i|^2 <= |dc|^2 + 2 sum_(i<10) |ds_i|^2 <= 21 d_ME^2
    (both orientations), plus the same margin: every centroid the exact test accepts in either
    orientation survives."""
    atlas, fib = small_workload
    order = np.argsort(atlas.bundle_of, kind="stable")
    cs = atlas.centroids[order]
    th = atlas.thresholds[atlas.bundle_of[order]].astype(np.float32)
    t2 = (th * th).astype(np.float32).astype(np.float64)
    c0 = np.round(cs[:, 10].astype(np.float64).mean(0)).astype(np.float32)
    P = inv_features((fib - c0).astype(np.float32))
    Q = inv_features((cs - c0).astype(np.float32))
    k = kappa(fmt)
    pn = (P.astype(np.float64) ** 2).sum(1)
    qn = (Q.astype(np.float64) ** 2).sum(1)
    alpha = f32_round(0.5 * (1 - k) * pn - (1e-5 * pn + 0.005), "down").astype(np.float64)
    G = 0.5 * (qn - 21 * t2 * (1 + RHO)) - 0.5 * k * qn - (1e-5 * (qn + 21 * t2) + 0.005)
    rn, up = (bf16_rn, bf16_ru) if fmt == "bf16" else (tf32_rn, tf32_up)
    Pt, Qt, pad = rn(P).astype(np.float64), rn(Q).astype(np.float64), up(f32_round(-G, "up"))
    dot = Pt @ Qt.T + pad.astype(np.float64)[None, :]
    mag = np.abs(Pt) @ np.abs(Qt).T + np.abs(pad.astype(np.float64))[None, :]
    keep_worst = dot - GAMMA * mag >= alpha[:, None]
    dme, _, _ = oracle.dme_matrix(fib, cs)
    accepted = dme ** 2 <= t2[None, :] * (1 + 1e-6)
    assert accepted.sum() > 1000
    assert not (accepted & ~keep_worst).any()
    assert (dot + GAMMA * mag >= alpha[:, None]).mean() < 0.05


def test_orientation_free_identity_is_a_lower_bound():
    """The inequalities behind the features on random fibers: I' <= min(S_direct, S_reversed),
    and I' reaches that bound where it should: for a centroid equal to the fiber (both zero)."""
    rng = np.random.default_rng(2)
    A = rng.normal(0, 20, size=(30, 21, 3)).astype(np.float32)
    B = rng.normal(0, 20, size=(40, 21, 3)).astype(np.float32)
    FA, FB = inv_features(A).astype(np.float64), inv_features(B).astype(np.float64)
    I = ((FA[:, None] - FB[None]) ** 2).sum(-1)
    Sd = ((A[:, None].astype(np.float64) - B[None]) ** 2).sum((-1, -2))
    Sr = ((A[:, None].astype(np.float64) - B[None, :, ::-1]) ** 2).sum((-1, -2))
    assert np.all(I <= np.minimum(Sd, Sr) * (1 + 1e-6) + 1e-6)
    FA2 = inv_features(A[:, ::-1]).astype(np.float64)  # the features ignore the orientation
    np.testing.assert_allclose(FA2, FA, rtol=1e-6, atol=1e-4)
    assert np.all(((FA[:, None] - FA[None]) ** 2).sum(-1).diagonal() == 0)
