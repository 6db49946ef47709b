"""Soundness of the fused mode's test1 screen, checked on the CPU.

SEG_MODE_CULLED_FUSED keeps a (fiber, centroid) pair for the exact test when, in FP32,
    t = fma(z, q.z, fma(y, q.y, fma(x, q.x, q.w)))  >=  he,
with (x, y, z) the fiber's centre point minus the atlas centre, q = (centred centroid centre
point, w), w = (theta^2 - |b|^2)/2 + 1e-5 (|b|^2 + theta^2) + 1e-3 (the atlas's test1 row),
h = |a|^2/2 - 1e-5 |a|^2 - 1e-3, and
    he = h + max(0, fma(0.5, tmin - bb, -(1e-5 (tmin + |h|) + 1e-4))),
tmin the chunk's smallest theta^2 and bb the fiber's best bound so far. The exact test then
keeps the pair when the FP32 squared centre distance of the raw points is <= min(theta^2, bb).
This test emulates those FP32 steps in numpy (an FMA as the exact product and sum rounded once
to FP32, through float64) on pairs built to sit on that bound, in every direction, at
coordinates of up to 100 mm from the atlas centre, and checks that each pair the exact centre
test accepts passes the screen: the threshold's rise with the best never drops a pair that
could still win.
"""
import numpy as np

F = np.float32


def fma32(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64)
            + np.asarray(c, np.float64)).astype(F)


def pd2_32(a, b):
    """The exact test's FP32 squared distance of two raw points."""
    d = (a - b).astype(F)
    return fma32(d[:, 0], d[:, 0], fma32(d[:, 1], d[:, 1], (d[:, 2] * d[:, 2]).astype(F)))


def screen_row(b, c0, t2):
    """The atlas's test1 row of a centroid centre point b (raw) with threshold^2 t2."""
    q = (b - c0).astype(F)
    r2 = fma32(q[:, 0], q[:, 0], fma32(q[:, 1], q[:, 1], (q[:, 2] * q[:, 2]).astype(F)))
    w = (F(0.5) * (t2 - r2).astype(F)).astype(F)
    w = (w + (F(1e-5) * (r2 + t2).astype(F)).astype(F)).astype(F)
    w = (w + F(1e-3)).astype(F)
    return q, w


def fiber_h(a, c0):
    p = (a - c0).astype(F)
    r2 = fma32(p[:, 0], p[:, 0], fma32(p[:, 1], p[:, 1], (p[:, 2] * p[:, 2]).astype(F)))
    h = ((F(0.5) * r2).astype(F) - (F(1e-5) * r2).astype(F)).astype(F)
    return p, (h - F(1e-3)).astype(F)


def test_tightened_test1_keeps_every_pair_the_exact_test_accepts():
    rng = np.random.default_rng(11)
    n = 400_000
    c0 = rng.uniform(-20, 20, 3).astype(F)
    a = (c0 + rng.uniform(-100, 100, (n, 3))).astype(F)
    theta = rng.uniform(2.0, 12.0, n)
    t2 = (theta * theta).astype(F)
    # the fiber's best so far: none (inf), above theta^2, or below it (where it tightens)
    kind = rng.integers(0, 3, n)
    bb = np.where(kind == 0, np.inf,
                  np.where(kind == 1, t2 * rng.uniform(1.0, 2.0, n),
                           t2 * rng.uniform(0.01, 1.0, n))).astype(F)
    bound = np.minimum(t2.astype(np.float64), bb.astype(np.float64))
    # centroid centre points at (just inside) the bound's distance, in random directions
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = np.sqrt(bound) * rng.uniform(0.999, 1.0, n)
    b = (a.astype(np.float64) + u * r[:, None]).astype(F)
    # the chunk's smallest theta^2: this centroid's or a smaller one of the same chunk
    tmin = np.where(rng.random(n) < 0.5, t2, (t2 * rng.uniform(0.5, 1.0, n)).astype(F))
    tmin = tmin.astype(F)

    exact = pd2_32(a, b).astype(np.float64) <= bound  # the exact FP32 centre test
    q, w = screen_row(b, c0, t2)
    p, h = fiber_h(a, c0)
    t = fma32(p[:, 2], q[:, 2], fma32(p[:, 1], q[:, 1], fma32(p[:, 0], q[:, 0], w)))
    with np.errstate(invalid="ignore"):
        margin = (F(1e-5) * (tmin + np.abs(h)).astype(F)).astype(F) + F(1e-4)
        rise = fma32(F(0.5), (tmin - bb).astype(F), -margin.astype(F))
    rise = np.where(np.isnan(rise), F(0), np.maximum(F(0), rise)).astype(F)
    he = (h + rise).astype(F)
    kept = t >= he
    missed = exact & ~kept
    assert exact.sum() > n // 2
    assert not missed.any(), f"{int(missed.sum())} accepted pairs dropped by the screen"
    # the rise does its job: with a best well below the chunk's smallest threshold, a centroid
    # beyond the best (by more than the gap between its own threshold and the chunk's smallest,
    # which the screen does not know, and than test1's own slack, which grows with the squared
    # distance from the atlas centre) is dropped although it is within its threshold
    t2d, tmd = t2.astype(np.float64), tmin.astype(np.float64)
    bbd = np.where(kind == 2, bb.astype(np.float64), 0.0)  # (rows with a finite best only)
    pa2 = (p.astype(np.float64) ** 2).sum(axis=1)
    r2_far = bbd + (t2d - tmd) + 0.25 * (t2d - bbd) + 1.0 + 1e-4 * pa2
    sel = (kind == 2) & (bbd < 0.5 * tmd) & (r2_far < 0.95 * t2d)
    r_far = np.sqrt(np.where(sel, r2_far, 1.0))
    b_far = (a.astype(np.float64) + u * r_far[:, None]).astype(F)
    q, w = screen_row(b_far, c0, t2)
    t = fma32(p[:, 2], q[:, 2], fma32(p[:, 1], q[:, 1], fma32(p[:, 0], q[:, 0], w)))
    assert sel.sum() > 1000
    assert not (t >= he)[sel].any()
    # without the rise the same pairs pass test1 (the threshold alone keeps them)
    assert (t >= h)[sel].all()
