"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics, not by itself.

* hand-derived worked examples (tests/golden/worked_examples.json; Eq. 1, Eq. 2, Algorithm 1);
* closed forms on straight fibers, a library special case (point fibers reduce Eq. 2 to the
  Euclidean distance, checked against scipy's cdist);
* invariants of Eq. 2: d(a,a) = 0, symmetry, reversal symmetry, triangle inequality, invariance
  under a shared rigid motion;
* labelling against an independent brute force written as a sort over all candidates;
* the progressive-discarding cascade (Section 2.3) against the plain definition;
* the gradient against closed forms and central finite differences.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _rand_fibers(rng, n, scale=30.0):
    base = rng.normal(0, scale, size=(n, 1, 3))
    walk = np.cumsum(rng.normal(0, 2.0, size=(n, 21, 3)), axis=1)
    return (base + walk).astype(np.float32)


def _rev(x):
    return x[..., ::-1, :]


@pytest.fixture(scope="module")
def gold():
    with open(GOLD) as fh:
        return json.load(fh)


def test_worked_examples_dme(gold):
    for case in gold["dme_cases"]:
        a = np.array(case["a"], np.float32)[None]
        b = np.array(case["b"], np.float32)[None]
        dme, dd, dr = oracle.dme_matrix(a, b)
        assert dd[0, 0] == pytest.approx(case["dd"], abs=1e-12), case["name"]
        assert dr[0, 0] == pytest.approx(case["dr"], abs=1e-12), case["name"]
        assert dme[0, 0] == pytest.approx(case["dme"], abs=1e-12), case["name"]


def test_worked_examples_labels(gold):
    fib = np.array(gold["fiber"], np.float32)[None]
    for case in gold["label_cases"]:
        cen = np.array(case["centroids"], np.float32)
        for mode in ("brute", "cascade"):
            r = oracle.label(fib, cen, case["bundle_of"], case["thresholds"], mode)
            assert r["labels"][0] == case["label"], (case["name"], mode)
            assert r["cidx"][0] == case["cidx"], (case["name"], mode)
            if case["dist"] is None:
                assert math.isinf(r["dist"][0])
            else:
                assert r["dist"][0] == pytest.approx(case["dist"], abs=1e-12)


def test_parallel_offsets_closed_form():
    """Straight fiber vs the same fiber shifted by delta: d_ME = |delta| whenever the fiber is
    long enough that the reversed orientation is worse (Eq. 2). Covers each coordinate and
    both signs, so a dropped term or a sign slip shows up."""
    rng = np.random.default_rng(7)
    t = np.arange(21)[:, None]
    for _ in range(50):
        d = rng.normal(0, 3, size=3)
        direction = rng.normal(size=3)
        direction /= np.linalg.norm(direction)
        a = (t * 2.0 * direction + rng.normal(0, 20, size=3)).astype(np.float64)
        b = a + d
        dme, dd, dr = oracle.dme_matrix(a[None].astype(np.float32), b[None].astype(np.float32))
        a32, b32 = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
        exact = np.linalg.norm(b32 - a32, axis=1).max()  # float32 rounding of the inputs
        assert dd[0, 0] == pytest.approx(exact, rel=1e-12)
        assert dd[0, 0] == pytest.approx(np.linalg.norm(d), abs=1e-4)
        assert dme[0, 0] == dd[0, 0]


def test_point_fibers_reduce_to_euclidean():
    """If every point of a and of b is the same point, Eq. 2 is the Euclidean distance."""
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(3)
    p = rng.uniform(-80, 80, size=(13, 3)).astype(np.float32)
    q = rng.uniform(-80, 80, size=(9, 3)).astype(np.float32)
    A = np.repeat(p[:, None, :], 21, axis=1)
    B = np.repeat(q[:, None, :], 21, axis=1)
    dme, dd, dr = oracle.dme_matrix(A, B)
    ref = cdist(p.astype(np.float64), q.astype(np.float64))
    np.testing.assert_allclose(dme, ref, rtol=1e-15, atol=0)
    np.testing.assert_allclose(dd, ref, rtol=1e-15, atol=0)
    np.testing.assert_allclose(dr, ref, rtol=1e-15, atol=0)


def test_single_point_changes_each_coordinate():
    """Moving one point of b by a known vector changes only that point distance; checks every
    point index in both orientations (a wrong reversal index fails here)."""
    a = np.zeros((21, 3), np.float32)
    a[:, 0] = np.arange(21) * 0.01  # nearly a point: reversal distances stay below 0.2
    for i in range(21):
        for axis in range(3):
            b = a.copy()
            b[i, axis] += 7.0
            dme, dd, dr = oracle.dme_matrix(a[None], b[None])
            assert dd[0, 0] == pytest.approx(7.0, abs=1e-5)
            # reversed: point j pairs with b[20-j]; the moved point pairs with a[20-i]
            mv = b[i].astype(np.float64) - a[20 - i].astype(np.float64)
            assert dr[0, 0] == pytest.approx(np.linalg.norm(mv), abs=1e-5)


def test_identities():
    rng = np.random.default_rng(11)
    A = _rand_fibers(rng, 40)
    B = _rand_fibers(rng, 30)
    dAA, _, _ = oracle.dme_matrix(A, A)
    assert np.all(np.diag(dAA) == 0.0)
    dAB, ddAB, drAB = oracle.dme_matrix(A, B)
    dBA, ddBA, drBA = oracle.dme_matrix(B, A)
    np.testing.assert_array_equal(dAB, dBA.T)
    np.testing.assert_array_equal(ddAB, ddBA.T)
    # reversal: d(a, flip b) swaps the two orientation maxima; d(flip a, flip b) = d(a, b)
    dAfB, ddAfB, drAfB = oracle.dme_matrix(A, _rev(B).copy())
    np.testing.assert_array_equal(ddAfB, drAB)
    np.testing.assert_array_equal(drAfB, ddAB)
    dfAfB, _, _ = oracle.dme_matrix(_rev(A).copy(), _rev(B).copy())
    np.testing.assert_array_equal(dfAfB, dAB)
    # d(a, flip a) = 0
    dAfA, _, _ = oracle.dme_matrix(A, _rev(A).copy())
    assert np.all(np.diag(dAfA) == 0.0)


def test_triangle_inequality():
    rng = np.random.default_rng(5)
    X = _rand_fibers(rng, 25, scale=5.0)
    D, _, _ = oracle.dme_matrix(X, X)
    viol = D[:, None, :] - (D[:, :, None] + D[None, :, :])
    assert viol.max() <= 1e-9


def test_rigid_invariance():
    rng = np.random.default_rng(9)
    A = _rand_fibers(rng, 20).astype(np.float64)
    B = _rand_fibers(rng, 15).astype(np.float64)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    t = rng.normal(0, 10, size=3)
    D0, _, _ = oracle.dme_matrix(A.astype(np.float32), B.astype(np.float32))
    D1, _, _ = oracle.dme_matrix((A @ R.T + t).astype(np.float32), (B @ R.T + t).astype(np.float32))
    np.testing.assert_allclose(D1, D0, atol=2e-4)  # float32 rounding of the moved inputs


def _brute_by_sort(fib, cen, bundle_of, thr):
    """Independent labelling: list every (d_ME, bundle, centroid) candidate, drop the ones above
    their threshold, take the first in (distance, bundle, centroid) order."""
    fib = fib.astype(np.float64)
    cen = cen.astype(np.float64)
    out = []
    for f in range(fib.shape[0]):
        cands = []
        for c in range(cen.shape[0]):
            direct = np.sqrt(((fib[f] - cen[c]) ** 2).sum(axis=1)).max()
            flipped = np.sqrt(((fib[f] - cen[c][::-1]) ** 2).sum(axis=1)).max()
            d = min(direct, flipped)
            if d <= float(np.float32(thr[bundle_of[c]])):
                cands.append((d, int(bundle_of[c]), c))
        if cands:
            d, b, c = min(cands)
            out.append((b, d, c))
        else:
            out.append((-1, math.inf, -1))
    return out


def test_labels_vs_sorted_brute_force():
    rng = np.random.default_rng(21)
    cen = _rand_fibers(rng, 30, scale=6.0)
    bundle_of = rng.integers(0, 7, size=30).astype(np.int32)
    thr = rng.uniform(3, 9, size=7).astype(np.float32)
    fib = (cen[rng.integers(0, 30, size=60)] + rng.normal(0, 1.2, size=(60, 21, 3))).astype(
        np.float32)
    fib[::3] = fib[::3, ::-1]
    ref = _brute_by_sort(fib, cen, bundle_of, thr)
    for mode in ("brute", "cascade"):
        r = oracle.label(fib, cen, bundle_of, thr, mode)
        for f, (b, d, c) in enumerate(ref):
            assert r["labels"][f] == b
            assert r["cidx"][f] == c
            if b >= 0:
                assert r["dist"][f] == pytest.approx(d, rel=1e-15)
    assert sum(1 for x in ref if x[0] >= 0) > 10


def test_exact_ties_and_threshold_edges():
    """Distances landing exactly on thresholds and on each other (integer offsets)."""
    t = np.arange(21, dtype=np.float32)
    base = np.stack([t, 0 * t, 0 * t], axis=1)
    offs = [(0, 3, 4), (0, 0, 5), (0, 4, 3), (0, 0, 6), (0, 0, 2), (0, 2, 0)]
    cen = np.stack([base + np.array(o, np.float32) for o in offs] +
                   [base[::-1] + np.array(o, np.float32) for o in offs])  # reversed copies
    bundle_of = np.array([2, 1, 1, 0, 3, 3, 4, 5, 5, 6, 7, 7], np.int32)
    for thr in ([6.0, 5.0, 5.0, 1.9, 9, 9, 9, 9], [6.0, 5.0, 4.9, 2.0, 9, 9, 9, 9],
                [4.0, 4.0, 4.0, 4.0, 4.0, 4.0, 4.0, 4.0], [1, 1, 1, 1, 5.0, 5.0, 6.0, 1.9],
                [1, 1, 1, 1, 4.9, 5.0, 5.9, 2.0]):
        thr = np.array(thr, np.float32)
        ref = _brute_by_sort(base[None], cen, bundle_of, thr)
        for mode in ("brute", "cascade"):
            r = oracle.label(base[None], cen, bundle_of, thr, mode)
            assert (r["labels"][0], r["cidx"][0]) == (ref[0][0], ref[0][2])


def test_cascade_equals_brute_on_small_workload(small_workload):
    atlas, fib = small_workload
    rb = oracle.label(fib, atlas.centroids, atlas.bundle_of, atlas.thresholds, "brute")
    rc = oracle.label(fib, atlas.centroids, atlas.bundle_of, atlas.thresholds, "cascade")
    for k in ("labels", "dist", "cidx", "orient", "argmax"):
        np.testing.assert_array_equal(rb[k], rc[k])
    frac = (rb["labels"] >= 0).mean()
    assert 0.5 < frac < 0.95
    counts = rc["counts"]
    assert counts[4] == fib.shape[0] * atlas.M  # every pair reaches test1
    assert counts[0] == counts[4]  # one point distance per pair in test1
    assert counts[5] <= counts[4] and counts[6] <= counts[5] and counts[7] <= counts[6]


def test_nonfinite_fiber():
    rng = np.random.default_rng(1)
    cen = _rand_fibers(rng, 5)
    fib = cen[:3].copy()
    fib[1, 4, 2] = np.nan
    fib[2, 0, 0] = np.inf
    for mode in ("brute", "cascade"):
        r = oracle.label(fib, cen, np.zeros(5, np.int32), np.array([100.0], np.float32), mode)
        assert r["labels"][0] == 0 and r["dist"][0] == 0.0
        assert list(r["labels"][1:]) == [-1, -1]
        assert np.isnan(r["dist"][1:]).all()


def test_near_tie_flags():
    t = np.arange(21, dtype=np.float32)
    base = np.stack([t, 0 * t, 0 * t], axis=1)
    cen = np.stack([base + np.array(o, np.float32) for o in [(0, 0, 3), (0, 3.001, 0),
                                                               (0, 0, 20)]])
    bo = np.array([0, 1, 2], np.int32)
    fib = np.stack([base, base + np.array([0, 0, 18.0], np.float32),
                    base + np.array([0, 0, 8.0], np.float32)])
    thr = np.array([5.0, 5.0, 5.0], np.float32)
    r = oracle.label(fib, cen, bo, thr)
    flag = oracle.near_tie(fib, cen, bo, thr, r["labels"], r["dist"])
    # fiber 0: bundles 0 and 1 at 3 and 3.001 -> runner-up within 2e-3; fiber 1: bundle 2 at
    # 2; fiber 2: bundle 0 at 5 exactly = its threshold -> near threshold
    assert list(flag) == [1, 0, 1]
    thr2 = np.array([5.0, 5.0, 2.5], np.float32)
    r2 = oracle.label(fib, cen, bo, thr2)
    assert list(oracle.near_tie(fib, cen, bo, thr2, r2["labels"], r2["dist"])) == [1, 0, 1]


def test_near_tie_pruned_equals_brute(small_workload):
    """The pruned near-tie scan skips only centroids farther than theta + tol, which neither
    condition can use: its flags equal the full scan's on the hand-built cases above and on the
    whole 10,000-fiber x 1,000-centroid workload, at the parity tolerance and at a tolerance so
    wide that many fibers are flagged."""
    t = np.arange(21, dtype=np.float32)
    base = np.stack([t, 0 * t, 0 * t], axis=1)
    cen = np.stack([base + np.array(o, np.float32) for o in [(0, 0, 3), (0, 3.001, 0),
                                                               (0, 0, 20)]])
    bo = np.array([0, 1, 2], np.int32)
    fib = np.stack([base, base + np.array([0, 0, 18.0], np.float32),
                    base + np.array([0, 0, 8.0], np.float32)])
    for thr in (np.array([5.0, 5.0, 5.0], np.float32), np.array([5.0, 5.0, 2.5], np.float32)):
        r = oracle.label(fib, cen, bo, thr)
        a = oracle.near_tie(fib, cen, bo, thr, r["labels"], r["dist"])
        b = oracle.near_tie(fib, cen, bo, thr, r["labels"], r["dist"], pruned=True)
        assert list(a) == list(b)
    atlas, f = small_workload
    r = oracle.label(f, atlas.centroids, atlas.bundle_of, atlas.thresholds, "cascade")
    for tol in (2e-3, 1.0):
        a = oracle.near_tie(f, atlas.centroids, atlas.bundle_of, atlas.thresholds, r["labels"],
                            r["dist"], tol)
        b = oracle.near_tie(f, atlas.centroids, atlas.bundle_of, atlas.thresholds, r["labels"],
                            r["dist"], tol, pruned=True)
        np.testing.assert_array_equal(a, b)
        if tol > 0.1:
            assert a.sum() > 40


def test_dme_pairs_equals_matrix_diagonal():
    """One pair per fiber gives the diagonal of the full d_ME matrix; a negative index gives
    NaN."""
    rng = np.random.default_rng(5)
    fib = _rand_fibers(rng, 40)
    cen = _rand_fibers(rng, 40)
    d, dd, dr = oracle.dme_matrix(fib, cen)
    idx = np.arange(40, dtype=np.int32)
    p, pd, pr = oracle.dme_pairs(fib, cen, idx)
    np.testing.assert_array_equal(p, np.diagonal(d))
    np.testing.assert_array_equal(pd, np.diagonal(dd))
    np.testing.assert_array_equal(pr, np.diagonal(dr))
    idx[3] = -1
    p, _, _ = oracle.dme_pairs(fib, cen, idx)
    assert np.isnan(p[3]) and np.isfinite(np.delete(p, 3)).all()


def _line(step, n=21):
    t = np.arange(n, dtype=np.float64)
    return np.stack([step * t, 0 * t, 0 * t], axis=1)


def test_lengths_closed_forms():
    """Eq. 3's fiber and centroid lengths, read as the arc length of the 21-point polyline: a
    straight fiber with spacing s has length 20 s; 21 points on a circle of radius R at equal
    angle steps phi have length 20 * 2 R sin(phi / 2)."""
    R, phi = 7.0, 0.1
    t = np.arange(21)
    circ = np.stack([R * np.cos(phi * t), R * np.sin(phi * t), 0 * t], axis=1)
    ln = oracle.lengths(np.stack([_line(1.5), circ]).astype(np.float32))
    assert ln[0] == pytest.approx(30.0, abs=1e-12)
    assert ln[1] == pytest.approx(20 * 2 * R * np.sin(phi / 2), rel=1e-6)


def test_tn_worked_example():
    """Eq. 3 on a hand-computed pair: fiber x_i = i (length 20) and centroid x_i = 1.1 i (length
    22). The direct point distances are 0.1 i, so d_ME = 2.0 (point 20; the reversed maximum is
    22); TN = (|20 - 22| / 22 + 1)^2 - 1 = 23/121; D = 2 + 23/121 = 2.190082... With
    theta = 3 every classification labels the fiber (at D with TN); with theta = 2.1 Eq. 2
    alone passes it (2.0 <= 2.1 < D). The paper's direction inference picks the direct
    orientation here (end points 2.0 against 22)."""
    fib = _line(1.0)[None].astype(np.float32)
    cen = _line(1.1)[None].astype(np.float32)
    D = 2.0 + 23.0 / 121.0
    for th, want_tn in ((3.0, True), (2.1, False)):
        thr = np.array([th], np.float32)
        r = oracle.label_cls(fib, cen, [0], thr, "eq2")
        assert r["labels"][0] == 0 and r["dist"][0] == pytest.approx(2.0, abs=1e-5)
        for cls in ("eq2_tn", "paper"):
            r = oracle.label_cls(fib, cen, [0], thr, cls)
            if want_tn:
                assert r["labels"][0] == 0 and r["dist"][0] == pytest.approx(D, abs=1e-5)
                assert r["orient"][0] == 0
            else:
                assert r["labels"][0] == -1 and np.isinf(r["dist"][0])
    # equal lengths: TN = 0 and D = d_ME (a rigid translation keeps the length)
    r = oracle.label_cls(fib, fib + np.float32(1.5), [0], [3.0], "eq2_tn")
    assert r["dist"][0] == pytest.approx(np.sqrt(3 * 1.5 ** 2), abs=1e-6)


def test_direction_inference_can_miss_the_closer_orientation():
    """Section 2.4 infers the orientation from test2's end points and runs tests 3-4 in that
    orientation only. Fiber a: 21 points on 95% of a circle of radius 5 (end points 1.564 mm
    apart). Centroid b: a reversed in its interior (b_j = a_(20-j), 0 < j < 20) with its end
    points 0.5 mm above a's own (b_0 = a_0 + 0.5 z, b_20 = a_20 + 0.5 z). The end points favour
    the direct orientation (0.5 against sqrt(1.564^2 + 0.25)), but the direct interior pairs
    opposite sides of the loop (maximum near 10 mm), while the reversed interior matches
    exactly, so Eq. 2's d_ME is the reversed end-point distance. Eq. 2 (with or without TN)
    labels the fiber; the paper's algorithm discards the centroid and leaves it unlabelled."""
    R = 5.0
    ang = 2 * np.pi * 0.95 * np.arange(21) / 20
    a = np.stack([R * np.cos(ang), R * np.sin(ang), 0 * ang], axis=1)
    b = a[::-1].copy()
    b[0] = a[0] + [0, 0, 0.5]
    b[20] = a[20] + [0, 0, 0.5]
    a32, b32 = a.astype(np.float32)[None], b.astype(np.float32)[None]
    a64, b64 = a32[0].astype(np.float64), b32[0].astype(np.float64)
    dr = max(np.linalg.norm(a64[0] - b64[20]), np.linalg.norm(a64[20] - b64[0]))
    assert 1.6 < dr < 1.7
    thr = np.array([3.0], np.float32)
    r = oracle.label_cls(a32, b32, [0], thr, "eq2")
    assert r["labels"][0] == 0 and r["orient"][0] == 1
    assert r["dist"][0] == pytest.approx(dr, abs=1e-12)
    r = oracle.label_cls(a32, b32, [0], thr, "eq2_tn")
    assert r["labels"][0] == 0 and r["orient"][0] == 1 and r["dist"][0] > dr
    r = oracle.label_cls(a32, b32, [0], thr, "paper")
    assert r["labels"][0] == -1


def test_near_tie_cls_flags_ambiguous_direction():
    """A palindromic fiber (a_i = a_(20-i), a hairpin) sees the same end-point distances in
    both orientations, so an FP32 implementation may infer either: the paper classification
    flags it when the centroid passes; an unambiguous straight fiber is not flagged."""
    t = np.arange(21, dtype=np.float64)
    hair = np.stack([10 - np.abs(10 - t), 0 * t, 0 * t], axis=1)
    cen = hair.copy()
    cen[4] += [0, 0.8, 0]            # direct and reversed maxima differ: 0.8 against 0.8 at 16
    cen[16] += [0, 0.3, 0]
    fib = np.stack([hair, _line(1.0)]).astype(np.float32)
    cens = np.stack([cen, _line(1.0) + [0, 0, 1.0]]).astype(np.float32)
    thr = np.array([3.0, 3.0], np.float32)
    r = oracle.label_cls(fib, cens, [0, 1], thr, "paper")
    assert list(r["labels"]) == [0, 1]
    flag = oracle.near_tie_cls(fib, cens, [0, 1], thr, "paper", r["labels"], r["dist"])
    assert list(flag) == [1, 0]
    flag = oracle.near_tie_cls(fib, cens, [0, 1], thr, "eq2_tn", r["labels"], r["dist"])
    assert flag[1] == 0


def test_resample_closed_forms():
    """Arc-length resampling to 21 points (Section 2.3): a straight streamline with uneven
    vertex spacing resamples to x = k L / 20 exactly; 201 vertices at equal angle steps on a
    circle (200 equal chords) resample onto vertices 0, 10, ..., 200; a zero-length segment
    (a repeated vertex) changes nothing; a single point gives 21 copies; no point gives NaN."""
    line = np.array([[0, 0, 0], [1, 0, 0], [5, 0, 0], [5, 0, 0], [20, 0, 0]], np.float32)
    R = 9.0
    ang = np.linspace(0.0, 1.5 * np.pi, 201)
    circ = np.stack([R * np.cos(ang), R * np.sin(ang), 0 * ang], axis=1).astype(np.float32)
    single = np.array([[3, -2, 7]], np.float32)
    pts = np.concatenate([line, circ, single])
    off = np.array([0, 5, 206, 207, 207], np.int64)  # the last streamline has no point
    r = oracle.resample(pts, off)
    np.testing.assert_allclose(r[0, :, 0], np.arange(21.0), atol=1e-12)
    assert not r[0, :, 1:].any()
    np.testing.assert_allclose(r[1], circ[::10].astype(np.float64), atol=1e-5)
    np.testing.assert_array_equal(r[2], np.repeat(single.astype(np.float64), 21, axis=0))
    assert np.isnan(r[3]).all()
    # resampling an already equidistant 21-point fiber returns it
    t = np.arange(21, dtype=np.float32)
    fib = np.stack([2 * t, 0 * t, 0 * t], axis=1)
    np.testing.assert_allclose(oracle.resample(fib, [0, 21])[0], fib, atol=1e-12)


def test_multi_label_hand_cases():
    """Every bundle a fiber passes (Section 2.4): a straight fiber against parallel copies at
    distances 1 (bundle 2), 3 (bundle 0), 4.5 (bundle 1, threshold 4) and 6 (bundle 3,
    threshold 7): d_ME of a parallel offset is the offset, so the fiber passes bundles 0, 2 and
    3 (3 via a centroid farther than bundle 1's, which fails); the closest-bundle label is 2.
    A second fiber far from everything passes none; a bundle at exactly its threshold passes
    (d <= theta) and is flagged ambiguous."""
    line = _line(1.0)
    offs = [(0, 0, 3.0), (0, 4.5, 0), (0, 0, -1.0), (0, -6.0, 0), (5.0, 0, 0)]
    cen = np.stack([line + np.array(o) for o in offs]).astype(np.float32)
    bo = np.array([0, 1, 2, 3, 4], np.int32)
    thr = np.array([5.0, 4.0, 5.0, 7.0, 5.0], np.float32)  # bundle 4: exactly at theta
    fib = np.stack([line, line + [0, 0, 100.0]]).astype(np.float32)
    bits, amb = oracle.label_multi(fib, cen, bo, thr)
    assert bits.shape == (2, 1)
    assert bits[0, 0] == (1 << 0) | (1 << 2) | (1 << 3) | (1 << 4)
    assert bits[1, 0] == 0 and amb[1, 0] == 0
    assert amb[0, 0] == 1 << 4
    r = oracle.label(fib, cen, bo, thr)
    assert r["labels"][0] == 2
    # with TN (equal lengths: TN = 0) the same bundles
    bits_tn, _ = oracle.label_multi(fib, cen, bo, thr, "eq2_tn")
    np.testing.assert_array_equal(bits_tn, bits)


def test_grad_translation_closed_form():
    """One fiber, one centroid, translation only: dC/dt = u = r/|r| at the argmax point."""
    t = np.arange(21, dtype=np.float32)
    fib = np.stack([t, 0 * t, 0 * t], axis=1)[None]
    cen = fib.copy()
    cen[0, 13] += np.array([1.0, -2.0, 2.0], np.float32)  # argmax point 13, |r| = 3
    aff = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float64)
    g = oracle.grad(fib, aff, cen, [0], [10.0])
    assert g["cost"] == pytest.approx(3.0, abs=1e-12)
    u = -np.array([1.0, -2.0, 2.0]) / 3.0
    np.testing.assert_allclose(g["grad_affine"][9:], u, atol=1e-15)
    np.testing.assert_allclose(g["grad_affine"][:9].reshape(3, 3), np.outer(u, fib[0, 13]),
                               atol=1e-12)
    gc = np.zeros((1, 21, 3))
    gc[0, 13] = -u
    np.testing.assert_allclose(g["grad_centroids"], gc, atol=1e-15)
    assert g["argmax"][0] == 13 and g["orient"][0] == 0


def test_grad_reversed_orientation_closed_form():
    """Same as above with the centroid stored in reversed point order: the argmax fiber point
    13 pairs with centroid point 20 - 13 = 7 (Eq. 2 reversal), which takes the gradient."""
    t = np.arange(21, dtype=np.float32)
    fib = np.stack([t, 0 * t, 0 * t], axis=1)[None]
    cen = fib[:, ::-1].copy()
    cen[0, 7] += np.array([2.0, 1.0, -2.0], np.float32)
    aff = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0], np.float64)
    g = oracle.grad(fib, aff, cen, [0], [10.0])
    assert g["orient"][0] == 1 and g["argmax"][0] == 13
    assert g["cost"] == pytest.approx(3.0, abs=1e-12)
    u = -np.array([2.0, 1.0, -2.0]) / 3.0
    np.testing.assert_allclose(g["grad_affine"][9:], u, atol=1e-15)
    gc = np.zeros((1, 21, 3))
    gc[0, 7] = -u
    np.testing.assert_allclose(g["grad_centroids"], gc, atol=1e-15)


def _stable_case(seed=4, n=60, m=25):
    rng = np.random.default_rng(seed)
    cen = _rand_fibers(rng, m, scale=8.0)
    fib = (cen[rng.integers(0, m, size=n)] + rng.normal(0, 1.0, size=(n, 21, 3))).astype(
        np.float32)
    fib[::2] = fib[::2, ::-1]
    bo = (np.arange(m) % 5).astype(np.int32)
    thr = np.full(5, 6.0, np.float32)
    return fib, cen, bo, thr


def test_grad_frozen_structure_fd():
    """Central differences (h = 1e-3, Richardson-extrapolated with h/2 so the O(h^2) curvature
    term of |r| drops out) of the frozen-structure cost match the analytic gradient for the
    affine and the centroid coordinates."""
    fib, cen, bo, thr = _stable_case()
    aff = np.array([1.01, 0.02, -0.01, -0.015, 0.99, 0.03, 0.01, -0.02, 1.0, 0.5, -0.3, 0.2])
    g = oracle.grad(fib, aff, cen, bo, thr)
    frozen = (g["cidx"], g["orient"], g["argmax"])
    assert (g["cidx"] >= 0).sum() > 20

    def cost_aff(a):
        return oracle.grad(fib, a, cen, bo, thr, frozen=frozen, want_cen=False)["cost"]

    def richardson(f, x0, e, h):
        d1 = (f(x0 + h * e) - f(x0 - h * e)) / (2 * h)
        d2 = (f(x0 + 0.5 * h * e) - f(x0 - 0.5 * h * e)) / h
        return (4 * d2 - d1) / 3

    for k in range(12):
        e = np.zeros(12)
        e[k] = 1.0
        fd = richardson(cost_aff, aff, e, 1e-3)
        assert fd == pytest.approx(g["grad_affine"][k], rel=1e-6, abs=1e-6)
    rng = np.random.default_rng(0)
    used = np.unique(g["cidx"][g["cidx"] >= 0])
    c64 = cen.astype(np.float64)

    def cost_cen(flat):
        # steps are powers of two, so float32 holds the moved coordinates exactly
        return oracle.grad(fib, aff, flat.reshape(cen.shape).astype(np.float32), bo, thr,
                           frozen=frozen, want_cen=False)["cost"]

    for _ in range(12):
        c = int(rng.choice(used))
        p, ax = int(rng.integers(21)), int(rng.integers(3))
        e = np.zeros(c64.size)
        e[(c * 21 + p) * 3 + ax] = 1.0
        fd = richardson(cost_cen, c64.reshape(-1), e, 2.0 ** -8)
        assert fd == pytest.approx(g["grad_centroids"][c, p, ax], rel=1e-5, abs=1e-5)


def test_grad_free_structure_fd():
    """Central differences of the full forward (labels recomputed) agree on the affine gradient
    when no fiber changes its structure within +-h."""
    fib, cen, bo, thr = _stable_case(seed=8)
    aff = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1, 0.1, 0.2, -0.1], np.float64)
    g = oracle.grad(fib, aff, cen, bo, thr)
    h = 1e-4
    for k in range(12):
        e = np.zeros(12)
        e[k] = h
        gp = oracle.grad(fib, aff + e, cen, bo, thr, want_cen=False)
        gm = oracle.grad(fib, aff - e, cen, bo, thr, want_cen=False)
        same = all(np.array_equal(gp[x], g[x]) and np.array_equal(gm[x], g[x])
                   for x in ("cidx", "orient", "argmax"))
        if not same:
            continue
        fd = (gp["cost"] - gm["cost"]) / (2 * h)
        assert fd == pytest.approx(g["grad_affine"][k], rel=1e-5, abs=1e-5)
