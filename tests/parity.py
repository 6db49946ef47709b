"""Comparison of the CUDA path's labelling with the FP64 oracle at the stated tolerances:
distances within 1e-3 mm for every labelled fiber, identical labels for every decidable fiber
(oracle.near_tie at 2e-3 mm flags the others, which are counted), and a chosen centroid whose
own oracle distance is within 1e-3 mm of the oracle's best."""
import numpy as np

import oracle

DIST_TOL = 1e-3
TIE_TOL = 2e-3


def compare(fib, cen, bundle_of, thr, labels, dist, cidx=None, orient=None, nthreads=0):
    fib = np.ascontiguousarray(fib, np.float32)
    ref = oracle.label(fib, cen, bundle_of, thr, "brute", nthreads=nthreads)
    flag = oracle.near_tie(fib, cen, bundle_of, thr, ref["labels"], ref["dist"], TIE_TOL,
                           nthreads=nthreads)
    labels = np.asarray(labels)
    dist = np.asarray(dist, np.float64)
    dec = flag == 0
    bad = np.nonzero(dec & (labels != ref["labels"]))[0]
    assert bad.size == 0, (f"{bad.size} decidable label mismatches, first {bad[:5]}: gpu "
                           f"{labels[bad[:5]]} oracle {ref['labels'][bad[:5]]} "
                           f"dist {ref['dist'][bad[:5]]}")
    both = (labels >= 0) & (ref["labels"] >= 0)
    if both.any():
        err = np.abs(dist[both] - ref["dist"][both])
        assert err.max() <= DIST_TOL, f"max distance error {err.max()}"
    unl = labels < 0
    fin = np.isfinite(fib.reshape(len(fib), -1)).all(axis=1)
    assert np.all(np.isinf(dist[unl & fin])), "unlabelled fibers must have dist +inf"
    assert np.all(np.isnan(dist[~fin])), "non-finite fibers must have dist NaN"
    assert np.all(labels[~fin] == -1)
    if cidx is not None:
        cidx = np.asarray(cidx)
        assert np.all((cidx >= 0) == (labels >= 0))
        lab = np.nonzero(labels >= 0)[0]
        if lab.size:
            assert np.all(np.asarray(bundle_of)[cidx[lab]] == labels[lab])
            # the chosen centroid really is at the reported distance (both orientations)
            d, dd, dr = oracle.dme_matrix(fib[lab], np.asarray(cen)[cidx[lab]])
            own = np.diagonal(d)
            assert np.abs(own - dist[lab]).max() <= DIST_TOL
            if orient is not None:
                o = np.asarray(orient)[lab]
                od = np.where(o == 0, np.diagonal(dd), np.diagonal(dr))
                assert np.abs(od - dist[lab]).max() <= DIST_TOL
    return dict(near_ties=int(flag.sum()), n=len(fib), labelled=int((labels >= 0).sum()),
                ref=ref, flag=flag)


def compare_all(fib, cen, bundle_of, thr, labels, dist, cidx=None, orient=None, ref=None,
                count_ties: bool = True, nthreads=0):
    """Every fiber against the oracle's cascade (identical to the brute definition, pinned on
    the CPU), at sizes where the brute near-tie scan over all fibers would be too slow: the
    near-tie flag is computed exactly (oracle.near_tie, pruned) for the fibers whose labels
    differ, which must all be near-ties, and, if count_ties, for all fibers to report how many
    are not decidable. ref: a precomputed oracle.label(..., "cascade") result."""
    fib = np.ascontiguousarray(fib, np.float32)
    if ref is None:
        ref = oracle.label(fib, cen, bundle_of, thr, "cascade", nthreads=nthreads)
    labels = np.asarray(labels)
    dist = np.asarray(dist, np.float64)
    diff = np.nonzero(labels != ref["labels"])[0]
    if diff.size:
        fl = oracle.near_tie(fib[diff], cen, bundle_of, thr, ref["labels"][diff],
                             ref["dist"][diff], TIE_TOL, nthreads=nthreads, pruned=True)
        bad = diff[fl == 0]
        assert bad.size == 0, (f"{bad.size} decidable label mismatches, first {bad[:5]}: gpu "
                               f"{labels[bad[:5]]} oracle {ref['labels'][bad[:5]]}")
    both = (labels >= 0) & (ref["labels"] >= 0)
    if both.any():
        err = np.abs(dist[both] - ref["dist"][both])
        assert err.max() <= DIST_TOL, f"max distance error {err.max()}"
    fin = np.isfinite(fib.reshape(len(fib), -1)).all(axis=1)
    assert np.all(np.isinf(dist[(labels < 0) & fin]))
    assert np.all(np.isnan(dist[~fin])) and np.all(labels[~fin] == -1)
    if cidx is not None:
        cidx = np.asarray(cidx)
        assert np.all((cidx >= 0) == (labels >= 0))
        lab = np.nonzero(labels >= 0)[0]
        assert np.all(np.asarray(bundle_of)[cidx[lab]] == labels[lab])
        own, dd, dr = oracle.dme_pairs(fib[lab], cen, cidx[lab], nthreads=nthreads)
        assert np.abs(own - dist[lab]).max() <= DIST_TOL
        if orient is not None:
            o = np.asarray(orient)[lab]
            assert np.abs(np.where(o == 0, dd, dr) - dist[lab]).max() <= DIST_TOL
    ties = None
    if count_ties:
        ties = int(oracle.near_tie(fib, cen, bundle_of, thr, ref["labels"], ref["dist"],
                                   TIE_TOL, nthreads=nthreads, pruned=True).sum())
    return dict(n=len(fib), labelled=int((labels >= 0).sum()), mismatches=int(diff.size),
                near_ties=ties, ref=ref)
