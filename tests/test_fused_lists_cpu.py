"""The fused kernel's per-warp lists, replayed on the CPU.

A warp of SEG_MODE_CULLED_FUSED keeps two lists in shared memory, 64 entries each: the test1
survivors waiting for test2 (filled column by column after each chunk's test1; whenever 32 or
more wait, the newest 32 go through one round of test2) and the pairs that passed test2 waiting
for test3/test4 (whenever 32 or more wait, the newest 32 go through one round). At the end of a
group the rest of each list runs as one partial round. This test replays that bookkeeping on
random and extreme survivor masks (every fiber passing every centroid of every chunk, single
survivors, empty chunks) and checks that neither list ever holds more than its 64 entries and
that every survivor reaches test2 exactly once and every test2 pass reaches test3 exactly once.
"""
import numpy as np
import pytest

CAP = 64


def replay(masks, passes_test2):
    """masks: per chunk, 32 uint32 test1 masks (lane = fiber, bit = column). passes_test2:
    the set of (chunk, column, fiber) that pass test2. Returns the pairs seen by test2 and
    test3 and the largest fill of each list."""
    al, qe = [], []
    seen2, seen3 = [], []
    peak_a = peak_q = 0

    def test3_round(entries):
        seen3.extend(entries)

    def test2_round(entries):
        nonlocal qe, peak_q
        seen2.extend(entries)
        qe = qe + [e for e in entries if e in passes_test2]
        peak_q = max(peak_q, len(qe))
        assert len(qe) <= CAP
        if len(qe) >= 32:
            test3_round(qe[-32:])
            qe = qe[:-32]

    for cc, m in enumerate(masks):
        cols = 0
        for v in m:
            cols |= int(v)
        for b in range(32):
            if not (cols >> b) & 1:
                continue
            for lane in range(32):
                if (int(m[lane]) >> b) & 1:
                    al.append((cc, b, lane))
            peak_a = max(peak_a, len(al))
            assert len(al) <= CAP
            if len(al) >= 32:
                test2_round(al[-32:])
                al = al[:-32]
    if al:
        test2_round(al)
    if qe:
        test3_round(qe)
    return seen2, seen3, peak_a, peak_q


@pytest.mark.parametrize("case", ["random", "dense", "single", "mixed"])
def test_lists_never_overflow_and_lose_nothing(case):
    rng = np.random.default_rng({"random": 1, "dense": 2, "single": 3, "mixed": 4}[case])
    n_chunks = 40
    if case == "random":
        masks = rng.integers(0, 2 ** 32, (n_chunks, 32), dtype=np.uint64) & \
            rng.integers(0, 2 ** 32, (n_chunks, 32), dtype=np.uint64)
    elif case == "dense":
        masks = np.full((n_chunks, 32), 0xFFFFFFFF, dtype=np.uint64)
    elif case == "single":
        masks = np.zeros((n_chunks, 32), dtype=np.uint64)
        masks[np.arange(n_chunks), rng.integers(0, 32, n_chunks)] = \
            np.uint64(1) << rng.integers(0, 32, n_chunks).astype(np.uint64)
    else:
        masks = np.where(rng.random((n_chunks, 1)) < 0.3, np.uint64(0xFFFFFFFF),
                         rng.integers(0, 2 ** 32, (n_chunks, 32), dtype=np.uint64)
                         & rng.integers(0, 2 ** 32, (n_chunks, 32), dtype=np.uint64)
                         & rng.integers(0, 2 ** 32, (n_chunks, 32), dtype=np.uint64))
        masks[rng.random(n_chunks) < 0.2] = 0
    pairs = {(cc, b, lane) for cc in range(n_chunks) for lane in range(32) for b in range(32)
             if (int(masks[cc, lane]) >> b) & 1}
    passes = {p for p in pairs if rng.random() < 0.4}
    seen2, seen3, peak_a, peak_q = replay(masks, passes)
    assert sorted(seen2) == sorted(pairs)          # each survivor reaches test2 exactly once
    assert sorted(seen3) == sorted(passes)         # each test2 pass reaches test3 exactly once
    assert peak_a <= CAP and peak_q <= CAP
