// Exact FP32 d_ME^2 of one (fiber, centroid) pair with progressive discarding.
//
// Section 2.3: test1 uses the centre point, which serves both orientations (point 10 pairs with
// 20 - 10 = 10); test2 the end points, per orientation; test3 four intermediate points; test4 all
// remaining points. An orientation stops as soon as its partial maximum exceeds the bound
// (Section 2.4 evaluates the discarding criterion after each point distance; here after each
// stage, which discards the same pairs). Squared distances throughout, no sqrt (the maximum of
// squares is the square of the maximum).
#pragma once

#include "seg_common.cuh"

namespace seg {

__device__ __forceinline__ float pd2(const float* a, int i, const float* b, int j) {
    float dx = a[3 * i] - b[3 * j];
    float dy = a[3 * i + 1] - b[3 * j + 1];
    float dz = a[3 * i + 2] - b[3 * j + 2];
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Points of test3 (any choice is exact; these spread between the centre and the ends).
__device__ __forceinline__ int test3_point(int q) {
    return q == 0 ? 5 : q == 1 ? 15 : q == 2 ? 3 : 17;
}

__device__ __forceinline__ bool is_early_point(int i) {
    return i == 0 || i == 3 || i == 5 || i == CENTRE || i == 15 || i == 17 || i == NPTS - 1;
}

// Polyline arc length of 21 points (FP32, fixed order): the l_S / l_C of Eq. 3.
__device__ __forceinline__ float poly_length(const float* a) {
    float l = 0.0f;
#pragma unroll
    for (int i = 0; i + 1 < NPTS; ++i) l += sqrtf(pd2(a, i, a, i + 1));
    return l;
}

// Eq. 3: TN = (|l_S - l_C| / max(l_S, l_C) + 1)^2 - 1 = t (t + 2), t the relative difference;
// two zero lengths give 0.
__device__ __forceinline__ float tn_term(float ls, float lc) {
    const float m = fmaxf(ls, lc);
    const float t = m > 0.0f ? fabsf(ls - lc) / m : 0.0f;
    return t * (t + 2.0f);
}

// Classifications (AtlasView::cls): 0 Eq. 2; 1 Eq. 2 + TN; 2 the paper's new algorithm
// (direction inferred from test2, TN). With TN the packed key holds the classification
// distance D = d + TN itself (non-negative floats order as their bits) instead of d^2.
constexpr int CLS_EQ2 = 0, CLS_EQ2_TN = 1, CLS_PAPER = 2;

// Bound on a candidate's squared point distances implied by the best key value so far: any
// pair with d^2 above it cannot beat that key (D >= d), rounded up so exits stay strict. NaN
// (no key yet) stays NaN, which fminf ignores.
__device__ __forceinline__ float key_bound2(float kf, int cls) {
    return cls == CLS_EQ2 ? kf : __fmul_ru(kf, kf);
}

// The key value of a pair whose exact d^2 (in its orientation) passed the bound: d^2, or with
// TN D = d + TN, which must itself pass theta (lazy TN: computed only here). False when it
// fails.
__device__ __forceinline__ bool key_value(int cls, float d2, float thr2, float ls, float lc,
                                          float& kf) {
    if (cls == CLS_EQ2) {
        kf = d2;
        return true;
    }
    kf = sqrtf(d2) + tn_term(ls, lc);
    return kf <= sqrtf(thr2);  // sqrtf(theta * theta) is theta again in IEEE arithmetic
}

// a: fiber coordinates (63, registers or shared); b: centroid coordinates (63).
// Returns true when min over orientations of max_i d^2 <= bound2, with d2 = that minimum and
// o = 0 (direct) or 1 (reversed, only when strictly smaller). With cls == CLS_PAPER the
// orientation is inferred from test2's end points (the smaller partial maximum, ties direct,
// Section 2.4) and tests 3-4 run in that orientation only.
__device__ __forceinline__ bool exact_pair(const float* a, const float* b, float bound2,
                                           float& d2, int& o, int cls = CLS_EQ2) {
    float c = pd2(a, CENTRE, b, CENTRE);
    if (!(c <= bound2)) return false;
    float md = fmaxf(c, fmaxf(pd2(a, 0, b, 0), pd2(a, NPTS - 1, b, NPTS - 1)));
    float mr = fmaxf(c, fmaxf(pd2(a, 0, b, NPTS - 1), pd2(a, NPTS - 1, b, 0)));
    bool ad = md <= bound2, ar = mr <= bound2;
    if (cls == CLS_PAPER) {
        const bool direct = md <= mr;
        ad = ad && direct;
        ar = ar && !direct;
    }
    if (!(ad || ar)) return false;
    if (ad) {
#pragma unroll
        for (int q = 0; q < 4; ++q) md = fmaxf(md, pd2(a, test3_point(q), b, test3_point(q)));
        ad = md <= bound2;
    }
    if (ar) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            mr = fmaxf(mr, pd2(a, test3_point(q), b, NPTS - 1 - test3_point(q)));
        ar = mr <= bound2;
    }
    if (!(ad || ar)) return false;
    if (ad) {
#pragma unroll
        for (int i = 1; i < NPTS - 1; ++i)
            if (!is_early_point(i)) md = fmaxf(md, pd2(a, i, b, i));
        ad = md <= bound2;
    }
    if (ar) {
#pragma unroll
        for (int i = 1; i < NPTS - 1; ++i)
            if (!is_early_point(i)) mr = fmaxf(mr, pd2(a, i, b, NPTS - 1 - i));
        ar = mr <= bound2;
    }
    if (!(ad || ar)) return false;
    if (ad && (!ar || md <= mr)) {
        d2 = md;
        o = 0;
    } else {
        d2 = mr;
        o = 1;
    }
    return true;
}

}  // namespace seg
