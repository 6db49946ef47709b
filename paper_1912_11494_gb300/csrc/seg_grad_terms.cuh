// Per-fiber terms of the adjoint of the segmentation cost (not in the paper), shared by
// seg_grad and seg_grad_noalloc.
//
// C(T) = sum over labelled fibers f of d_ME(T f, c_sigma(f)), T f = A f + t on every point. With
// the structure (centroid sigma, orientation o, argmax point i*) fixed, d_ME = |r| with
// r = T(a_i*) - c_pi(i*), pi(i) = i or 20 - i (Eq. 2), and
//   dC/dA_rc += u_r a_i*,c,  dC/dt_r += u_r,  dC/dc_pi(i*),r -= u_r,  u = r / |r|.
//
// Accuracy. The argmax point is found on FP32 transformed points (the same arithmetic as
// seg_apply_affine, so it matches the forward pass). The residual r at that point is then
// recomputed with error-free FP32 transformations (Knuth's TwoSum, and the exact product error
// fma(a, x, -a*x)) over the affine split into FP32 high and low parts, so the cancellation
// between |T a| ~ 100 mm and |c| ~ 100 mm costs no digits: r comes out correctly rounded to
// within a few units of 2^-44 |T a|, and u, |r| and every per-fiber term carry a few FP32 ulps
// of relative error. All arithmetic here is FP32.
#pragma once

#include "seg_exact.cuh"

namespace seg {

struct AffineDS {
    float hi[12];  // A row-major, then t, rounded to FP32
    float lo[12];  // the FP32 rounding of (value - hi)
};

// FP32 transform of one point with the high part (seg_apply_affine's arithmetic).
__device__ __forceinline__ void affine_point_hi(const AffineDS& T, const float* x, float* y) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        y[r] = fmaf(T.hi[3 * r], x[0],
                    fmaf(T.hi[3 * r + 1], x[1], fmaf(T.hi[3 * r + 2], x[2], T.hi[9 + r])));
}

// s + e = a + b exactly (Knuth's TwoSum; the _rn intrinsics keep the compiler from fusing or
// reassociating).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Component r of T(x) - c, accurate to a few units of 2^-44 of the largest term.
__device__ __forceinline__ float residual_ds(const AffineDS& T, int r, const float* x, float c) {
    float s = T.hi[9 + r], err = 0.0f;
    float e;
    two_sum(s, -c, s, e);
    err = __fadd_rn(err, e);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p = __fmul_rn(T.hi[3 * r + k], x[k]);
        const float pe = __fmaf_rn(T.hi[3 * r + k], x[k], -p);  // exact product error
        two_sum(s, p, s, e);
        err = __fadd_rn(err, __fadd_rn(e, pe));
        err = __fmaf_rn(T.lo[3 * r + k], x[k], err);
    }
    err = __fadd_rn(err, T.lo[9 + r]);
    return __fadd_rn(s, err);
}

struct FiberGrad {
    bool valid;    // labelled fiber with a nonzero distance
    float d;       // |r| (0 for a labelled fiber on its centroid)
    int is;        // argmax point of the fiber
    int j;         // the centroid point it pairs with
    float u[3];    // r / |r|
    float x[3];    // the untransformed fiber point is
};

// b: the centroid's 63 coordinates; o: the saved orientation.
__device__ __forceinline__ FiberGrad fiber_grad(const AffineDS& T, const float* x, const float* b,
                                                int o) {
    float y[NC];
#pragma unroll
    for (int p = 0; p < NPTS; ++p) affine_point_hi(T, x + 3 * p, y + 3 * p);
    float best = -1.0f;
    int is = 0;
#pragma unroll
    for (int i = 0; i < NPTS; ++i) {
        const float d2 = pd2(y, i, b, o ? NPTS - 1 - i : i);
        if (d2 > best) {  // lowest index among equal maxima
            best = d2;
            is = i;
        }
    }
    FiberGrad g;
    g.is = is;
    g.j = o ? NPTS - 1 - is : is;
#pragma unroll
    for (int k = 0; k < 3; ++k) g.x[k] = x[3 * is + k];
    float r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = residual_ds(T, k, g.x, b[3 * g.j + k]);
    g.d = sqrtf(fmaf(r[0], r[0], fmaf(r[1], r[1], r[2] * r[2])));
    g.valid = g.d > 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) g.u[k] = g.valid ? r[k] / g.d : 0.0f;
    return g;
}

// Host: split the caller's FP64 affine into FP32 high and low parts; false if not finite.
inline bool split_affine(const double* h, AffineDS* T) {
    for (int k = 0; k < 12; ++k) {
        if (!std::isfinite(h[k])) return false;
        T->hi[k] = (float)h[k];
        T->lo[k] = (float)(h[k] - (double)T->hi[k]);
    }
    return true;
}

}  // namespace seg
