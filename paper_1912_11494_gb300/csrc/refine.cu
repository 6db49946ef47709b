// Subject-to-atlas affine refinement driven by the adjoint (not in the paper; the paper segments
// subjects already registered to the atlas). Each iteration runs the library's own path on the
// device: seg_apply_affine, seg_label and seg_grad, and reads back 12 gradient values, the cost
// and the number of labelled fibers.
//
// Objective: J(T) = sum over labelled fibers of d_ME(T f, c_sigma(f)) + P * (unlabelled fibers),
// P the largest bundle threshold. A fiber that becomes labelled lowers J (its d_ME <= theta <= P),
// so the optimiser cannot gain by moving fibers out of every bundle, and the gradient is
// seg_grad's (the penalty is piecewise constant). The 12 values are optimised in a centred and
// scaled frame, T x = A (x - m) + m + t' with m the fibers' mean point, variables (R A, t') with R
// their RMS radius about m, so that a unit step in any variable moves points by about 1 mm; the
// update is Adam's (per-variable normalised moments) with a learning rate in millimetres, halved
// whenever J does not improve on the best so far. The best T seen is returned.
#include <algorithm>
#include <cmath>

#include "seg_internal.cuh"

namespace seg {
namespace {

// Sums of the fibers' point coordinates and squared norms (FP32 per block, then atomics: only
// the preconditioning depends on them, never a result).
__global__ void k_point_moments(const float* __restrict__ fib, long long npoints,
                                float* __restrict__ acc) {
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npoints;
         p += (long long)gridDim.x * blockDim.x) {
        const float x = fib[3 * p], y = fib[3 * p + 1], z = fib[3 * p + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) continue;
        s[0] += x;
        s[1] += y;
        s[2] += z;
        s[3] += fmaf(x, x, fmaf(y, y, z * z));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float v = s[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(acc + k, v);
    }
}

__global__ void k_count_labelled(const int* __restrict__ cidx, long long n,
                                 unsigned long long* __restrict__ count) {
    unsigned long long c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        c += cidx[i] >= 0 ? 1ull : 0ull;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

}  // namespace

seg_status refine_launch(const seg_atlas* atlas, const AtlasView& at, ScratchArena* scratch,
                         std::mutex* mu, const float* fib, long long n, int mode, double* aff,
                         int iters, double step_mm, double penalty, double* cost_out,
                         int* iters_done, cudaStream_t st) {
    const size_t off_y = 0;
    const size_t off_lab = off_y + ((size_t)n * NC * 4 + 255) / 256 * 256;
    const size_t off_cidx = off_lab + ((size_t)n * 4 + 255) / 256 * 256;
    const size_t off_or = off_cidx + ((size_t)n * 4 + 255) / 256 * 256;
    const size_t off_small = off_or + ((size_t)n + 255) / 256 * 256;
    const size_t bytes = off_small + 256;
    std::lock_guard<std::mutex> lock(*mu);
    void* base = nullptr;
    seg_status s = scratch_acquire(scratch, bytes, st, &base);
    if (s != SEG_OK) return s;
    char* b = static_cast<char*>(base);
    float* y = reinterpret_cast<float*>(b + off_y);
    int* lab = reinterpret_cast<int*>(b + off_lab);
    int* cidx = reinterpret_cast<int*>(b + off_cidx);
    unsigned char* orient = reinterpret_cast<unsigned char*>(b + off_or);
    double* d_grad = reinterpret_cast<double*>(b + off_small);         // [12]
    double* d_cost = d_grad + 12;                                       // [1]
    unsigned long long* d_count = reinterpret_cast<unsigned long long*>(d_cost + 1);
    float* d_mom = reinterpret_cast<float*>(d_count + 1);               // [4]
    auto done = [&](seg_status r) {
        const seg_status rr = scratch_release(scratch, st);
        return r != SEG_OK ? r : rr;
    };
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMemsetAsync(d_mom, 0, 4 * sizeof(float), st);
    if (!e) {
        k_point_moments<<<sms * 8, 256, 0, st>>>(fib, n * NPTS, d_mom);
        e = cudaGetLastError();
    }
    float mom[4];
    if (!e) e = cudaMemcpyAsync(mom, d_mom, sizeof(mom), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return done(cuda_fail(e, "seg_refine_affine: moments"));
    const double np = (double)n * NPTS;
    const double m[3] = {mom[0] / np, mom[1] / np, mom[2] / np};
    const double R = std::sqrt(std::max(1e-6, mom[3] / np - (m[0] * m[0] + m[1] * m[1] +
                                                            m[2] * m[2])));
    // centred variables u = (R A row-major, t'), t' = t + A m - m
    auto to_u = [&](const double* a12, double* u) {
        for (int k = 0; k < 9; ++k) u[k] = R * a12[k];
        for (int r = 0; r < 3; ++r)
            u[9 + r] = a12[9 + r] + a12[3 * r] * m[0] + a12[3 * r + 1] * m[1] +
                       a12[3 * r + 2] * m[2] - m[r];
    };
    auto to_aff = [&](const double* u, double* a12) {
        for (int k = 0; k < 9; ++k) a12[k] = u[k] / R;
        for (int r = 0; r < 3; ++r)
            a12[9 + r] = u[9 + r] - (a12[3 * r] * m[0] + a12[3 * r + 1] * m[1] +
                                     a12[3 * r + 2] * m[2]) + m[r];
    };
    // J and its gradient in u at the affine a12
    auto evaluate = [&](const double* a12, double* J, double* gu) -> seg_status {
        seg_status r = seg_apply_affine(fib, n, a12, y, st);
        if (r == SEG_OK)
            r = seg_label(atlas, y, n, (seg_mode)mode, lab, nullptr, cidx, orient, st);
        if (r == SEG_OK)
            r = seg_grad(atlas, fib, n, a12, cidx, orient, d_grad, nullptr, d_cost, st);
        if (r != SEG_OK) return r;
        cudaError_t e2 = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st);
        if (!e2) {
            k_count_labelled<<<sms * 8, 256, 0, st>>>(cidx, n, d_count);
            e2 = cudaGetLastError();
        }
        double h[13];
        unsigned long long cnt = 0;
        if (!e2)
            e2 = cudaMemcpyAsync(h, d_grad, 13 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (!e2) e2 = cudaMemcpyAsync(&cnt, d_count, sizeof(cnt), cudaMemcpyDeviceToHost, st);
        if (!e2) e2 = cudaStreamSynchronize(st);
        if (e2) return cuda_fail(e2, "seg_refine_affine: evaluation");
        *J = h[12] + penalty * (double)(n - (long long)cnt);
        // chain rule to the centred variables: dJ/dt' = dJ/dt, dJ/d(R A_rc) = (dJ/dA_rc -
        // dJ/dt_r m_c) / R
        for (int r = 0; r < 3; ++r) {
            gu[9 + r] = h[9 + r];
            for (int c = 0; c < 3; ++c) gu[3 * r + c] = (h[3 * r + c] - h[9 + r] * m[c]) / R;
        }
        return SEG_OK;
    };
    double u[12], best_u[12], g[12], mv[12] = {0}, vv[12] = {0};
    to_u(aff, u);
    std::copy(u, u + 12, best_u);
    double J = 0.0, bestJ = 0.0, lr = step_mm;
    double a12[12];
    std::copy(aff, aff + 12, a12);
    s = evaluate(a12, &J, g);
    if (s != SEG_OK) return done(s);
    bestJ = J;
    if (cost_out) cost_out[0] = J;
    int it = 0;
    const double b1 = 0.9, b2 = 0.999;
    for (it = 1; it <= iters; ++it) {
        for (int k = 0; k < 12; ++k) {
            mv[k] = b1 * mv[k] + (1 - b1) * g[k];
            vv[k] = b2 * vv[k] + (1 - b2) * g[k] * g[k];
            const double mh = mv[k] / (1 - std::pow(b1, it)), vh = vv[k] / (1 - std::pow(b2, it));
            if (vh > 0.0) u[k] -= lr * mh / std::sqrt(vh);  // Adam's normalised step
        }
        to_aff(u, a12);
        s = evaluate(a12, &J, g);
        if (s != SEG_OK) return done(s);
        if (cost_out) cost_out[it] = J;
        if (J < bestJ) {
            bestJ = J;
            std::copy(u, u + 12, best_u);
        } else {
            lr *= 0.5;  // no improvement: shorter steps from here
        }
    }
    to_aff(best_u, aff);
    if (iters_done) *iters_done = it - 1;
    return done(SEG_OK);
}

}  // namespace seg
