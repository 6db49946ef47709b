// Affine transform of fibers and the adjoint of the segmentation cost (not in the paper).
//
// C(T) = sum over labelled fibers f of d_ME(T f, c_sigma(f)); the per-fiber terms (argmax point,
// residual, unit vector) are computed in FP32 by fiber_grad (seg_grad_terms.cuh), with the
// residual recovered by error-free transformations. The sum over fibers of the 13 affine/cost
// terms is FP64 with a fixed assignment of fibers to threads and a fixed tree, so it is
// deterministic. The centroid gradient is summed exactly: each term -u_r is rounded to a
// multiple of 2^-36 and added as a 64-bit integer (integer addition is exact and does not depend
// on the order), then each coordinate is converted to FP32 once; so the centroid gradient is
// deterministic and within half an FP32 ulp plus count x 2^-37 of the sum of the FP32 terms.
#include <algorithm>

#include "seg_internal.cuh"
#include "seg_grad_terms.cuh"

namespace seg {
namespace {

__global__ void k_apply_affine(const float* __restrict__ in, long long npoints, AffineDS T,
                               float* __restrict__ out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npoints;
         p += (long long)gridDim.x * blockDim.x) {
        float x[3] = {in[3 * p], in[3 * p + 1], in[3 * p + 2]};
        float y[3];
        affine_point_hi(T, x, y);
        out[3 * p] = y[0];
        out[3 * p + 1] = y[1];
        out[3 * p + 2] = y[2];
    }
}

constexpr int GRAD_THREADS = 256;
constexpr int GRAD_BLOCKS = 1024;  // fixed, so the FP64 summation order never changes
constexpr float CEN_SCALE = 68719476736.0f;  // 2^36: fixed point of the centroid gradient
// |term| <= 1, so 2^27 contributions to one coordinate stay below 2^63
constexpr long long GRAD_MAX_FIBERS = 1LL << 27;

__global__ void __launch_bounds__(GRAD_THREADS)
k_grad(const float* __restrict__ fib, long long n, AffineDS T, const int* __restrict__ cidx,
       const unsigned char* __restrict__ orient, AtlasView at, const int* __restrict__ inv_perm,
       unsigned long long* __restrict__ gcen_fx, double* __restrict__ partial) {
    double acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = 0.0;
    for (long long f = blockIdx.x * (long long)GRAD_THREADS + threadIdx.x; f < n;
         f += (long long)GRAD_BLOCKS * GRAD_THREADS) {
        const int c = cidx[f];
        if (c < 0 || c >= at.M) continue;
        const float* b = at.cen + (size_t)inv_perm[c] * CROW;
        const FiberGrad g = fiber_grad(T, fib + f * NC, b, orient[f] ? 1 : 0);
        acc[12] += (double)g.d;
        if (!g.valid) continue;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[3 * r + q] += (double)(g.u[r] * g.x[q]);
            acc[9 + r] += (double)g.u[r];
            if (gcen_fx) {
                const long long v = __float2ll_rn(-g.u[r] * CEN_SCALE);
                atomicAdd(gcen_fx + ((size_t)c * NPTS + g.j) * 3 + r, (unsigned long long)v);
            }
        }
    }
    __shared__ double red[GRAD_THREADS / 32][13];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
        double v = 0.0;
        for (int w = 0; w < GRAD_THREADS / 32; ++w) v += red[w][threadIdx.x];
        partial[blockIdx.x * 13 + threadIdx.x] = v;
    }
}

__global__ void k_grad_final(const double* __restrict__ partial, double* __restrict__ grad_aff,
                             double* __restrict__ cost) {
    // one warp per output value, fixed order: deterministic
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 13) return;
    double v = 0.0;
    for (int b = lane; b < GRAD_BLOCKS; b += 32) v += partial[b * 13 + k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) {
        if (k < 12)
            grad_aff[k] = v;
        else if (cost)
            *cost = v;
    }
}

// Fixed point -> FP32: the integer is rounded to FP32 once, then scaled by 2^-36 (exact).
__global__ void k_grad_cen_out(const unsigned long long* __restrict__ gcen_fx, long long count,
                               float* __restrict__ grad_cen) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        grad_cen[i] = __ll2float_rn((long long)gcen_fx[i]) * (1.0f / CEN_SCALE);
}

}  // namespace

seg_status grad_launch(const AtlasView& at, const int* inv_perm, ScratchArena* scratch,
                       std::mutex* mu, const float* fib, long long n, const double* h_aff,
                       const int* cidx, const unsigned char* orient, double* grad_aff,
                       float* grad_cen, double* cost, cudaStream_t st) {
    AffineDS T;
    if (!split_affine(h_aff, &T)) return fail(SEG_ERR_INVALID_ARG, "seg_grad: non-finite affine");
    if (n > GRAD_MAX_FIBERS)
        return fail(SEG_ERR_INVALID_ARG, "seg_grad: n=%lld exceeds %lld fibers per call", n,
                    GRAD_MAX_FIBERS);
    const size_t part_bytes = sizeof(double) * GRAD_BLOCKS * 13;
    const long long ncoord = (long long)at.M * NC;
    const size_t bytes = part_bytes + (grad_cen ? sizeof(unsigned long long) * ncoord : 0);
    std::lock_guard<std::mutex> lock(*mu);
    void* buf = nullptr;
    seg_status s = scratch_acquire(scratch, bytes, st, &buf);
    if (s != SEG_OK) return s;
    unsigned long long* gfx =
        grad_cen ? reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + part_bytes)
                 : nullptr;
    cudaError_t e = cudaSuccess;
    if (gfx) e = cudaMemsetAsync(gfx, 0, sizeof(unsigned long long) * ncoord, st);
    if (!e) {
        k_grad<<<GRAD_BLOCKS, GRAD_THREADS, 0, st>>>(fib, n, T, cidx, orient, at, inv_perm, gfx,
                                                     (double*)buf);
        e = cudaGetLastError();
    }
    if (!e) {
        k_grad_final<<<1, 13 * 32, 0, st>>>((const double*)buf, grad_aff, cost);
        e = cudaGetLastError();
    }
    if (!e && gfx) {
        const long long blocks = std::min<long long>((ncoord + 255) / 256, 152 * 8);
        k_grad_cen_out<<<(unsigned)blocks, 256, 0, st>>>(gfx, ncoord, grad_cen);
        e = cudaGetLastError();
    }
    seg_status r = scratch_release(scratch, st);
    if (e) return cuda_fail(e, "seg_grad");
    return r;
}

seg_status apply_affine_launch(const float* in, long long n, const double* h_aff, float* out,
                               cudaStream_t st) {
    AffineDS T;
    if (!split_affine(h_aff, &T))
        return fail(SEG_ERR_INVALID_ARG, "seg_apply_affine: non-finite affine");
    const long long np = n * NPTS;
    long long blocks = (np + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_apply_affine<<<(unsigned)blocks, 256, 0, st>>>(in, np, T, out);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "seg_apply_affine") : SEG_OK;
}

}  // namespace seg
