// seg_grad_noalloc: the gradient of seg_grad for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a host-side allocator
// callback, a plugin whose host framework owns every device allocation, or a process whose
// device memory is fully reserved up front. seg_grad needs a small FP64 scratch buffer for its
// cross-fiber reduction and takes it from the atlas's growable arena, which may allocate. This
// entry point keeps that scratch in a fixed array compiled into the library instead, so it
// allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
//
// The array holds one 13-value FP64 partial sum per block of 256 fibers, so one call handles at
// most NA_MAX_BLOCKS * 256 = 4,194,304 fibers; larger calls are rejected. Every GPU that loads
// the library holds the array (1.7 MB) until the process exits. All calls share it, so calls
// whose work overlaps on the GPU race on it (serialize them, e.g. on one stream). Every call
// writes every slot it later reads, so nothing needs clearing between calls.
//
// In host code the array's name is only a host-side stand-in, not a device address. Every call
// looks up the array's device address with cudaGetSymbolAddress while the caller's device is
// current (the first call on a device may load the module there; make that first call before
// any stream capture).
#include "seg_internal.cuh"
#include "seg_grad_terms.cuh"

namespace seg {
namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_MAX_BLOCKS = 16384;
constexpr long long NA_MAX_FIBERS = NA_MAX_BLOCKS * NA_THREADS;  // 4,194,304

static __device__ __align__(256) double g_na_partials[NA_MAX_BLOCKS * 13];

// One thread per fiber: the per-fiber terms of seg_grad (fiber_grad), summed per block in FP64
// into partial[blockIdx.x]; the centroid gradient is an FP32 atomic sum (seg_grad sums it in
// fixed point, which needs scratch sized by the atlas).
__global__ void __launch_bounds__(NA_THREADS)
k_grad_na(const float* __restrict__ fib, long long n, AffineDS T, const int* __restrict__ cidx,
          const unsigned char* __restrict__ orient, AtlasView at, const int* __restrict__ inv_perm,
          float* __restrict__ grad_cen, double* __restrict__ partial) {
    double acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = 0.0;
    const long long f = (long long)blockIdx.x * NA_THREADS + threadIdx.x;
    if (f < n) {
        const int c = cidx[f];
        if (c >= 0 && c < at.M) {
            const float* b = at.cen + (size_t)inv_perm[c] * CROW;
            const FiberGrad g = fiber_grad(T, fib + f * NC, b, orient[f] ? 1 : 0);
            acc[12] = (double)g.d;
            if (g.valid) {
#pragma unroll
                for (int r = 0; r < 3; ++r) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) acc[3 * r + q] = (double)(g.u[r] * g.x[q]);
                    acc[9 + r] = (double)g.u[r];
                    if (grad_cen)
                        atomicAdd(grad_cen + ((size_t)c * NPTS + g.j) * 3 + r, -g.u[r]);
                }
            }
        }
    }
    __shared__ double red[NA_THREADS / 32][13];
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
        for (int w = 0; w < NA_THREADS / 32; ++w) v += red[w][threadIdx.x];
        partial[blockIdx.x * 13 + threadIdx.x] = v;
    }
}

// Fixed-order sum of the nb block partials (one warp per value): deterministic.
__global__ void k_grad_na_final(const double* __restrict__ partial, int nb,
                                double* __restrict__ grad_aff, double* __restrict__ cost) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 13) return;
    double v = 0.0;
    for (int b = lane; b < nb; b += 32) v += partial[b * 13 + k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) {
        if (k < 12)
            grad_aff[k] = v;
        else if (cost)
            *cost = v;
    }
}

// Device address of g_na_partials in the current device's copy of the module. Looked up on
// every call (cheap once the module is loaded), so a device reset that reloads the module at
// another address is harmless.
seg_status na_scratch(double** out) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_na_partials);
    if (e != cudaSuccess || !p)
        return cuda_fail(e ? e : cudaErrorInvalidSymbol,
                         "seg_grad_noalloc: cudaGetSymbolAddress of the static scratch");
    *out = p;
    return SEG_OK;
}

}  // namespace

seg_status grad_noalloc_launch(const AtlasView& at, const int* inv_perm, const float* fib,
                               long long n, const double* h_aff, const int* cidx,
                               const unsigned char* orient, double* grad_aff, float* grad_cen,
                               double* cost, cudaStream_t st) {
    if (n > NA_MAX_FIBERS)
        return fail(SEG_ERR_INVALID_ARG,
                    "seg_grad_noalloc: n=%lld exceeds the static scratch limit of %lld fibers "
                    "per call",
                    (long long)n, (long long)NA_MAX_FIBERS);
    AffineDS T;
    if (!split_affine(h_aff, &T))
        return fail(SEG_ERR_INVALID_ARG, "seg_grad_noalloc: non-finite affine");
    double* partial = nullptr;
    seg_status s = na_scratch(&partial);
    if (s != SEG_OK) return s;
    const int nb = (int)((n + NA_THREADS - 1) / NA_THREADS);
    cudaError_t e = cudaSuccess;
    if (grad_cen) e = cudaMemsetAsync(grad_cen, 0, sizeof(float) * (size_t)at.M * NC, st);
    if (!e && nb > 0) {
        k_grad_na<<<nb, NA_THREADS, 0, st>>>(fib, n, T, cidx, orient, at, inv_perm, grad_cen,
                                              partial);
        e = cudaGetLastError();
    }
    if (!e) {
        k_grad_na_final<<<1, 13 * 32, 0, st>>>(partial, nb, grad_aff, cost);
        e = cudaGetLastError();
    }
    return e ? cuda_fail(e, "seg_grad_noalloc") : SEG_OK;
}

}  // namespace seg
