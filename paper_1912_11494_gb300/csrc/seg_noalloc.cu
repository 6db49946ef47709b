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
// In host code the array's name is only a host-side stand-in, not a device address. The first
// call on each device looks up the array's device address with cudaGetSymbolAddress while that
// device is current and caches it; make that first call before any stream capture.
#include <mutex>

#include "seg_internal.cuh"
#include "seg_exact.cuh"

namespace seg {
namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_MAX_BLOCKS = 16384;
constexpr long long NA_MAX_FIBERS = NA_MAX_BLOCKS * NA_THREADS;  // 4,194,304
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_na_partials[NA_MAX_BLOCKS * 13];

std::mutex g_na_mu;
double* g_na_ptr[NA_MAX_DEVICES] = {};

struct NaAffine {
    float m[12];
};

__device__ __forceinline__ void na_affine_point(const NaAffine& T, const float* x, float* y) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        y[r] = fmaf(T.m[3 * r], x[0], fmaf(T.m[3 * r + 1], x[1], fmaf(T.m[3 * r + 2], x[2], T.m[9 + r])));
}

// One thread per fiber: the same per-fiber terms as seg_grad (argmax point of the saved
// orientation, u = r / |r|), summed per block in FP64 into partial[blockIdx.x].
__global__ void __launch_bounds__(NA_THREADS)
k_grad_na(const float* __restrict__ fib, long long n, NaAffine T, const int* __restrict__ cidx,
          const unsigned char* __restrict__ orient, AtlasView at, const int* __restrict__ inv_perm,
          float* __restrict__ grad_cen, double* __restrict__ partial) {
    double acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = 0.0;
    const long long f = (long long)blockIdx.x * NA_THREADS + threadIdx.x;
    if (f < n) {
        const int c = cidx[f];
        if (c >= 0 && c < at.M) {
            const int o = orient[f] ? 1 : 0;
            const float* x = fib + f * NC;
            const float* b = at.cen + (size_t)inv_perm[c] * CROW;
            float y[NC];
#pragma unroll
            for (int p = 0; p < NPTS; ++p) na_affine_point(T, x + 3 * p, y + 3 * p);
            float best = -1.0f;
            int is = 0;
#pragma unroll
            for (int i = 0; i < NPTS; ++i) {
                const float d2 = pd2(y, i, b, o ? NPTS - 1 - i : i);
                if (d2 > best) {
                    best = d2;
                    is = i;
                }
            }
            const int j = o ? NPTS - 1 - is : is;
            const float r0 = y[3 * is] - b[3 * j], r1 = y[3 * is + 1] - b[3 * j + 1],
                        r2 = y[3 * is + 2] - b[3 * j + 2];
            const float d = sqrtf(best);
            acc[12] = (double)d;
            if (d > 0.0f) {
                const float u[3] = {r0 / d, r1 / d, r2 / d};
                const float xs[3] = {x[3 * is], x[3 * is + 1], x[3 * is + 2]};
#pragma unroll
                for (int r = 0; r < 3; ++r) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) acc[3 * r + q] = (double)(u[r] * xs[q]);
                    acc[9 + r] = (double)u[r];
                    if (grad_cen) atomicAdd(grad_cen + ((size_t)c * NPTS + j) * 3 + r, -u[r]);
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

// Device address of g_na_partials for the current device, looked up once per device.
seg_status na_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return cuda_fail(e, "seg_grad_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES)
        return fail(SEG_ERR_UNSUPPORTED, "seg_grad_noalloc: device ordinal %d >= %d", dev,
                    NA_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_na_partials);
        if (e != cudaSuccess || !p)
            return cuda_fail(e ? e : cudaErrorInvalidSymbol,
                             "seg_grad_noalloc: cudaGetSymbolAddress of the static scratch");
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
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
    NaAffine T;
    for (int k = 0; k < 12; ++k) {
        if (!std::isfinite(h_aff[k]))
            return fail(SEG_ERR_INVALID_ARG, "seg_grad_noalloc: non-finite affine");
        T.m[k] = (float)h_aff[k];
    }
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
