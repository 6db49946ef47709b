// Affine transform of fibers and the adjoint of the segmentation cost (not in the paper).
//
// C(T) = sum over labelled fibers f of d_ME(T f, c_sigma(f)), T f = A f + t on every point. With
// the structure (centroid sigma, orientation o, argmax point i*) fixed, d_ME = |r| with
// r = T(a_i*) - c_pi(i*), pi(i) = i or 20 - i (Eq. 2), so
//   dC/dA_rc += u_r a_i*,c,  dC/dt_r += u_r,  dC/dc_pi(i*),r -= u_r,  u = r / |r|.
// Per-fiber terms are FP32. The sum over fibers of the 13 affine/cost terms is FP64 with a fixed
// assignment of fibers to threads and a fixed tree, so it is deterministic; the centroid gradient
// is an FP32 scatter-add.
#include "seg_internal.cuh"
#include "seg_exact.cuh"

namespace seg {
namespace {

struct Affine {
    float m[12];  // A row-major, then t
};

__device__ __forceinline__ void affine_point(const Affine& T, const float* x, float* y) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        y[r] = fmaf(T.m[3 * r], x[0], fmaf(T.m[3 * r + 1], x[1], fmaf(T.m[3 * r + 2], x[2], T.m[9 + r])));
}

__global__ void k_apply_affine(const float* __restrict__ in, long long npoints, Affine T,
                               float* __restrict__ out) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npoints;
         p += (long long)gridDim.x * blockDim.x) {
        float x[3] = {in[3 * p], in[3 * p + 1], in[3 * p + 2]};
        float y[3];
        affine_point(T, x, y);
        out[3 * p] = y[0];
        out[3 * p + 1] = y[1];
        out[3 * p + 2] = y[2];
    }
}

constexpr int GRAD_THREADS = 256;
constexpr int GRAD_BLOCKS = 1024;  // fixed, so the FP64 summation order never changes

__global__ void __launch_bounds__(GRAD_THREADS)
k_grad(const float* __restrict__ fib, long long n, Affine T, const int* __restrict__ cidx,
       const unsigned char* __restrict__ orient, AtlasView at, const int* __restrict__ inv_perm,
       float* __restrict__ grad_cen, double* __restrict__ partial) {
    double acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = 0.0;
    for (long long f = blockIdx.x * (long long)GRAD_THREADS + threadIdx.x; f < n;
         f += (long long)GRAD_BLOCKS * GRAD_THREADS) {
        const int c = cidx[f];
        if (c < 0 || c >= at.M) continue;
        const int o = orient[f] ? 1 : 0;
        const float* x = fib + f * NC;
        const float* b = at.cen + (size_t)inv_perm[c] * CROW;
        float y[NC];
#pragma unroll
        for (int p = 0; p < NPTS; ++p) affine_point(T, x + 3 * p, y + 3 * p);
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
        acc[12] += (double)d;
        if (d > 0.0f) {
            const float u[3] = {r0 / d, r1 / d, r2 / d};
            const float xs[3] = {x[3 * is], x[3 * is + 1], x[3 * is + 2]};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int q = 0; q < 3; ++q) acc[3 * r + q] += (double)(u[r] * xs[q]);
                acc[9 + r] += (double)u[r];
                if (grad_cen) atomicAdd(grad_cen + ((size_t)c * NPTS + j) * 3 + r, -u[r]);
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

bool load_affine(const double* h, Affine* T) {
    for (int k = 0; k < 12; ++k) {
        if (!std::isfinite(h[k])) return false;
        T->m[k] = (float)h[k];
    }
    return true;
}

}  // namespace

seg_status grad_launch(const AtlasView& at, const int* inv_perm, ScratchArena* scratch,
                       std::mutex* mu, const float* fib, long long n, const double* h_aff,
                       const int* cidx, const unsigned char* orient, double* grad_aff,
                       float* grad_cen, double* cost, cudaStream_t st) {
    Affine T;
    if (!load_affine(h_aff, &T)) return fail(SEG_ERR_INVALID_ARG, "seg_grad: non-finite affine");
    std::lock_guard<std::mutex> lock(*mu);
    void* buf = nullptr;
    seg_status s = scratch_acquire(scratch, sizeof(double) * GRAD_BLOCKS * 13, st, &buf);
    if (s != SEG_OK) return s;
    cudaError_t e = cudaSuccess;
    if (grad_cen)
        e = cudaMemsetAsync(grad_cen, 0, sizeof(float) * (size_t)at.M * NC, st);
    if (!e) {
        k_grad<<<GRAD_BLOCKS, GRAD_THREADS, 0, st>>>(fib, n, T, cidx, orient, at, inv_perm,
                                                     grad_cen, (double*)buf);
        e = cudaGetLastError();
    }
    if (!e) {
        k_grad_final<<<1, 13 * 32, 0, st>>>((const double*)buf, grad_aff, cost);
        e = cudaGetLastError();
    }
    seg_status r = scratch_release(scratch, st);
    if (e) return cuda_fail(e, "seg_grad");
    return r;
}

seg_status apply_affine_launch(const float* in, long long n, const double* h_aff, float* out,
                               cudaStream_t st) {
    Affine T;
    if (!load_affine(h_aff, &T))
        return fail(SEG_ERR_INVALID_ARG, "seg_apply_affine: non-finite affine");
    const long long np = n * NPTS;
    long long blocks = (np + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_apply_affine<<<(unsigned)blocks, 256, 0, st>>>(in, np, T, out);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "seg_apply_affine") : SEG_OK;
}

}  // namespace seg
