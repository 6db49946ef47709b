// Resampling of raw streamlines to 21 arc-length-equidistant points (Section 2.3 works on fibers
// of 21 equidistant points), ahead of the labelling.
//
// One warp per streamline (CSR: points [P][3], offsets [n+1]). The lanes read 32 consecutive
// points at a time (coalesced), each lane measures one segment, and a warp scan gives the
// segments' cumulative arc lengths; the running total across chunks is carried as an
// unevaluated FP32 sum (TwoSum), so the cumulative lengths keep FP32 accuracy over thousands of
// segments. Pass 1 computes the total length L; pass 2 repeats the same arithmetic and the lane
// whose segment interval (c_j, c_j+1] holds s_k = k L / 20 writes output point k by linear
// interpolation (exactly one lane per target: the intervals tile (0, L]); points 0 and 20 are
// the streamline's end points. A streamline with one point or zero length gives 21 copies of its first point,
// one with no points NaN. The second pass mostly hits L2 (a warp's streamline is a few KB).
#include <algorithm>

#include "seg_internal.cuh"

namespace seg {
namespace {

constexpr int RS_WARPS = 8;

__device__ __forceinline__ void rs_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The warp's pass over the segments of points p[0 .. m-1]: calls emit(c0, c1, len, pj, pj1) for
// every segment (lane-parallel, 32 at a time) with its interval (c0, c1] of cumulative arc
// length, and returns the total length L. The interval ends are a running maximum of the
// rounded cumulative sums, so they never decrease and the intervals tile (0, L] exactly: every
// s in (0, L] lies in exactly one of them (rounding cannot drop or duplicate a target). Both
// passes run the identical arithmetic, so they see the same intervals and the same L.
template <class Emit>
__device__ __forceinline__ float segment_pass(const float* __restrict__ p, long long m, int lane,
                                              Emit emit) {
    float hi = 0.0f, lo = 0.0f;  // running total hi + lo of the segment lengths
    float top = 0.0f;            // the largest interval end so far
    for (long long base = 0; base + 1 < m; base += 32) {
        const long long j = base + lane;
        float a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f}, len = 0.0f;
        if (j + 1 < m) {
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                a[r] = __ldg(p + 3 * j + r);
                b[r] = __ldg(p + 3 * (j + 1) + r);
            }
            const float dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
            len = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
        float incl = len;  // inclusive scan of the chunk's segment lengths
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        float c1 = fmaxf(top, hi + (lo + incl));  // running maximum of the ends
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float v = __shfl_up_sync(0xffffffffu, c1, off);
            if (lane >= off) c1 = fmaxf(c1, v);
        }
        float c0 = __shfl_up_sync(0xffffffffu, c1, 1);
        if (lane == 0) c0 = top;
        if (j + 1 < m) emit(c0, c1, len, a, b);
        const float chunk = __shfl_sync(0xffffffffu, incl, 31);
        top = __shfl_sync(0xffffffffu, c1, 31);
        float e;
        rs_two_sum(hi, chunk, hi, e);
        lo += e;
    }
    return top;
}

__global__ void __launch_bounds__(RS_WARPS * 32)
k_resample(const float* __restrict__ pts, const long long* __restrict__ off, long long n,
           float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long W = (long long)gridDim.x * RS_WARPS;
    for (long long f = (long long)blockIdx.x * RS_WARPS + (threadIdx.x >> 5); f < n; f += W) {
        const long long p0 = off[f], m = off[f + 1] - p0;
        float* o = out + f * NC;
        if (m <= 0) {
            for (int k = lane; k < NC; k += 32) o[k] = NAN;
            continue;
        }
        const float* p = pts + 3 * p0;
        const float L = segment_pass(p, m, lane, [](float, float, float, const float*,
                                                    const float*) {});
        if (lane < 3) {
            o[lane] = __ldg(p + lane);
            o[3 * (NPTS - 1) + lane] = __ldg(p + 3 * (m - 1) + lane);
        }
        if (!(L > 0.0f)) {  // a single point or zero length: copies of the first point
            for (int k = 3 + lane; k < 3 * (NPTS - 1); k += 32) o[k] = __ldg(p + k % 3);
            continue;
        }
        // target k's arc length, k L / 20 as k times the rounded L / 20 (non-decreasing in k,
        // below L for k <= 19, and the same expression wherever it is compared)
        const float step = L / (float)(NPTS - 1), inv = 1.0f / step;
        auto target = [step](int k) { return (float)k * step; };
        segment_pass(p, m, lane, [&](float c0, float c1, float len, const float* a,
                                     const float* b) {
            // the targets in (c0, c1]: start from an estimate of the first one and settle it
            // with the exact comparisons, so the segment that holds a target writes it
            int k = (int)(c0 * inv);
            k = max(1, min(NPTS - 2, k));
            while (k > 1 && target(k - 1) > c0) --k;
            while (k <= NPTS - 2 && target(k) <= c0) ++k;
            for (; k <= NPTS - 2 && target(k) <= c1; ++k) {
                const float w =
                    len > 0.0f ? fminf(1.0f, fmaxf(0.0f, (target(k) - c0) / len)) : 0.0f;
#pragma unroll
                for (int r = 0; r < 3; ++r) o[3 * k + r] = fmaf(w, b[r] - a[r], a[r]);
            }
        });
    }
}

}  // namespace

seg_status resample_launch(const float* pts, const long long* off, long long n, float* out,
                           cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks =
        std::min<long long>((n + RS_WARPS - 1) / RS_WARPS, (long long)sms * 16);
    k_resample<<<(unsigned)blocks, RS_WARPS * 32, 0, st>>>(pts, off, n, out);
    const cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "seg_resample") : SEG_OK;
}

}  // namespace seg
