// Internal declarations shared by the libseg CUDA sources (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "seg.h"

namespace seg {

constexpr int NPTS = SEG_NPTS;   // 21 points per fiber (Section 2.3 resampling)
constexpr int NC = NPTS * 3;     // 63 coordinates
constexpr int CROW = 64;         // padded centroid row (floats) in the sorted copy
constexpr int CROW4 = NPTS;      // point-major centroid row: one float4 (x, y, z, 0) per point
constexpr int CENTRE = 10;       // test1 point; maps to itself under reversal (20 - 10)

// Device status word bits (sticky until seg_sync_status reads them).
constexpr unsigned ST_TIMEOUT = 1u;
constexpr unsigned ST_OVERFLOW = 2u;

constexpr int MPAD = 2048;    // the sorted atlas is padded to a multiple of this many centroids

// Locality order of the GEMM modes: the centre point's cell (LOC_CELL_MM cells, 2^LOC_BITS per
// axis around the atlas centre, clamped) taken along a three-dimensional Hilbert curve, whose
// consecutive cells always share a face, so that a run of consecutive positions covers a compact
// region. The fibers are counting-sorted on it on the device and the centroid columns ordered
// by it on the host.
constexpr int LOC_BITS = 7;          // 128 cells per axis
constexpr float LOC_CELL_MM = 2.0f;  // a 256 mm cube

// Position of cell (x, y, z), each in [0, 2^LOC_BITS), along the Hilbert curve, in
// [0, 2^(3 LOC_BITS)). Skilling's transform (J. Skilling, "Programming the Hilbert curve", AIP
// Conf. Proc. 707, 2004): undo the excess rotations and reflections level by level, Gray-code
// across the axes, then interleave the bits (bit b of axis i goes to bit 3b + 2 - i).
__host__ __device__ inline uint32_t hilbert_index3(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t X[3] = {x, y, z};
    for (uint32_t Q = 1u << (LOC_BITS - 1); Q > 1u; Q >>= 1) {
        const uint32_t P = Q - 1u;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;                               // reflect the lower bits of axis 0
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;    // swap the lower bits of 0 and i
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = 1u << (LOC_BITS - 1); Q > 1u; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1u;
    uint32_t h = 0;
    for (int b = 0; b < LOC_BITS; ++b)
        for (int i = 0; i < 3; ++i) h |= (((X[i] ^ t) >> b) & 1u) << (3 * b + 2 - i);
    return h;
}

// Read-only device view of an atlas, sorted bundle-major (the visiting order of Algorithm 1).
struct AtlasView {
    int M;                      // centroids
    int B;                      // bundles
    int M_pad;                  // M rounded up to MPAD
    float c0x, c0y, c0z;        // centring offset (mean centroid centre point)
    const float* cen;           // [M][64]: 63 coordinates, [63] = 0
    const float4* scr;          // [M]: centre point xyz and theta^2 of the centroid's bundle
    // [M_pad]: centred centre point b' and (theta^2 - |b'|^2)/2 + slack, the test1 screen in
    // dot-product form; padding rows never pass (w = -inf)
    const float4* scr2;
    const float* thr2;          // [M]: theta^2 (float32 product theta*theta)
    const int* bundle;          // [M]: bundle index (caller numbering)
    const int* perm;            // [M]: caller's centroid index of sorted position
    unsigned* status;           // device status word
    int cls;                    // classification: 0 Eq. 2, 1 Eq. 2 + TN, 2 the paper's
                                // direction inference + TN (seg_classification); cen[63] of
                                // each row holds the centroid's length for the TN term
    unsigned long long wait_ns; // limit of the kernels' first bounded waits (default 2 s; the
                                // drain waits after an abort always keep 2 s)
    unsigned* multi;            // seg_label_multi: [n][multi_words] bundle bits of every
                                // passing pair (caller's fiber order), or NULL
    long long multi_words;
};

#ifdef __CUDACC__
// Bound on a pair's squared point distances: theta^2 alone when every passing bundle is
// wanted (seg_label_multi), else also the best key so far (kb2, see key_bound2).
__device__ __forceinline__ float pair_bound2(const AtlasView& at, float t2, float kb2) {
    return at.multi ? t2 : fminf(t2, kb2);
}

// Records a passing pair's bundle for fiber f (caller order) in the multi-label output.
__device__ __forceinline__ void multi_mark(const AtlasView& at, long long f, int bundle) {
    if (at.multi)
        atomicOr(at.multi + f * at.multi_words + (bundle >> 5), 1u << (bundle & 31));
}
#endif

// One subject of a batched call (device table; entry nsubj holds only tile0 = total tiles).
struct BatchEntry {
    const float* fib;
    long long n;
    int* labels;
    float* dist;
    long long tile0;  // first work item (32-fiber tile) of this subject (plain mode)
    long long first;  // its first fiber in the concatenation of all subjects (GEMM modes)
};

// Where the GEMM modes read fibers and write results: one subject (fib, outputs given to the
// kernel), or several subjects concatenated into one virtual array of fibers, index i being
// fiber i - table[k].first of subject k = the last entry with table[k].first <= i (entry
// nsubj holds first = the total, so empty subjects are never chosen for a valid i).
struct FiberSrc {
    const float* fib;
    const BatchEntry* table;
    int nsubj;
    __device__ __forceinline__ int subject(long long i) const {
        int lo = 0, hi = nsubj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (table[mid].first <= i) lo = mid; else hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ const float* row(long long i) const {
        if (!table) return fib + (size_t)i * (3 * SEG_NPTS);
        const int k = subject(i);
        return table[k].fib + (size_t)(i - table[k].first) * (3 * SEG_NPTS);
    }
};

// Plain exact labelling of n fibers (SEG_MODE_PLAIN).
cudaError_t launch_label_plain(const AtlasView& at, const float* fib, long long n, int* labels,
                               float* dist, int* cidx, unsigned char* orient, cudaStream_t st,
                               int config = 0);
cudaError_t launch_label_plain_batch(const BatchEntry* table, int nsubj,
                                     unsigned long long* counter, const AtlasView& at, int sms,
                                     cudaStream_t st, int config);
constexpr int PLAIN_TILE = 32;  // fibers per work item of the plain kernels
extern const int kPlainConfigs[][2];
extern const int kNumPlainConfigs;

}  // namespace seg
