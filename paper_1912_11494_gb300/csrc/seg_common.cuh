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
};

// One subject of a batched call (device table; entry nsubj holds only tile0 = total tiles).
struct BatchEntry {
    const float* fib;
    long long n;
    int* labels;
    float* dist;
    long long tile0;  // first work item (32-fiber tile) of this subject
    long long pad;
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
