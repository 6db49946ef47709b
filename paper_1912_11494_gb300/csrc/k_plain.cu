// SEG_MODE_PLAIN: exact FP32 labelling (Algorithm 1 with the progressive discarding of
// Section 2.3, closest bundle of Section 2.4).
//
// Work split: every warp owns a tile of TW = 32 consecutive fibers for the whole atlas and runs
// independently of the other warps of its CTA (no CTA barrier anywhere), so no fiber result
// crosses warps and the latency of one warp's exact checks is hidden by the others. The warp's
// tile (32 x 252 B) is copied into its slice of shared memory by the TMA engine (1D bulk copy).
// The atlas is walked in chunks of 32*C centroids, sorted bundle-major; each lane keeps C
// centroids of the chunk in registers (the next chunk is prefetched while the current one is
// screened) and the fibers of the tile are broadcast from shared memory.
//
// test1 (Section 2.3: the centre point, shared by both orientations) is evaluated in dot-product
// form, |a-b|^2 <= theta^2  <=>  a.b + (theta^2 - |b|^2)/2 >= |a|^2/2, i.e. three FMAs and one
// compare per pair, with a rounding slack that only ever keeps more pairs (the slack covers the
// FP32 error of the dot form, so no pair the exact test would accept is dropped). The warp only
// looks at which pairs passed when its vote over a block of K fibers says one did; passing pairs
// are appended to the warp's queue and drained 32 at a time, one pair per lane, through the
// exact FP32 cascade (test1..test4 on squared distances, bound min(theta^2, best^2)). The result
// is merged into the fiber's packed key (d^2 bits, sorted centroid index, orientation) with a
// shared-memory atomicMin. The key order is (distance, bundle-major centroid index), i.e.
// Algorithm 1's strict-decrease update over its visiting order.
#include <math.h>

#include "seg_exact.cuh"
#include "seg_internal.cuh"
#include "seg_ptx.cuh"

namespace seg {
namespace {

constexpr int PW = 4;    // independent warps per CTA
constexpr int TW = 32;   // fibers per warp tile

constexpr int QCAP = 1024;  // per-warp queue of test1 survivors, drained after the screen

template <int PC, int PK>
struct WarpSmem {
    static constexpr int QW = QCAP;
    static constexpr size_t fc_off = 0;                        // [TW][63] floats
    static constexpr size_t fs_off = fc_off + TW * NC * 4;     // [TW][2] float4
    static constexpr size_t key_off = fs_off + TW * 32;        // [TW] u64
    static constexpr size_t ls_off = key_off + TW * 8;         // [TW] fiber lengths (TN)
    static constexpr size_t q_off = ls_off + TW * 4;           // [QW] u32
    static constexpr size_t bar_off = (q_off + QW * 4 + 15) / 16 * 16;
    static constexpr size_t bytes = bar_off + 16;
};

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// max over C values with 3-input max
template <int C>
__device__ __forceinline__ float maxn(const float* t) {
    if constexpr (C == 1) {
        return t[0];
    } else if constexpr (C == 2) {
        return fmaxf(t[0], t[1]);
    } else {
        float m = fmax3(t[0], t[1], t[2]);
#pragma unroll
        for (int c = 3; c + 1 < C; c += 2) m = fmax3(m, t[c], t[c + 1]);
        if constexpr (C % 2 == 0) m = fmaxf(m, t[C - 1]);
        return m;
    }
}

__device__ __forceinline__ float key_best2(unsigned long long k) {
    return __uint_as_float((unsigned)(k >> 32));  // NaN for the empty key: fminf ignores it
}

// Exact check of one queued pair e = (sorted centroid << 8 | tile fiber); merges into the
// fiber's key. The centroid row (256 B, aligned) is loaded in one batch of 16-byte loads so a
// check costs one memory round trip; the fiber comes from shared memory.
__device__ __forceinline__ void exact_and_merge(const AtlasView& at, const float* fc,
                                                const float* ls, unsigned long long* key,
                                                unsigned e, long long f0) {
    const int c = (int)(e >> 8);
    const int f = (int)(e & 255u);
    float b[CROW];
    const float4* b4 = reinterpret_cast<const float4*>(at.cen + (size_t)c * CROW);
#pragma unroll
    for (int q = 0; q < CROW / 4; ++q) {
        const float4 v = __ldg(b4 + q);
        b[4 * q] = v.x;
        b[4 * q + 1] = v.y;
        b[4 * q + 2] = v.z;
        b[4 * q + 3] = v.w;
    }
    const float t2 = __ldg(at.thr2 + c);
    const float bound = pair_bound2(at, t2, key_bound2(key_best2(key[f]), at.cls));
    float d2, kf;
    int o;
    // b[63] is the centroid's length (the TN term of Eq. 3)
    if (exact_pair(fc + f * NC, b, bound, d2, o, at.cls) &&
        key_value(at.cls, d2, t2, ls[f], b[CROW - 1], kf)) {
        multi_mark(at, f0 + f, at.bundle[c]);
        const unsigned long long k = ((unsigned long long)__float_as_uint(kf) << 32) |
                                     ((unsigned long long)c << 1) | (unsigned)o;
        atomicMin(key + f, k);
    }
}

// Label the TW fibers starting at f0 of one subject; the calling warp owns the tile and the
// slice ws of shared memory (its mbarrier initialised; `phase` = tiles this warp did before).
template <int PC, int PK>
__device__ __forceinline__ void plain_tile(const float* __restrict__ fib, long long n,
                                           long long f0, const AtlasView& at, int fib_aligned,
                                           int* __restrict__ labels, float* __restrict__ dist,
                                           int* __restrict__ cidx,
                                           unsigned char* __restrict__ orient,
                                           unsigned char* ws, uint32_t phase) {
    using WS = WarpSmem<PC, PK>;
    constexpr int CH = 32 * PC;
    const int lane = threadIdx.x & 31;
    float* fc = reinterpret_cast<float*>(ws + WS::fc_off);
    float4* fs = reinterpret_cast<float4*>(ws + WS::fs_off);
    unsigned long long* key = reinterpret_cast<unsigned long long*>(ws + WS::key_off);
    float* ls = reinterpret_cast<float*>(ws + WS::ls_off);
    unsigned* q = reinterpret_cast<unsigned*>(ws + WS::q_off);
    uint64_t* bar = reinterpret_cast<uint64_t*>(ws + WS::bar_off);
    const int nf = (int)min((long long)TW, n - f0);
    const bool tma_tile = fib_aligned && nf == TW;
    __syncwarp();
    if (tma_tile) {
        if (lane == 0) {
            fence_proxy_async_smem();  // earlier tiles' reads of this slice precede the copy
            mbar_arrive_expect_tx(bar, (uint32_t)(TW * NC * 4));
            bulk_g2s(fc, fib + f0 * NC, (uint32_t)(TW * NC * 4), bar);
        }
    } else {
        for (int k = lane; k < nf * NC; k += 32) fc[k] = __ldg(fib + f0 * NC + k);
    }
    key[lane] = ~0ull;
    // first centroid chunk goes to registers while the tile arrives
    float4 nxt[PC];
#pragma unroll
    for (int c = 0; c < PC; ++c) nxt[c] = __ldg(at.scr2 + c * 32 + lane);
    (void)WS::QW;
    int ok = 1;
    if (tma_tile && lane == 0) ok = (int)mbar_wait_bounded(bar, phase & 1u, at.wait_ns);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) {
        if (lane == 0) {
            atomicOr(at.status, ST_TIMEOUT);
            mbar_wait_bounded(bar, phase & 1u);
        }
        return;
    }
    // per-fiber screening data: centred centre point and |a|^2/2 minus its rounding slack,
    // each value twice so a packed FP32x2 FMA can use it against two centroids at once;
    // a fiber with a non-finite coordinate gets NaN (never passes) and is reported as such.
    {
        float x = 0.f, y = 0.f, z = 0.f, h = INFINITY;
        if (lane < nf) {
            const float* a = fc + lane * NC;
            bool finite = true;
            for (int k = 0; k < NC; ++k) finite = finite && isfinite(a[k]);
            x = a[3 * CENTRE] - at.c0x;
            y = a[3 * CENTRE + 1] - at.c0y;
            z = a[3 * CENTRE + 2] - at.c0z;
            const float r2 = fmaf(x, x, fmaf(y, y, z * z));
            h = finite ? 0.5f * r2 - 1e-5f * r2 - 1e-3f : NAN;
        }
        fs[2 * lane] = make_float4(x, x, y, y);
        fs[2 * lane + 1] = make_float4(z, z, h, h);
        ls[lane] = at.cls != 0 && lane < nf ? poly_length(fc + lane * NC) : 0.0f;
    }
    __syncwarp();

    const unsigned lt = (1u << lane) - 1u;
    const int nch = at.M_pad / CH;
    const int nfk = (nf + PK - 1) / PK * PK;
    // The screen runs until the atlas is done or the queue is full; then the queue is drained
    // outside the screen loop (so the two never hold registers at the same time) and the
    // screen resumes at the ballot where it stopped: chunk jres, fiber block fres, and within
    // that block the (fiber, centroid slot) index rres. Every drain empties the queue and the
    // next ballot adds at most 32 entries, so each round makes progress.
    int jres = 0, fres = 0, rres = 0;
    bool first = true;
    for (;;) {
        int qn = 0;
        bool full = false;
        int j = jres;
        if (!first) {
#pragma unroll
            for (int c = 0; c < PC; ++c) nxt[c] = __ldg(at.scr2 + (size_t)j * CH + c * 32 + lane);
        }
        first = false;
        int rskip = rres;
        for (; j < nch; ++j) {
            // centroids c and c+1 of the lane side by side for packed FP32x2 math
            float2 bx[PC / 2], by[PC / 2], bz[PC / 2], mg[PC / 2];
#pragma unroll
            for (int p = 0; p < PC / 2; ++p) {
                bx[p] = make_float2(nxt[2 * p].x, nxt[2 * p + 1].x);
                by[p] = make_float2(nxt[2 * p].y, nxt[2 * p + 1].y);
                bz[p] = make_float2(nxt[2 * p].z, nxt[2 * p + 1].z);
                mg[p] = make_float2(nxt[2 * p].w, nxt[2 * p + 1].w);
            }
            if (j + 1 < nch) {
#pragma unroll
                for (int c = 0; c < PC; ++c)
                    nxt[c] = __ldg(at.scr2 + (size_t)(j + 1) * CH + c * 32 + lane);
            }
            const unsigned cbase = (unsigned)(j * CH + lane);
            for (int f = (j == jres ? fres : 0); f < nfk; f += PK) {
                // score_k = max_c (a_k.b_c + mg_c) - h_k >= 0  <=>  a centroid passes test1
                float sk[PK];
#pragma unroll
                for (int k = 0; k < PK; ++k) {
                    const float4 a0 = fs[2 * (f + k)], a1 = fs[2 * (f + k) + 1];
                    float t[PC];
#pragma unroll
                    for (int p = 0; p < PC / 2; ++p) {
                        float2 u = __ffma2_rn(make_float2(a0.x, a0.y), bx[p], mg[p]);
                        u = __ffma2_rn(make_float2(a0.z, a0.w), by[p], u);
                        u = __ffma2_rn(make_float2(a1.x, a1.y), bz[p], u);
                        t[2 * p] = u.x;
                        t[2 * p + 1] = u.y;
                    }
                    sk[k] = maxn<PC>(t) - a1.z;
                }
                if (__any_sync(0xffffffffu, maxn<PK>(sk) >= 0.0f)) {
#pragma unroll
                    for (int k = 0; k < PK; ++k) {
                        if (!full && __any_sync(0xffffffffu, sk[k] >= 0.0f)) {
                            const float4 a0 = fs[2 * (f + k)], a1 = fs[2 * (f + k) + 1];
#pragma unroll
                            for (int c = 0; c < PC; ++c) {
                                if (full || k * PC + c < rskip) continue;
                                const float bxc = c & 1 ? bx[c / 2].y : bx[c / 2].x;
                                const float byc = c & 1 ? by[c / 2].y : by[c / 2].x;
                                const float bzc = c & 1 ? bz[c / 2].y : bz[c / 2].x;
                                const float mgc = c & 1 ? mg[c / 2].y : mg[c / 2].x;
                                const float t =
                                    fmaf(a1.x, bzc, fmaf(a0.z, byc, fmaf(a0.x, bxc, mgc)));
                                const bool p = t >= a1.z;
                                const unsigned m = __ballot_sync(0xffffffffu, p);
                                if (m) {
                                    if (qn + 32 > QCAP) {
                                        full = true;
                                        rres = k * PC + c;
                                    } else {
                                        if (p)
                                            q[qn + __popc(m & lt)] =
                                                ((cbase + (unsigned)(c * 32)) << 8) |
                                                (unsigned)(f + k);
                                        qn += __popc(m);
                                    }
                                }
                            }
                        }
                    }
                }
                rskip = 0;
                if (full) {
                    fres = f;
                    break;
                }
            }
            if (full) {
                jres = j;
                break;
            }
        }
        __syncwarp();
        for (int i = lane; i < qn; i += 32) exact_and_merge(at, fc, ls, key, q[i], f0);
        __syncwarp();
        if (!full) break;
    }

    if (lane < nf) {
        const long long gi = f0 + lane;
        const unsigned long long k = key[lane];
        if (isnan(fs[2 * lane + 1].z)) {
            labels[gi] = -1;
            if (dist) dist[gi] = NAN;
            if (cidx) cidx[gi] = -1;
            if (orient) orient[gi] = 0;
        } else if (k == ~0ull) {
            labels[gi] = -1;
            if (dist) dist[gi] = INFINITY;
            if (cidx) cidx[gi] = -1;
            if (orient) orient[gi] = 0;
        } else {
            const int c = (int)((k & 0xffffffffull) >> 1);
            labels[gi] = at.bundle[c];
            const float kf = __uint_as_float((unsigned)(k >> 32));
            if (dist) dist[gi] = at.cls != 0 ? kf : sqrtf(kf);  // D, or sqrt(d^2)
            if (cidx) cidx[gi] = at.perm[c];
            if (orient) orient[gi] = (unsigned char)(k & 1ull);
        }
    }
}

template <int PC, int PK>
__global__ void __launch_bounds__(PW * 32)
k_label_plain(const float* __restrict__ fib, long long n, AtlasView at, int fib_aligned,
              int* __restrict__ labels, float* __restrict__ dist, int* __restrict__ cidx,
              unsigned char* __restrict__ orient) {
    using WS = WarpSmem<PC, PK>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* ws = smem + warp * WS::bytes;
    const long long f0 = ((long long)blockIdx.x * PW + warp) * TW;
    if (f0 >= n) return;  // warp-uniform
    if (lane == 0) {
        mbar_init(reinterpret_cast<uint64_t*>(ws + WS::bar_off), 1);
        fence_mbar_init();
    }
    plain_tile<PC, PK>(fib, n, f0, at, fib_aligned, labels, dist, cidx, orient, ws, 0u);
}

// Many subjects in one persistent launch: every warp takes (subject, tile) work items from a
// global counter until the table's tiles are exhausted (no warp ever waits for another).
template <int PC, int PK>
__global__ void __launch_bounds__(PW * 32)
k_label_plain_batch(const BatchEntry* __restrict__ table, int nsubj,
                    unsigned long long* __restrict__ counter, AtlasView at) {
    using WS = WarpSmem<PC, PK>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* ws = smem + warp * WS::bytes;
    if (lane == 0) {
        mbar_init(reinterpret_cast<uint64_t*>(ws + WS::bar_off), 1);
        fence_mbar_init();
    }
    const long long total = table[nsubj].tile0;
    uint32_t done = 0;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((long long)t >= total) break;
        int lo = 0, hi = nsubj - 1;  // last subject whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (table[mid].tile0 <= (long long)t) lo = mid; else hi = mid - 1;
        }
        const BatchEntry e = table[lo];
        const long long f0 = ((long long)t - e.tile0) * TW;
        plain_tile<PC, PK>(e.fib, e.n, f0, at, ((uintptr_t)e.fib % 16) == 0, e.labels, e.dist,
                           nullptr, nullptr, ws, done);
        if (((uintptr_t)e.fib % 16) == 0 && min((long long)TW, e.n - f0) == TW) ++done;
    }
}

}  // namespace

namespace {

template <int PC, int PK>
cudaError_t launch_cfg(const AtlasView& at, const float* fib, long long n, int* labels,
                       float* dist, int* cidx, unsigned char* orient, cudaStream_t st) {
    static_assert(TW % PK == 0 && MPAD % (32 * PC) == 0, "tile shape");
    const size_t smem = PW * WarpSmem<PC, PK>::bytes;
    auto kern = k_label_plain<PC, PK>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const long long tiles = (n + TW - 1) / TW;
    const long long grid = (tiles + PW - 1) / PW;
    const int aligned = ((uintptr_t)fib % 16) == 0;
    kern<<<(unsigned)grid, PW * 32, smem, st>>>(fib, n, at, aligned, labels, dist, cidx, orient);
    return cudaGetLastError();
}

}  // namespace

template <int PC, int PK>
cudaError_t launch_batch_cfg(const BatchEntry* table, int nsubj, unsigned long long* counter,
                             const AtlasView& at, int sms, cudaStream_t st) {
    const size_t smem = PW * WarpSmem<PC, PK>::bytes;
    auto kern = k_label_plain_batch<PC, PK>;
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PW * 32, smem);
    if (e) return e;
    if (per_sm < 1) per_sm = 1;
    kern<<<(unsigned)(sms * per_sm), PW * 32, smem, st>>>(table, nsubj, counter, at);
    return cudaGetLastError();
}

// Tile shapes (centroids per lane, fibers per vote) the autotuner chooses from.
// Entry 0 is the default (fastest measured on the 4,145,000 x 10,000 workload).
const int kPlainConfigs[][2] = {{8, 4}, {4, 2}, {4, 4}, {8, 2}, {2, 8}, {4, 8}};
static_assert(true, "every C above is even: the screen pairs centroids for FP32x2 math");
const int kNumPlainConfigs = 6;

cudaError_t launch_label_plain(const AtlasView& at, const float* fib, long long n, int* labels,
                               float* dist, int* cidx, unsigned char* orient, cudaStream_t st,
                               int config) {
    if (n <= 0) return cudaSuccess;
    switch (config) {
        case 1: return launch_cfg<4, 2>(at, fib, n, labels, dist, cidx, orient, st);
        case 2: return launch_cfg<4, 4>(at, fib, n, labels, dist, cidx, orient, st);
        case 3: return launch_cfg<8, 2>(at, fib, n, labels, dist, cidx, orient, st);
        case 4: return launch_cfg<2, 8>(at, fib, n, labels, dist, cidx, orient, st);
        case 5: return launch_cfg<4, 8>(at, fib, n, labels, dist, cidx, orient, st);
        default: return launch_cfg<8, 4>(at, fib, n, labels, dist, cidx, orient, st);
    }
}

cudaError_t launch_label_plain_batch(const BatchEntry* table, int nsubj,
                                     unsigned long long* counter, const AtlasView& at, int sms,
                                     cudaStream_t st, int config) {
    switch (config) {
        case 1: return launch_batch_cfg<4, 2>(table, nsubj, counter, at, sms, st);
        case 2: return launch_batch_cfg<4, 4>(table, nsubj, counter, at, sms, st);
        case 3: return launch_batch_cfg<8, 2>(table, nsubj, counter, at, sms, st);
        case 4: return launch_batch_cfg<2, 8>(table, nsubj, counter, at, sms, st);
        case 5: return launch_batch_cfg<4, 8>(table, nsubj, counter, at, sms, st);
        default: return launch_batch_cfg<8, 4>(table, nsubj, counter, at, sms, st);
    }
}

}  // namespace seg
