// SEG_MODE_GEMM_BF16 / SEG_MODE_GEMM_TF32: tensor-core lower-bound prune, then the exact FP32
// test on the survivors only. Not in the paper; labels and distances equal SEG_MODE_PLAIN's.
//
// Bound. For a fiber a and a centroid b taken in orientation o (points in order, or reversed as
// in Eq. 2), with p, q their 63 coordinates (centred by the same offset),
//     d_o^2 = max_i |a_i - b_o(i)|^2 >= (1/21) sum_i |a_i - b_o(i)|^2 = S / 21,
//     S = |p|^2 + |q|^2 - 2 p.q,
// so S > 21 theta^2 proves the orientation fails its threshold. p.q for all fibers x all 2M
// (centroid, orientation) columns is one GEMM [n x 64] x [64 x 2M] on the tensor cores, with the
// operands rounded to BF16 (or TF32) and FP32 accumulation in tensor memory. The rounding error
// |p.q - p~.q~| <= kappa |p||q| <= kappa (|p|^2 + |q|^2) / 2 (kappa = 2u + u^2 + accumulation)
// is separable, so the test folds into one compare per element:
//     keep (fiber i, column j)  <=>  p~_i.q~_j + pad_j >= alpha_i,
//     alpha_i = (1 - kappa)/2 |p_i|^2 - slack_i,
//     pad_j   >= -[(|q_j|^2 - 21 theta_j^2 (1 + rho)) / 2 - kappa/2 |q_j|^2 - slack_j],
// where pad_j is the 64th K column of the centroid operand (the fiber operand holds 1 there) and
// is rounded upward, and the slacks cover FP32 norms, the centring and the exact test's own
// rounding (rho). Every pair the exact FP32 test would accept therefore survives the prune.
//
// Kernels. A counting sort orders the fibers by the 2 mm cell of their centre point, so that
// the 32 fibers of a warp have nearly the same survivors. The fiber operand is written in that
// order. The screen is a persistent CTA per SM, warp-specialised: warp 0 issues TMA loads (R
// fiber tiles of 128 rows per work unit, double-buffered, and a ring of S centroid tiles of N
// columns), warp 1 issues tcgen05.mma (M=128, N, K) into one of 512/(R*N) TMEM accumulators of R*N
// columns, and eight epilogue warps read a finished accumulator with tcgen05.ld.red, which
// returns each row's max over 32 columns: only when that max reaches alpha in some row does the
// warp compare the individual values and write a block record (32 fibers x 32 columns, one
// column mask per fiber). A second kernel runs the exact test of Section 2.3 on every survivor
// of every block and merges the result into the fiber's packed key with atomicMin (same key as
// the plain kernel, so the tie rule of Algorithm 1 holds); the fibers whose survivors did not
// fit the record list are rescanned exactly, and a last kernel writes labels and distances in
// the caller's order.
//
// Orientation-free variant (SEG_MODE_GEMM_INV_*). With c = a_10 and s_i = (a_i + a_(20-i))/2,
// for x_i = a_i - b_i, y_i = a_(20-i) - b_(20-i) (or the reversed pairing) the identity
// |x|^2 + |y|^2 = |x + y|^2 / 2 + |x - y|^2 / 2 >= |x + y|^2 / 2 gives, in either orientation,
//     S >= |c_a - c_b|^2 + 2 sum_(i<10) |s_i(a) - s_i(b)|^2 = I(a, b),
// and x + y is the same vector for both orientations, so I is one column per centroid over 33
// features (c and sqrt(2) s_i) and the same separable margin applies. The same inequality,
// |u|^2 + |v|^2 >= |u + v|^2 / 2 with u = dc and v = sqrt(2) ds_9, merges the centre point and
// the innermost midpoint into g = c / sqrt(2) + s_9, which leaves 30 features and the pad column
// within K = 32: half the tensor-core work of the 64-wide directional operands. Survivors are
// checked in both orientations.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>

#include "seg_exact.cuh"
#include "seg_internal.cuh"
#include "seg_tc.cuh"

namespace seg {
namespace {

constexpr int EPI_WARPS = 8;       // two epilogue warps per TMEM lane quarter
constexpr int EPI_SUB = EPI_WARPS / 4;
constexpr int GEMM_THREADS = 64 + 32 * EPI_WARPS;  // warp 0 TMA, warp 1 MMA, then epilogue
constexpr int COL_ALIGN = 256;     // columns padded to a multiple of this
constexpr int SLOT_GRAB = 64;      // block records an epilogue warp reserves at a time
constexpr unsigned EMPTY_SLOT = 0xFFFFFFFFu;  // header of a reserved record left unused
constexpr unsigned long long NAN_KEY = ~0ull - 1ull;
constexpr float PAD_NEG = -1e30f;  // pad of padding columns: never survives

// Rounding constants: unit roundoff of the operand format and the FP32 accumulation bound for
// 64 terms (taken as 64 ulps, conservative for any summation order of the tensor core).
constexpr double U_BF16 = 1.0 / 512.0;    // 2^-9, round to nearest
constexpr double U_TF32 = 1.0 / 2048.0;   // 2^-11, round to nearest
constexpr double GAMMA_ACC = 64.0 / 8388608.0;
constexpr double RHO = 1e-5;              // relative slack for the exact test's FP32 rounding

__host__ __device__ inline double kappa_of(int fmt) {
    const double u = fmt == 1 ? U_BF16 : U_TF32;
    return 1.05 * (2.0 * u + u * u) + 2.0 * GAMMA_ACC;
}

// Survivors are kept as block records: one per (32 sorted fibers) x (32-column chunk) block of
// the product with at least one surviving element, holding the first fiber and column and one
// 32-bit column mask per fiber. With fibers in locality order a block holds about two hundred
// survivors on atlases shaped like the paper's, so the exact kernel stages its fiber and
// centroid rows once for all of them.
struct GemmScratch {
    void* a;                      // fiber operand [n_pad][64], rows in sorted order
    const unsigned* perm;         // [n] sorted position -> the caller's fiber index
    float* fs;                    // [n_pad][64] the fibers in sorted order (63 floats + 0)
    float* alpha;                 // [n_pad] (sorted order, as key and flag)
    unsigned long long* key;      // [n]
    unsigned char* flag;          // [n] survivors dropped for lack of list space
    const unsigned long long* amask;  // [n_units][awords] bit c: the unit's 32-column chunk c
                                      // may hold survivors (a tile is computed when any of its
                                      // chunks may; the epilogue reads only those chunks)
    int awords;
    const float4* cen_sp;         // the atlas's spatial-order arrays (GemmAtlas)
    const float4* end_sp;
    const float* thr2_sp;
    const int* sp_s;
    uint2* hdr;                   // [cap] {first sorted fiber, first column} or EMPTY_SLOT
    unsigned* mask;               // [cap][32] surviving columns of each of the 32 fibers
    unsigned long long wait_ns;   // limit of the screen's bounded waits (AtlasView::wait_ns)
    unsigned long long* cnt;      // [0] records reserved, [1] fibers flagged, [2] survivors,
                                  // [3] pairs in the blocks the tensor cores computed, [4] work
                                  // counter (the exact kernel's runs, the fused kernel's groups),
                                  // [5] point distances of the exact test
    long long cap;
};

// ---- operand preparation ---------------------------------------------------------------------

__device__ inline float tf32_rn(float x) {
    uint32_t u = __float_as_uint(x);
    u = (u + 0x1000u) & 0xFFFFE000u;  // round to nearest (ties away) at 10 mantissa bits
    return __uint_as_float(u);
}

__device__ inline float tf32_up(float x) {  // round toward +inf at 10 mantissa bits
    uint32_t u = __float_as_uint(x);
    if ((u & 0x1FFFu) == 0u) return x;
    if (x > 0.0f) u = (u + 0x2000u) & 0xFFFFE000u;
    else u &= 0xFFFFE000u;
    return __uint_as_float(u);
}

// Orientation-free features of 63 centred coordinates (30 values): g = c / sqrt(2) + s_9, then
// sqrt(2) s_i for i = 0..8, with c = point 10 and s_i the midpoint of points i and 20 - i.
__device__ inline void inv_features(const float* x, float* f) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        f[r] = x[3 * CENTRE + r] * 0.70710678118654752f + (x[27 + r] + x[33 + r]) * 0.5f;
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int r = 0; r < 3; ++r)
            f[3 + 3 * i + r] = (x[3 * i + r] + x[3 * (NPTS - 1 - i) + r]) * 0.70710678118654752f;
}

constexpr int NF_INV = 30;  // orientation-free features
constexpr int KE_INV = 32;  // their K width: 30 features, a zero, the pad column
constexpr int KE_DIR = 64;  // K width of the directional columns: 63 coordinates, the pad

// Orientation-free centroid columns: the centroid at spatial position j in column j, rows of
// KE_INV values.
__global__ void k_prep_b_inv(AtlasView at, const int* sp_s, int fmt, int cols, int cols_pad,
                             void* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols_pad) return;
    float q[NF_INV];
    float pad = PAD_NEG;
    if (j < cols) {
        const int sj = sp_s[j];
        const float* b = at.cen + (size_t)sj * CROW;
        float x[NC];
        for (int i = 0; i < NPTS; ++i) {
            x[3 * i] = b[3 * i] - at.c0x;
            x[3 * i + 1] = b[3 * i + 1] - at.c0y;
            x[3 * i + 2] = b[3 * i + 2] - at.c0z;
        }
        inv_features(x, q);
        double n2 = 0.0;
        for (int k = 0; k < NF_INV; ++k) n2 += (double)q[k] * q[k];
        const double t2 = (double)at.thr2[sj];
        const double kap = kappa_of(fmt);
        const double G = 0.5 * (n2 - 21.0 * t2 * (1.0 + RHO)) - 0.5 * kap * n2 -
                         (1e-5 * (n2 + 21.0 * t2) + 0.005);
        pad = (float)(-G);
        if ((double)pad < -G) pad = nextafterf(pad, INFINITY);
    } else {
        for (int k = 0; k < NF_INV; ++k) q[k] = 0.0f;
    }
    if (fmt == 1) {
        __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out) + (size_t)j * KE_INV;
        for (int k = 0; k < KE_INV - 1; ++k) o[k] = __float2bfloat16_rn(k < NF_INV ? q[k] : 0.0f);
        o[KE_INV - 1] = j < cols ? __float2bfloat16_ru(pad) : __float2bfloat16_rn(PAD_NEG);
    } else {
        float* o = reinterpret_cast<float*>(out) + (size_t)j * KE_INV;
        for (int k = 0; k < KE_INV - 1; ++k) o[k] = tf32_rn(k < NF_INV ? q[k] : 0.0f);
        o[KE_INV - 1] = j < cols ? tf32_up(pad) : tf32_rn(PAD_NEG);
    }
}

// Directional centroid columns: the centroid at spatial position c gives column 2c (points in
// order) and 2c+1 (reversed).
__global__ void k_prep_b(AtlasView at, const int* sp_s, int fmt, int cols, int cols_pad,
                         void* out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols_pad) return;
    float q[NC];
    float pad = PAD_NEG;
    if (j < cols) {
        const int s = sp_s[j >> 1], o = j & 1;
        const float* b = at.cen + (size_t)s * CROW;
        double n2 = 0.0;
        for (int i = 0; i < NPTS; ++i) {
            const int pi = o ? NPTS - 1 - i : i;
            q[3 * i] = b[3 * pi] - at.c0x;
            q[3 * i + 1] = b[3 * pi + 1] - at.c0y;
            q[3 * i + 2] = b[3 * pi + 2] - at.c0z;
            n2 += (double)q[3 * i] * q[3 * i] + (double)q[3 * i + 1] * q[3 * i + 1] +
                  (double)q[3 * i + 2] * q[3 * i + 2];
        }
        const double t2 = (double)at.thr2[s];
        const double kap = kappa_of(fmt);
        const double G = 0.5 * (n2 - 21.0 * t2 * (1.0 + RHO)) - 0.5 * kap * n2 -
                         (1e-5 * (n2 + 21.0 * t2) + 0.005);
        pad = (float)(-G);
        // round the float upward so the pad never undershoots -G
        if ((double)pad < -G) pad = nextafterf(pad, INFINITY);
    } else {
        for (int k = 0; k < NC; ++k) q[k] = 0.0f;
    }
    if (fmt == 1) {
        __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(out) + (size_t)j * 64;
        for (int k = 0; k < NC; ++k) o[k] = __float2bfloat16_rn(q[k]);
        o[63] = j < cols ? __float2bfloat16_ru(pad) : __float2bfloat16_rn(PAD_NEG);
    } else {
        float* o = reinterpret_cast<float*>(out) + (size_t)j * 64;
        for (int k = 0; k < NC; ++k) o[k] = tf32_rn(q[k]);
        o[63] = j < cols ? tf32_up(pad) : tf32_rn(PAD_NEG);
    }
}

// ---- locality order --------------------------------------------------------------------------
// Subjects arrive in arbitrary order, so the 32 fibers a warp of the screen reads would have
// unrelated survivor columns. A counting sort on the cell of the centre point (2 mm cells, a 128^3
// grid around the atlas centre, cells along a Hilbert curve: hilbert_index3) groups fibers that
// lie close together; every later kernel addresses fibers by their sorted position and reads the
// caller's row through perm[]. Results do not depend on the order (each fiber's key is its own
// minimum).
constexpr int NBINS = 1 << (3 * LOC_BITS);         // 2,097,152 cells
constexpr int SCAN_BLOCK = 1024;                   // bins scanned per block
constexpr int NTOP = NBINS / SCAN_BLOCK;           // 2,048 block totals

__device__ inline unsigned cell_of(float v, float c0) {
    const float t = floorf((v - c0) * (1.0f / LOC_CELL_MM)) + (float)(1 << (LOC_BITS - 1));
    return t >= 0.0f ? (unsigned)fminf(t, (float)((1 << LOC_BITS) - 1)) : 0u;  // NaN -> 0
}

__global__ void k_bin_count(FiberSrc src, long long n, AtlasView at,
                            unsigned* __restrict__ bin, unsigned* __restrict__ hist) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* c = src.row(i) + 3 * CENTRE;
    const unsigned b = hilbert_index3(cell_of(__ldg(c), at.c0x), cell_of(__ldg(c + 1), at.c0y),
                                      cell_of(__ldg(c + 2), at.c0z));
    bin[i] = b;
    atomicAdd(hist + b, 1u);
}

// Exclusive scan of each block of SCAN_BLOCK bins in place; block totals to top[].
__global__ void __launch_bounds__(SCAN_BLOCK) k_bin_scan(unsigned* __restrict__ hist,
                                                         unsigned* __restrict__ top) {
    __shared__ unsigned s_w[SCAN_BLOCK / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const unsigned v = hist[blockIdx.x * SCAN_BLOCK + t];
    unsigned x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned s = s_w[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        s_w[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    hist[blockIdx.x * SCAN_BLOCK + t] = x - v + (w ? s_w[w - 1] : 0u);
    if (t == SCAN_BLOCK - 1) top[blockIdx.x] = x + (w ? s_w[w - 1] : 0u);
}

// Exclusive scan of the NTOP block totals (one warp, NTOP / 32 values per lane).
__global__ void k_bin_scan_top(unsigned* __restrict__ top) {
    constexpr int PER = NTOP / 32;
    const int lane = threadIdx.x;
    unsigned v[PER], s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = top[lane * PER + k];
        s += v[k];
    }
    unsigned x = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    unsigned run = x - s;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        top[lane * PER + k] = run;
        run += v[k];
    }
}

__global__ void k_bin_scatter(const unsigned* __restrict__ bin, long long n,
                              unsigned* __restrict__ hist, const unsigned* __restrict__ top,
                              unsigned* __restrict__ perm) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned b = bin[i];
    perm[__ldg(top + b / SCAN_BLOCK) + atomicAdd(hist + b, 1u)] = (unsigned)i;
}

// Fiber rows in sorted order: centred coordinates (or the orientation-free features), 1 in
// the pad column, alpha_i; keys initialised. One warp per 32 rows: the rows perm[r0 .. r0+31]
// are copied (cp.async, all in flight together) into shared memory, each lane converts one row,
// and the 32 output rows go back out with coalesced stores.
//
// |p|^2 is summed in FP32 (fmaf, fixed order): the computed value is within 63 u_32 |p|^2 of the
// exact one, so n2 (1 - 4e-6) rounded down is a lower bound, and alpha is evaluated with
// downward rounding from it: alpha never exceeds (1 - kappa)/2 |p|^2 - 1e-5 |p|^2 - 0.005.
constexpr int PREP_WARPS = 4;
constexpr int PREP_STRIDE = 65;

template <int FMT, bool INV>
__global__ void __launch_bounds__(PREP_WARPS * 32, 4)
k_prep_a(FiberSrc fsrc, const unsigned* __restrict__ perm, long long n,
         long long n_pad, AtlasView at, void* __restrict__ out,
         float* __restrict__ alpha, unsigned long long* __restrict__ key,
         float* __restrict__ fs, float4* __restrict__ ubox) {
    __shared__ uint32_t s_buf[PREP_WARPS][32 * PREP_STRIDE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long r0 = ((long long)blockIdx.x * PREP_WARPS + w) * 32;
    if (r0 >= n_pad) return;
    const int rows_in = (int)max(0LL, min(32LL, n - r0));
    float* si = reinterpret_cast<float*>(s_buf[w]);
    const unsigned src_row = lane < rows_in ? __ldg(perm + r0 + lane) : 0u;
    // each lane finds its own row (for several subjects, a search of the work table), then
    // the warp copies the rows one after another
    const float* my_row = fsrc.row(src_row);
#pragma unroll 4
    for (int r = 0; r < rows_in; ++r) {  // all 63 x 32 copies in flight at once
        const float* src = shfl_ptr(my_row, r);
        cp_async4(si + r * PREP_STRIDE + lane, src + lane);
        if (lane < NC - 32) cp_async4(si + r * PREP_STRIDE + 32 + lane, src + 32 + lane);
    }
    cp_async_wait_all();
    __syncwarp();
    // each row's length (Eq. 3's l_S, for the TN term) in its free 64th slot
    si[lane * PREP_STRIDE + NC] = at.cls != 0 && lane < rows_in
                                      ? poly_length(si + lane * PREP_STRIDE) : 0.0f;
    __syncwarp();
    // the sorted copy of the rows (read by the exact re-check)
    float* fdst = fs + r0 * CROW;
#pragma unroll 4
    for (int k = lane; k < 32 * CROW; k += 32) {
        const int r = k / CROW, c = k % CROW;
        fdst[k] = r < rows_in ? si[r * PREP_STRIDE + c] : 0.0f;
    }
    const long long i = r0 + lane;
    float p[NC];
    bool finite = lane < rows_in;
    if (finite) {
#pragma unroll
        for (int t = 0; t < NPTS; ++t) {
            p[3 * t] = si[lane * PREP_STRIDE + 3 * t] - at.c0x;
            p[3 * t + 1] = si[lane * PREP_STRIDE + 3 * t + 1] - at.c0y;
            p[3 * t + 2] = si[lane * PREP_STRIDE + 3 * t + 2] - at.c0z;
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) finite = finite && isfinite(p[k]);
    }
    if (i < n) key[i] = finite ? ~0ull : NAN_KEY;  // a non-finite fiber gets the NaN key
    {   // centre-point box of the warp's finite fibers (empty: lo = +inf, hi = -inf)
        float lo[3], hi[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float c = finite ? si[lane * PREP_STRIDE + 3 * CENTRE + r] : 0.0f;
            lo[r] = finite ? c : INFINITY;
            hi[r] = finite ? c : -INFINITY;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                lo[r] = fminf(lo[r], __shfl_xor_sync(0xffffffffu, lo[r], off));
                hi[r] = fmaxf(hi[r], __shfl_xor_sync(0xffffffffu, hi[r], off));
            }
        }
        if (lane == 0) {
            ubox[2 * (r0 / 32)] = make_float4(lo[0], lo[1], lo[2], 0.0f);
            ubox[2 * (r0 / 32) + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
        }
    }
    float n2 = 0.0f;
    if (!finite) {
#pragma unroll
        for (int k = 0; k < NC; ++k) p[k] = 0.0f;
    } else if (INV) {
        float fe[NF_INV];
        inv_features(p, fe);
#pragma unroll
        for (int k = 0; k < NC; ++k) p[k] = k < NF_INV ? fe[k] : 0.0f;
#pragma unroll
        for (int k = 0; k < NF_INV; ++k) n2 = fmaf(p[k], p[k], n2);
    } else {
#pragma unroll
        for (int k = 0; k < NC; ++k) n2 = fmaf(p[k], p[k], n2);
    }
    const float c1 = __double2float_rd(0.5 * (1.0 - kappa_of(FMT)) - 1e-5);
    const float n2lo = __fmul_rd(n2, 0.999996f);
    alpha[i] = finite ? __fmaf_rd(n2lo, c1, -0.005f) : INFINITY;
    if (FMT == 0) return;  // SEG_MODE_PLAIN_CULLED: no tensor-core operand
    __syncwarp();  // every lane has its input row in registers: reuse the buffer for output
    uint32_t* so = s_buf[w];
    constexpr int KE = INV ? KE_INV : KE_DIR;     // row: KE - 1 values, then the pad column 1
    constexpr int words = FMT == 1 ? KE / 2 : KE;  // 32-bit words per output row
    constexpr int stride = words + 1;
    if (FMT == 1) {
#pragma unroll
        for (int k = 0; k < words - 1; ++k) {
            __nv_bfloat162 b = __floats2bfloat162_rn(p[2 * k], p[2 * k + 1]);
            so[lane * stride + k] = *reinterpret_cast<uint32_t*>(&b);
        }
        __nv_bfloat162 b = __floats2bfloat162_rn(p[KE - 2], 1.0f);
        so[lane * stride + words - 1] = *reinterpret_cast<uint32_t*>(&b);
    } else {
#pragma unroll
        for (int k = 0; k < words - 1; ++k) so[lane * stride + k] = __float_as_uint(tf32_rn(p[k]));
        so[lane * stride + words - 1] = __float_as_uint(1.0f);
    }
    __syncwarp();
    uint32_t* dst = reinterpret_cast<uint32_t*>(out) + r0 * words;
    for (int k = lane; k < 32 * words; k += 32) dst[k] = so[(k / words) * stride + (k % words)];
}

// ---- the tensor-core screen ------------------------------------------------------------------

// ---- block culling ---------------------------------------------------------------------------
// d_ME(a, b) >= |a_10 - b_10| in both orientations (the centre point pairs with itself, Eq. 2),
// so a (work unit x column tile) block whose centre-point boxes are farther apart than the
// largest threshold of the tile holds no pair that can pass: the screen skips it. The slack
// covers the FP32 rounding of the box distance and of the exact test.
struct UnitBox {
    float lx, ly, lz, hx, hy, hz;
};

__device__ inline UnitBox unit_box(const float4* __restrict__ ubox, long long u, int R) {
    UnitBox b{INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < 4 * R; ++k) {
        const float4 lo = __ldg(ubox + 2 * (u * 4 * R + k));
        const float4 hi = __ldg(ubox + 2 * (u * 4 * R + k) + 1);
        b.lx = fminf(b.lx, lo.x), b.ly = fminf(b.ly, lo.y), b.lz = fminf(b.lz, lo.z);
        b.hx = fmaxf(b.hx, hi.x), b.hy = fmaxf(b.hy, hi.y), b.hz = fmaxf(b.hz, hi.z);
    }
    return b;
}

// Squared gap between a unit's centre-point box and tile t's (0 where they meet).
__device__ inline float block_gap2(const UnitBox& b, const float4* __restrict__ tbox, int t) {
    const float4 lo = __ldg(tbox + 2 * t), hi = __ldg(tbox + 2 * t + 1);
    const float gx = fmaxf(0.0f, fmaxf(lo.x - b.hx, b.lx - hi.x));
    const float gy = fmaxf(0.0f, fmaxf(lo.y - b.hy, b.ly - hi.y));
    const float gz = fmaxf(0.0f, fmaxf(lo.z - b.hz, b.lz - hi.z));
    return gx * gx + gy * gy + gz * gz;
}

__device__ inline bool block_active(const UnitBox& b, const float4* __restrict__ tbox, int t) {
    const float lb2 = block_gap2(b, tbox, t);
    return !(lb2 > __ldg(&tbox[2 * t].w) * 1.0001f + 1e-3f);  // lo.w: max theta^2 of the tile
}

constexpr int MAXW = 64;  // mask words per unit: at most 4096 chunks (131,072 columns)

// The next tile with an active chunk in `bits` (word wd of a unit's chunk mask, CPT chunks per
// tile); clears that tile's bits.
template <int CPT>
__device__ __forceinline__ int next_tile(unsigned long long& bits, int wd) {
    const int gi = (__ffsll((long long)bits) - 1) / CPT;
    bits &= ~(((1ull << CPT) - 1) << (gi * CPT));
    return wd * (64 / CPT) + gi;
}

// The chunk masks of the units one thread of the screen visits (u, u + grid, ...), copied into
// a private ring of three shared-memory slots two units ahead with cp.async (one commit group
// per unit), so that the thread never stalls on the load of a unit's mask.
struct MaskRing {
    unsigned long long (*s)[MAXW];  // [3][MAXW]; words past awords stay zero
    int slot = 0;                   // slot of the current unit
    __device__ void init(unsigned long long (*ring)[MAXW], const GemmScratch& g, long long u0,
                         long long n_units) {
        s = ring;
        for (int i = 0; i < 3; ++i)
            for (int k = g.awords; k < MAXW; ++k) s[i][k] = 0ull;
        issue(g, u0, n_units, 0);
        issue(g, u0 + gridDim.x, n_units, 1);
    }
    __device__ void issue(const GemmScratch& g, long long u, long long n_units, int i) {
        if (u < n_units)
            for (int k = 0; k < g.awords; ++k) cp_async8(&s[i][k], g.amask + u * g.awords + k);
        cp_async_commit();
    }
    // the current unit u's words (its copies have landed); the copies for u + 2 grid start
    __device__ const unsigned long long* enter(const GemmScratch& g, long long u,
                                               long long n_units) {
        issue(g, u + 2 * (long long)gridDim.x, n_units, slot == 0 ? 2 : slot - 1);
        cp_async_wait_group<2>();
        return s[slot];
    }
    __device__ void leave() { slot = slot == 2 ? 0 : slot + 1; }
};
__device__ inline bool any_word(const unsigned long long* w, int words) {
    unsigned long long a = 0;
    for (int k = 0; k < words; ++k) a |= w[k];
    return a != 0;
}

// Active-chunk masks: one thread per work unit of R x 128 sorted fibers, one bit per 32-column
// chunk.
__global__ void k_block_mask(const float4* __restrict__ ubox, const float4* __restrict__ tbox,
                             long long n_units, int R, int n_chunks, int words,
                             unsigned long long* __restrict__ amask) {
    // one warp per unit; lane l tests chunks 32k + l
    const long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= n_units) return;
    const UnitBox b = unit_box(ubox, u, R);
    for (int wd = 0; wd < words; ++wd) {
        const int c0 = wd * 64 + lane, c1 = c0 + 32;
        const unsigned lo = __ballot_sync(0xffffffffu, c0 < n_chunks && block_active(b, tbox, c0));
        const unsigned hi = __ballot_sync(0xffffffffu, c1 < n_chunks && block_active(b, tbox, c1));
        if (lane == 0) amask[u * words + wd] = ((unsigned long long)hi << 32) | lo;
    }
}

// Centre-point box and max theta^2 of each 32-column chunk (`per` consecutive spatial
// centroids; an empty chunk never passes).
__global__ void k_tile_box(const float4* __restrict__ ctr_sp, int M, int per, int n_tiles,
                           float4* __restrict__ tbox) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, -INFINITY);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, INFINITY);
    for (int c = t * per; c < min(M, (t + 1) * per); ++c) {
        const float4 v = ctr_sp[c];
        lo.x = fminf(lo.x, v.x), lo.y = fminf(lo.y, v.y), lo.z = fminf(lo.z, v.z);
        hi.x = fmaxf(hi.x, v.x), hi.y = fmaxf(hi.y, v.y), hi.z = fmaxf(hi.z, v.z);
        lo.w = fmaxf(lo.w, v.w);  // the tile's largest theta^2
        hi.w = fminf(hi.w, v.w);  // and its smallest
    }
    tbox[2 * t] = lo;
    tbox[2 * t + 1] = hi;
}

// Boxes of windows of 32 consecutive chunk boxes (lo.w the largest theta^2, hi.w the smallest):
// a unit out of a window's reach is out of reach of each of its chunks.
__global__ void k_window_box(const float4* __restrict__ tbox, int n_chunks, int n_windows,
                             float4* __restrict__ wbox) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_windows) return;
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, -INFINITY);
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, INFINITY);
    for (int c = 32 * t; c < min(n_chunks, 32 * (t + 1)); ++c) {
        const float4 a = tbox[2 * c], b = tbox[2 * c + 1];
        lo.x = fminf(lo.x, a.x), lo.y = fminf(lo.y, a.y), lo.z = fminf(lo.z, a.z);
        hi.x = fmaxf(hi.x, b.x), hi.y = fmaxf(hi.y, b.y), hi.z = fmaxf(hi.z, b.z);
        lo.w = fmaxf(lo.w, a.w);
        hi.w = fminf(hi.w, b.w);
    }
    wbox[2 * t] = lo;
    wbox[2 * t + 1] = hi;
}

// Spatial-order copies of the atlas for the GEMM modes (centroid rows point-major: point i as
// the float4 (x, y, z, 0), CROW4 per row).
__global__ void k_prep_spatial(AtlasView at, const int* __restrict__ sp_s, float4* cen_sp,
                               float* thr2_sp, float4* ctr_sp, float4* scr_sp, float4* end_sp) {
    const int c = blockIdx.x * blockDim.y + threadIdx.y;
    if (c >= at.M) {  // scr_sp's pad up to a whole chunk: a row no fiber passes
        if (c < (at.M + 31) / 32 * 32 && threadIdx.x == 0)
            scr_sp[c] = make_float4(0.0f, 0.0f, 0.0f, -INFINITY);
        return;
    }
    const int s = sp_s[c];
    const float* src = at.cen + (size_t)s * CROW;
    for (int k = threadIdx.x; k < CROW4; k += blockDim.x)
        cen_sp[(size_t)c * CROW4 + k] =
            k < NPTS ? make_float4(src[3 * k], src[3 * k + 1], src[3 * k + 2],
                                   k == 0 ? src[CROW - 1] : 0.0f)  // point 0's w: the length
                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (threadIdx.x == 0) {
        thr2_sp[c] = at.thr2[s];
        scr_sp[c] = at.scr2[s];
        ctr_sp[c] = make_float4(src[3 * CENTRE], src[3 * CENTRE + 1], src[3 * CENTRE + 2],
                                at.thr2[s]);
        end_sp[3 * (size_t)c] = make_float4(src[0], src[1], src[2], src[CROW - 1]);
        end_sp[3 * (size_t)c + 1] = ctr_sp[c];
        const int L = 3 * (NPTS - 1);
        end_sp[3 * (size_t)c + 2] = make_float4(src[L], src[L + 1], src[L + 2], 0.0f);
    }
}

// KE: K width of the operands in elements (64 for the directional columns, 32 for the
// orientation-free ones). A row of KE elements is split into K regions of at most 128 bytes,
// each loaded by its own TMA box and swizzled at its width (128 or 64 bytes).
template <int FMT, int KE, int R, int N, int S, int ABUF>
struct GemmCfg {
    static constexpr int ELEM = FMT == 1 ? 2 : 4;
    static constexpr int ROWB = KE * ELEM;                     // bytes of one operand row
    static constexpr int REGB = ROWB < 128 ? ROWB : 128;       // bytes of a row in one region
    static constexpr int KREG = ROWB / REGB;                   // K regions per row
    static constexpr int KSTEPS = ROWB / 32;                   // MMA K steps (32 bytes each)
    static constexpr int A_TILE = 128 * ROWB;                  // one 128-row fiber tile
    static constexpr int A_REGION = 128 * REGB;                // bytes of one K region
    static constexpr int B_TILE = N * ROWB;
    static constexpr int B_REGION = N * REGB;
    static constexpr int ACC_COLS = R * N;                     // TMEM columns per accumulator
    static constexpr int NACC = 512 / ACC_COLS;                // accumulators in TMEM
    static constexpr int A_OFF = 0;
    static constexpr int B_OFF = A_OFF + ABUF * R * A_TILE;
    static constexpr int BAR_OFF = B_OFF + S * B_TILE;
    static constexpr int NBAR = 2 * ABUF + 2 * S + 2 * NACC + 1;
    static constexpr int SMEM = BAR_OFF + NBAR * 8 + 16 + 1024;  // + alignment slack
    static_assert(NACC >= 2 && NACC * ACC_COLS <= 512, "two or more accumulators in TMEM");
    static_assert(N % 32 == 0 && N >= 32 && N <= 256, "N");
    static_assert(REGB == 128 || REGB == 64, "swizzle width");
    static_assert(A_TILE % 1024 == 0 && B_TILE % 1024 == 0, "1024-byte aligned tiles");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

struct Waiter {
    volatile int* abort;
    unsigned* status;
    unsigned long long limit_ns;  // 0: a wait not complete at its first try times out at once
    // wait for `parity` on `bar`; false if the CTA is aborting (another role timed out) or this
    // wait ran past its limit (then it starts the abort)
    __device__ bool wait(uint64_t* bar, uint32_t parity) const {
        if (mbar_try_wait(bar, parity)) return true;
        if (limit_ns == 0) {
            *abort = 1;
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
        // poll; look at the abort flag and the clock only every 1024 polls, so a completed
        // phase is seen without the latency of a timer read
        uint64_t t0 = 0;
        for (uint32_t i = 0;; ++i) {
            if (mbar_try_wait(bar, parity)) return true;
            if ((i & 1023u) == 0u) {
                if (*abort) return false;
                const uint64_t now = globaltimer_ns();
                if (i == 0) {
                    t0 = now;
                } else if (now - t0 > limit_ns) {
                    *abort = 1;
                    atomicOr(status, ST_TIMEOUT);
                    return false;
                }
            }
        }
    }
};

// One epilogue warp's reservation of block records (SLOT_GRAB at a time from the global count).
struct SlotGrab {
    unsigned long long next = 0, end = 0;
    __device__ unsigned long long take(const GemmScratch& g, int lane) {
        if (next == end) {
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(g.cnt, (unsigned long long)SLOT_GRAB);
            next = __shfl_sync(0xffffffffu, b, 0);
            end = next + SLOT_GRAB;
        }
        return next++;
    }
    // mark the reserved records this warp did not use, so the exact kernel skips them
    __device__ void close(const GemmScratch& g, int lane) {
        for (unsigned long long b = next + lane; b < end; b += 32)
            if ((long long)b < g.cap) g.hdr[b] = make_uint2(EMPTY_SLOT, 0u);
        next = end;
    }
};

template <int FMT, int KE, int R, int N, int S, int ABUF>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
k_gemm_screen(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              long long n_units, int n_tiles, int cols, GemmScratch g, unsigned* status) {
    using C = GemmCfg<FMT, KE, R, N, S, ABUF>;
    constexpr int CPT = N / 32;  // 32-column chunks per tile
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::BAR_OFF);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + ABUF;
    uint64_t* b_full = bars + 2 * ABUF;
    uint64_t* b_empty = bars + 2 * ABUF + S;
    uint64_t* acc_full = bars + 2 * ABUF + 2 * S;
    uint64_t* acc_empty = acc_full + C::NACC;
    uint64_t* mma_done = acc_full + 2 * C::NACC;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ unsigned long long s_umask[2][3][MAXW];  // mask rings of warps 0 and 1

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < ABUF; ++i) {
            mbar_init(a_full + i, 1);
            mbar_init(a_empty + i, 1);
        }
        for (int i = 0; i < S; ++i) {
            mbar_init(b_full + i, 1);
            mbar_init(b_empty + i, 1);
        }
        for (int i = 0; i < C::NACC; ++i) {
            mbar_init(acc_full + i, 1);
            mbar_init(acc_empty + i, EPI_WARPS);
        }
        mbar_init(mma_done, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const Waiter W{&s_abort, status, g.wait_ns};

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
        int stage = 0;
        uint32_t b_phase = 0;     // bit s: parity to wait on b_empty[s]
        uint32_t b_used = 0;      // bit s: stage s received a load
        uint32_t a_used = 0, a_par = 0;
        long long it = 0;
        bool ok = true;
        MaskRing ring;
        ring.init(s_umask[0], g, blockIdx.x, n_units);
        for (long long u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            const unsigned long long* um = ring.enter(g, u, n_units);
            if (u + gridDim.x < n_units)  // the next unit's fiber tile is brought into L2
                bulk_prefetch_l2(static_cast<const unsigned char*>(g.a) +
                                     (size_t)(u + gridDim.x) * R * C::A_TILE,
                                 (uint32_t)(R * C::A_TILE));
            if (!any_word(um, g.awords)) {  // every block of the unit is culled
                ring.leave();
                continue;
            }
            const int ab = ABUF == 2 ? (int)(it & 1) : 0;
            const long long use = ABUF == 2 ? (it >> 1) : it;  // uses of this A buffer so far
            if (use > 0) ok = W.wait(a_empty + ab, (uint32_t)((use - 1) & 1));
            if (!ok) break;
            a_used |= 1u << ab;
            a_par = (a_par & ~(1u << ab)) | ((uint32_t)(use & 1) << ab);
            unsigned char* sA = smem + C::A_OFF + ab * R * C::A_TILE;
            mbar_arrive_expect_tx(a_full + ab, (uint32_t)(R * C::A_TILE));
            for (int r = 0; r < R; ++r)
                for (int kr = 0; kr < C::KREG; ++kr)
                    tma_load_2d(sA + r * C::A_TILE + kr * C::A_REGION, &tmA,
                                kr * (C::REGB / C::ELEM),
                                (int)((u * R + r) * 128), a_full + ab);
#pragma unroll 1
            for (int wd = 0; wd < g.awords && ok; ++wd)
            for (unsigned long long bits = um[wd]; bits;) {
                const int t = next_tile<CPT>(bits, wd);
                if (!W.wait(b_empty + stage, ((b_phase >> stage) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                b_phase ^= 1u << stage;
                b_used |= 1u << stage;
                unsigned char* sB = smem + C::B_OFF + stage * C::B_TILE;
                mbar_arrive_expect_tx(b_full + stage, (uint32_t)C::B_TILE);
                for (int kr = 0; kr < C::KREG; ++kr)
                    tma_load_2d(sB + kr * C::B_REGION, &tmB, kr * (C::REGB / C::ELEM), t * N,
                                b_full + stage);
                stage = stage + 1 == S ? 0 : stage + 1;
            }
            ++it;
            ring.leave();
        }
        cp_async_wait_all();  // the ring's last copies
        if (s_abort) {
            // copies this thread issued may still be landing: wait for each buffer's last load
            // (b_phase bit s flipped once per load, so its complement is the last load's parity)
            for (int i = 0; i < S; ++i)
                if ((b_used >> i) & 1u) mbar_wait_bounded(b_full + i, ((b_phase >> i) & 1u) ^ 1u);
            for (int i = 0; i < ABUF; ++i)
                if ((a_used >> i) & 1u) mbar_wait_bounded(a_full + i, (a_par >> i) & 1u);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = make_idesc(FMT, 128, N);
        int stage = 0;
        uint32_t b_phase = 0;
        long long it = 0, tile = 0;
        bool ok = true;
        long long active = 0;
        MaskRing ring;
        ring.init(s_umask[1], g, blockIdx.x, n_units);
        for (long long u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            const unsigned long long* um = ring.enter(g, u, n_units);
            if (!any_word(um, g.awords)) {
                ring.leave();
                continue;
            }
            const int ab = ABUF == 2 ? (int)(it & 1) : 0;
            const long long use = ABUF == 2 ? (it >> 1) : it;
            if (!W.wait(a_full + ab, (uint32_t)(use & 1))) break;
            tc_fence_after();
            const uint64_t ad_unit =
                make_sdesc<C::REGB>(smem_u32(smem + C::A_OFF + ab * R * C::A_TILE));
#pragma unroll 1
            for (int wd = 0; wd < g.awords && ok; ++wd)
            for (unsigned long long bits = um[wd]; bits;) {
                (void)next_tile<CPT>(bits, wd);
                ++active;
                const int cb = (int)(tile % C::NACC);
                const long long cuse = tile / C::NACC;
                if (!W.wait(b_full + stage, (b_phase >> stage) & 1u)) {
                    ok = false;
                    break;
                }
                b_phase ^= 1u << stage;
                if (cuse > 0 && !W.wait(acc_empty + cb, (uint32_t)((cuse - 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // descriptors of the stage's first K step; step kk starts 32 kk bytes into the
                // row (region, then offset), added to the address field (16-byte units)
                const uint64_t bd0 = make_sdesc<C::REGB>(
                    smem_u32(smem + C::B_OFF + stage * C::B_TILE));
                for (int r = 0; r < R; ++r) {
                    const uint32_t d = tmem + (uint32_t)(cb * C::ACC_COLS + r * N);
                    const uint64_t ad0 = ad_unit + (uint64_t)((r * C::A_TILE) >> 4);
#pragma unroll
                    for (int kk = 0; kk < C::KSTEPS; ++kk) {
                        const int reg = (kk * 32) / C::REGB;
                        const uint32_t koff = (uint32_t)((kk * 32) % C::REGB);
                        const uint64_t ad = ad0 + (uint64_t)((reg * C::A_REGION + koff) >> 4);
                        const uint64_t bd = bd0 + (uint64_t)((reg * C::B_REGION + koff) >> 4);
                        if (FMT == 1)
                            mma_f16(d, ad, bd, idesc, kk > 0);
                        else
                            mma_tf32(d, ad, bd, idesc, kk > 0);
                    }
                }
                mma_commit(b_empty + stage);
                mma_commit(acc_full + cb);
                stage = stage + 1 == S ? 0 : stage + 1;
                ++tile;
            }
            mma_commit(a_empty + ab);
            ++it;
            ring.leave();
        }
        cp_async_wait_all();  // the ring's last copies
        atomicAdd(g.cnt + 3, (unsigned long long)(active * R * 128 * N));
        // every MMA and every commit above has completed once this arrives
        mma_commit(mma_done);
        mbar_wait_bounded(mma_done, 0);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        // Warp w reads TMEM lane quarter w % 4 (the hardware's rule) and, with the other
        // EPI_SUB - 1 warps of the same quarter, a share of the 32-column chunks of each
        // accumulator. Two tcgen05.ld.red are in flight per wait.
        constexpr int CPR = N / 32;               // chunks per fiber tile row block
        constexpr int CHUNKS = R * CPR;           // chunks per accumulator
        const int q = warp & 3;
        const int sub = (warp - 2) >> 2;  // which of the quarter's EPI_SUB warps
        SlotGrab slots;
        unsigned long long surv = 0;
        long long tile = 0;
        bool ok = true;
        // each unit's alpha values and mask words (one per lane, handed out by shuffles) are
        // loaded one unit ahead, so that a unit never starts on a memory round trip
        float aln[4];
        unsigned long long mwn[2];  // mask words lane and lane + 32 of the next unit
        auto load_unit = [&](long long u) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                aln[r] = r < R && u < n_units
                             ? __ldg(g.alpha + (u * R + r) * 128 + 32 * q + lane)
                             : INFINITY;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                mwn[h] = u < n_units && lane + 32 * h < g.awords
                             ? __ldg(g.amask + u * g.awords + lane + 32 * h)
                             : 0ull;
        };
        load_unit(blockIdx.x);
        for (long long u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
            float al[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) al[r] = aln[r];
            const unsigned long long mword0 = mwn[0], mword1 = mwn[1];
            load_unit(u + gridDim.x);
            const unsigned fib0 = (unsigned)(u * R * 128 + 32 * q + lane);
            for (int wd = 0; wd < g.awords && ok; ++wd)
            for (unsigned long long bits =
                     __shfl_sync(0xffffffffu, wd < 32 ? mword0 : mword1, wd & 31);
                 bits;) {
                const unsigned long long word = bits;
                const int t = next_tile<CPT>(bits, wd);
                // this tile's chunk bits: chunk c of the tile's columns may hold survivors
                const unsigned tb =
                    (unsigned)((word >> ((t % (64 / CPT)) * CPT)) & ((1ull << CPT) - 1));
                const int cb = (int)(tile % C::NACC);
                if (!W.wait(acc_full + cb, (uint32_t)((tile / C::NACC) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cb * C::ACC_COLS);
#pragma unroll 1
                for (int c0 = sub; c0 < CHUNKS; c0 += 2 * EPI_SUB) {
                    float v[2][32], mx[2];
                    // chunks whose centroid box is out of reach are not read
                    const bool act0 = (tb >> (c0 % CPR)) & 1u;
                    const bool act1 = c0 + EPI_SUB < CHUNKS && ((tb >> ((c0 + EPI_SUB) % CPR)) & 1u);
                    if (!act0 && !act1) continue;
                    if (act0) tmem_ld_red32(tbase + (uint32_t)(32 * c0), v[0], mx[0]);
                    if (act1) tmem_ld_red32(tbase + (uint32_t)(32 * (c0 + EPI_SUB)), v[1], mx[1]);
                    tmem_wait_ld();
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h == 0 && !act0) continue;
                        if (h == 1 && !act1) break;
                        const int c = c0 + EPI_SUB * h;
                        const int r = c / CPR;
                        const float a = r == 0 ? al[0] : r == 1 ? al[1] : r == 2 ? al[2] : al[3];
                        if (!__any_sync(0xffffffffu, mx[h] >= a)) continue;
                        // rare: each lane's surviving columns of the chunk as a bit mask; the
                        // warp's 32 masks form one block record
                        const unsigned col0 = (unsigned)(t * N + (c % CPR) * 32);
                        unsigned mask = 0;
#pragma unroll
                        for (int i = 0; i < 32; ++i) mask |= (v[h][i] >= a ? 1u : 0u) << i;
                        if (col0 + 32 > (unsigned)cols)
                            mask &= col0 >= (unsigned)cols ? 0u : (1u << (cols - col0)) - 1u;
                        if (!__any_sync(0xffffffffu, mask != 0u)) continue;
                        surv += __popc(mask);
                        const unsigned long long b = slots.take(g, lane);
                        const unsigned f = fib0 + (unsigned)(r * 128);
                        if ((long long)b < g.cap) {
                            g.mask[b * 32 + lane] = mask;
                            if (lane == 0) g.hdr[b] = make_uint2(f - (unsigned)lane, col0);
                        } else if (mask != 0u && g.flag[f] == 0) {
                            g.flag[f] = 1;  // no room: the fiber is rescanned exactly
                            atomicAdd(g.cnt + 1, 1ull);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty + cb);
                ++tile;
            }
        }
        __syncwarp();
        slots.close(g, lane);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) surv += __shfl_down_sync(0xffffffffu, surv, off);
        if (lane == 0 && surv) atomicAdd(g.cnt + 2, surv);
    }
    // drain: make sure no TMA copy is still landing in this CTA's shared memory
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 512);
}

// ---- SEG_MODE_PLAIN_CULLED: test1 on CUDA cores over the culled blocks ---------------------------
// The same locality order and centre-point culling as the tensor-core modes, with the paper's own
// first discarding test in place of the GEMM bound: test1 (Section 2.3, the centre point, shared
// by both orientations) in the plain kernel's dot-product form, a'.b' + (theta^2 - |b'|^2)/2 >=
// |a'|^2 / 2 with its rounding slack (so every pair the exact FP32 test1 accepts is kept). One
// warp per 32-fiber group, lane = fiber: the 32-centroid chunks whose box is within reach of the
// group's centre-point box are tested (a warp ballot over 32 chunks at a time), each chunk's 32
// screen rows staged in shared memory and read as broadcasts; the surviving columns of a chunk
// form a block record in the tensor-core modes' format (orientation-free columns: spatial
// centroid index), checked by the same exact kernel.
constexpr int CS_WARPS = 8;

__global__ void __launch_bounds__(CS_WARPS * 32)
k_culled_screen(long long n, long long n_groups, AtlasView at, GemmScratch g,
                const float4* __restrict__ scr_sp, const float4* __restrict__ ubox,
                const float4* __restrict__ tbox, int n_chunks) {
    __shared__ float4 s_q[CS_WARPS][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SlotGrab slots;
    unsigned long long surv = 0, screened = 0;
    const long long W = (long long)gridDim.x * CS_WARPS;
    for (long long gi = (long long)blockIdx.x * CS_WARPS + w; gi < n_groups; gi += W) {
        const long long f = gi * 32 + lane;
        float x = 0.0f, y = 0.0f, z = 0.0f, h = NAN;  // NaN never passes
        if (f < n && g.key[f] != NAN_KEY) {
            const float* c = g.fs + (size_t)f * CROW + 3 * CENTRE;
            x = c[0] - at.c0x;
            y = c[1] - at.c0y;
            z = c[2] - at.c0z;
            const float r2 = fmaf(x, x, fmaf(y, y, z * z));
            h = 0.5f * r2 - 1e-5f * r2 - 1e-3f;
        }
        const float4 lo = __ldg(ubox + 2 * gi), hi = __ldg(ubox + 2 * gi + 1);
        if (!(lo.x <= hi.x)) continue;  // no finite fiber in the group
        const UnitBox box{lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
        for (int k0 = 0; k0 < n_chunks; k0 += 32) {
            const int c = k0 + lane;
            unsigned act = __ballot_sync(0xffffffffu, c < n_chunks && block_active(box, tbox, c));
            while (act) {
                const int cc = k0 + __ffs(act) - 1;
                act &= act - 1;
                const int j = 32 * cc + lane;
                __syncwarp();
                s_q[w][lane] = j < at.M ? __ldg(scr_sp + j) : make_float4(0.f, 0.f, 0.f, -INFINITY);
                __syncwarp();
                unsigned m = 0u;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float4 q = s_q[w][i];
                    const float t = fmaf(z, q.z, fmaf(y, q.y, fmaf(x, q.x, q.w)));
                    m |= (t >= h ? 1u : 0u) << i;
                }
                screened += 32;
                if (!__any_sync(0xffffffffu, m != 0u)) continue;
                surv += __popc(m);
                const unsigned long long b = slots.take(g, lane);
                if ((long long)b < g.cap) {
                    g.mask[b * 32 + lane] = m;
                    if (lane == 0) g.hdr[b] = make_uint2((unsigned)(gi * 32), (unsigned)(32 * cc));
                } else if (m != 0u && g.flag[f] == 0) {
                    g.flag[f] = 1;  // no room: the fiber is rescanned exactly
                    atomicAdd(g.cnt + 1, 1ull);
                }
            }
        }
    }
    __syncwarp();
    slots.close(g, lane);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        surv += __shfl_down_sync(0xffffffffu, surv, off);
        screened += __shfl_down_sync(0xffffffffu, screened, off);
    }
    if (lane == 0) {
        if (surv) atomicAdd(g.cnt + 2, surv);
        if (screened) atomicAdd(g.cnt + 3, screened);
    }
}

// ---- exact test of the survivors, overflow rescan, finalize ------------------------------------

__device__ inline unsigned long long pack_key(float d2, int s, int o) {
    return ((unsigned long long)__float_as_uint(d2) << 32) | ((unsigned long long)s << 1) |
           (unsigned)o;
}

// Exact test of the survivors, one block record per CTA at a time. The CTA copies (cp.async) the
// block's 32 fiber rows (contiguous in the sorted copy) and the chunk's centroid rows into shared
// memory, with theta^2 beside each centroid and each fiber's best d^2 so far; the next record's
// header and masks are loaded while the current one is tested. Warp 0 lists the block's
// (fiber, column) pairs in shared memory (a prefix sum of the mask popcounts places each fiber's
// pairs). Phase A runs test1 and test2 (Section 2.3) on every pair and queues the
// pairs with a live orientation; phase B runs test3 and test4 on the queue, so that the lanes of
// a warp do the same stage of the test: first each fiber's queued pair with the smallest partial
// maximum (usually its best), then the rest, most of which the tightened bound now discards
// early. The bound is min(theta^2, the fiber's best so far);
// exits are strict (> bound), so equal distances still reach the atomicMin of the packed key and
// the tie rule of Algorithm 1 holds.
constexpr int EX_THREADS = 128;
// Centroid rows in shared memory, point-major as in the atlas's spatial copy (CROW4 float4 per
// row, so one block of 16-byte copies stages them): a warp's 16-byte loads of the same point
// of eight consecutive rows fall in eight different bank groups (21 is odd). 32 rows for
// orientation-free columns, 16 for directional ones.
template <bool INV>
struct CenRows {
    static constexpr int ROWS = INV ? 32 : 16;
};
constexpr int FS_STRIDE = 68;    // fiber row in shared memory (16-byte aligned copies)
constexpr int EX_QCAP = 32 * 32; // a block has at most 1024 pairs
constexpr int EX_QLEN = 384;     // queued pairs per block; a pair past the queue is finished
                                 // at once by the thread that tested it
static_assert(EX_QLEN <= 512, "s_first keeps a queue index in nine bits");
constexpr int EX_RUN = 16;       // consecutive records a CTA takes at a time

// Squared distance of fiber point i (63-float row) and centroid point j (float4 row): the
// same arithmetic as pd2, with the centroid point read in one 16-byte load.
__device__ __forceinline__ float pd2v(const float* a, int i, const float4* b, int j) {
    const float4 q = b[j];
    const float dx = a[3 * i] - q.x;
    const float dy = a[3 * i + 1] - q.y;
    const float dz = a[3 * i + 2] - q.z;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Stages of the exact test in orientation O (0: points in order, 1: reversed as in Eq. 2).
template <int O>
__device__ __forceinline__ float ends2(const float* a, const float4* b) {
    constexpr int L = NPTS - 1;
    return fmaxf(pd2v(a, 0, b, O ? L : 0), pd2v(a, L, b, O ? 0 : L));
}
template <int O>
__device__ __forceinline__ float mid4(const float* a, const float4* b, float m) {
    constexpr int L = NPTS - 1;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        m = fmaxf(m, pd2v(a, test3_point(q), b, O ? L - test3_point(q) : test3_point(q)));
    return m;
}
template <int O>
__device__ __forceinline__ float rest17(const float* a, const float4* b, float m) {
    constexpr int L = NPTS - 1;
#pragma unroll
    for (int i = 1; i < L; ++i)
        if (!is_early_point(i)) m = fmaxf(m, pd2v(a, i, b, O ? L - i : i));
    return m;
}

// ---- SEG_MODE_CULLED_FUSED: culling, test1 and the exact test in one pass per fiber group -----
// One warp owns a 32-fiber group of the locality order from start to finish: it gathers the
// group's 32 rows from the caller's array into shared memory once (odd row stride, so lanes
// reading different rows at one column never share a bank), tests the group's centre-point box
// against the 32-centroid chunks (a window of 32 chunks out of reach is skipped whole, the
// others take a ballot over their 32 chunks), and runs test1 in
// dot-product form for every pair of a chunk in reach (lane = fiber, the chunk's 32 screen rows
// read as broadcasts). The pairs that pass join a short per-warp list, column by column, and
// every 32 of them are one round of test2 (centre and end points, both orientations) with one
// pair per lane; the pairs that pass test2 join a second list, and every 32 of those are one
// round of test3 and test4 (Section 2.3). So the lanes of a round do the same stage of the
// test, whatever the chunk and column their pairs came from. Each fiber's packed key lives in
// shared memory (atomicMin; its high word is the fiber's best value, the bound of every later
// test), so there is no sorted copy, no record list and no overflow path. Groups come from a
// work counter.
constexpr int FZ_WARPS = 4;
constexpr int FZ_CTAS = 5;         // resident CTAs per SM (96 registers a thread)
constexpr int FZ_STRIDE = NC + 2;  // 65 floats per fiber row in shared memory (odd)

constexpr int FZ_QLEN = 64;  // queued pairs per warp: fewer than 32 wait, plus one round
constexpr int FZ_ALEN = 64;  // test1 survivors per warp: fewer than 32 wait, plus a column
constexpr int FZ_MAX_M = 1 << 25;  // a queued pair packs the centroid index in 25 bits

// 10,144 bytes a warp: five 4-warp CTAs an SM (with the 80 registers a thread that six would
// leave, and test1's rows read through L1, the kernel is slower).
struct FzWarp {
    float f[32 * FZ_STRIDE];   // the group's fiber rows (column 63: the fiber's length, for TN)
    float4 q[32];              // the current chunk's test1 rows
    unsigned long long key[32];  // packed keys; the high word is the fiber's best value so far
    float2 qm[FZ_QLEN];        // queued pairs: partial maxima after test2 (direct, reversed)
    unsigned qe[FZ_QLEN];      //   fiber | live direct << 5 | live reversed << 6 | centroid << 7
    unsigned al[FZ_ALEN];      // pairs that passed test1, waiting for test2: fiber | centroid << 5
    float box[8];              // the group's centre-point box (lo xyz, hi xyz)
};

// A fiber's best key value so far (the float bits in its key's high word; all ones when none).
__device__ __forceinline__ float fz_best(const FzWarp& S, int fl) {
    return __uint_as_float(reinterpret_cast<const unsigned*>(S.key)[2 * fl + 1]);
}

// Phase A of a pair: test1 and test2 (centre and end points) of fiber a (shared, 63 floats)
// against the centroid's points 0, 10, 20, both orientations (the one the end points infer with
// cls == CLS_PAPER). The same arithmetic as the exact kernel's. Returns the live orientations (bit 0 direct, bit 1
// reversed) and their partial maxima.
__device__ __forceinline__ float pd2q(float3 p, float4 q) {
    const float dx = p.x - q.x;
    const float dy = p.y - q.y;
    const float dz = p.z - q.z;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// test3 and test4 stages (as mid4 / rest17) in an orientation o chosen per lane: fiber point i
// pairs with centroid point i (o = 0) or 20 - i (o = 1).
__device__ __forceinline__ float fz_mid4(const float* a, const float4* b, float m, int o) {
    constexpr int L = NPTS - 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = test3_point(q);
        m = fmaxf(m, pd2v(a, i, b, o ? L - i : i));
    }
    return m;
}
__device__ __forceinline__ float fz_rest17(const float* a, const float4* b, float m, int o) {
    constexpr int L = NPTS - 1;
#pragma unroll
    for (int i = 1; i < L; ++i)
        if (!is_early_point(i)) m = fmaxf(m, pd2v(a, i, b, o ? L - i : i));
    return m;
}

// p0, p10, p20: the fiber's points 0, 10, 20; q0, q10, q20: the centroid's.
__device__ __forceinline__ unsigned fz_phase_a(float3 p0, float3 p10, float3 p20, float4 q0,
                                               float4 q10, float4 q20, float bound, int cls,
                                               float& md, float& mr, unsigned& npd) {
    const float c = pd2q(p10, q10);
    npd += 1;
    if (!(c <= bound)) return 0u;
    md = fmaxf(c, fmaxf(pd2q(p0, q0), pd2q(p20, q20)));
    mr = fmaxf(c, fmaxf(pd2q(p0, q20), pd2q(p20, q0)));
    npd += 4;
    bool ad = md <= bound, ar = mr <= bound;
    if (cls == CLS_PAPER) {  // direction inferred from the end points
        const bool direct = md <= mr;
        ad = ad && direct;
        ar = ar && !direct;
    }
    return (ad ? 1u : 0u) | (ar ? 2u : 0u);
}

// Phase B of a queued pair: test3 and test4 in its live orientations against min(theta^2, the
// fiber's best so far), then the merge into the fiber's packed key (Algorithm 1's tie rule:
// exits are strict, so equal values still reach the atomicMin of the key).
template <bool EXT>
__device__ __forceinline__ void fz_phase_b(FzWarp& S, int e, const AtlasView& at,
                                           const GemmScratch& g, const unsigned* perm,
                                           long long f0, unsigned& npd) {
    const unsigned fl_bits = S.qe[e];
    const int fl = (int)(fl_bits & 31u), j = (int)(fl_bits >> 7);
    const float2 mm = S.qm[e];
    const float* a = S.f + fl * FZ_STRIDE;
    const float4* b = g.cen_sp + (size_t)j * CROW4;
    const float t2 = __ldg(g.thr2_sp + j);
    const float bound = pair_bound2(at, t2, key_bound2(fz_best(S, fl), at.cls));
    float md = mm.x, mr = mm.y;
    bool ad = ((fl_bits >> 5) & 1u) && md <= bound;
    bool ar = ((fl_bits >> 6) & 1u) && mr <= bound;
    // Each lane's first live orientation runs in one code path for the whole warp (the
    // centroid point it pairs with is picked per lane), so a round whose pairs differ in
    // orientation does not run twice; the reversed one runs again only where both are live.
    const int o = ad ? 0 : 1;
    float m = ad ? md : mr;
    bool live = ad || ar;
    bool live2 = ad && ar;
    float m2 = mr;
    if (live) { m = fz_mid4(a, b, m, o); live = m <= bound; npd += 4; }
    if (live2) { m2 = fz_mid4(a, b, m2, 1); live2 = m2 <= bound; npd += 4; }
    if (live) { m = fz_rest17(a, b, m, o); live = m <= bound; npd += 14; }
    if (live2) { m2 = fz_rest17(a, b, m2, 1); live2 = m2 <= bound; npd += 14; }
    if (o == 0) {
        md = m;
        ad = live;
        mr = m2;
        ar = live2;
    } else {
        mr = m;
        ar = live;
    }
    if (!(ad || ar)) return;
    const bool dir = ad && (!ar || md <= mr);
    const float d2 = dir ? md : mr;
    float kf;
    if (key_value(at.cls, d2, t2, a[NC], __ldg(&b[0].w), kf)) {
        const int sidx = __ldg(g.sp_s + j);
        atomicMin(&S.key[fl], pack_key(kf, sidx, dir ? 0 : 1));
        if (EXT && at.multi) multi_mark(at, perm[f0 + fl], at.bundle[sidx]);
    }
}

template <bool EXT>
__global__ void __launch_bounds__(FZ_WARPS * 32, FZ_CTAS)
k_fused(FiberSrc src, const unsigned* __restrict__ perm, long long n, long long n_groups,
        AtlasView at_in, GemmScratch g, const float4* __restrict__ scr_sp,
        const float4* __restrict__ tbox, const float4* __restrict__ wbox, int n_chunks,
        int* labels, float* dist, int* cidx, unsigned char* orient) {
    extern __shared__ __align__(16) unsigned char fz_smem[];
    AtlasView at = at_in;
    if (!EXT) {
        at.cls = CLS_EQ2;
        at.multi = nullptr;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    FzWarp& S = reinterpret_cast<FzWarp*>(fz_smem)[w];
    unsigned npd = 0;
    // groups taken from a counter (their costs vary with the density of the atlas around
    // them; a fixed stride left a long tail), the next one fetched while this one finishes
    long long grp = 0;
    if (lane == 0) grp = (long long)atomicAdd(g.cnt + 4, 1ull);
    grp = __shfl_sync(0xffffffffu, grp, 0);
    while (grp < n_groups) {
        const long long f0 = grp * 32;
        const int rows_in = (int)max(0LL, min(32LL, n - f0));
        int qn = 0;  // queued pairs (warp-uniform)
        int na = 0;  // listed test1 survivors (warp-uniform)
        // one round of test2 (centre and end points) on 32 listed pairs (`valid`: this lane's
        // entry is one); the pairs that pass join the queue, and each full 32 of the queue is
        // one round of test3/test4
        auto test2_round = [&](unsigned ent, bool valid) {
            const int fl = (int)(ent & 31u), j = (int)(ent >> 5);
            const float4* r = g.end_sp + 3 * (size_t)j;
            const float4 q10 = __ldg(r + 1);  // w: theta^2
            const float4 q0 = __ldg(r), q20 = __ldg(r + 2);
            const float* a = S.f + fl * FZ_STRIDE;
            const float3 p0 = make_float3(a[0], a[1], a[2]);
            const float3 p10 = make_float3(a[3 * CENTRE], a[3 * CENTRE + 1], a[3 * CENTRE + 2]);
            const float3 p20 = make_float3(a[3 * (NPTS - 1)], a[3 * (NPTS - 1) + 1],
                                           a[3 * (NPTS - 1) + 2]);
            unsigned live = 0u;
            float md = 0.0f, mr = 0.0f;
            if (valid)
                live = fz_phase_a(p0, p10, p20, q0, q10, q20,
                                  pair_bound2(at, q10.w, key_bound2(fz_best(S, fl), at.cls)),
                                  at.cls, md, mr, npd);
            const unsigned bal = __ballot_sync(0xffffffffu, live != 0u);
            if (live) {
                const int e = qn + __popc(bal & ((1u << lane) - 1u));
                S.qm[e] = make_float2(md, mr);
                S.qe[e] = (unsigned)fl | (live << 5) | ((unsigned)j << 7);
            }
            qn += __popc(bal);
            __syncwarp();
            if (qn >= 32) {  // one coherent round of test3/test4: the newest 32
                qn -= 32;
                fz_phase_b<EXT>(S, qn + lane, at, g, perm, f0, npd);
                __syncwarp();
            }
        };
        // 1. the group's rows (all copies in flight together)
        const unsigned my_src = lane < rows_in ? __ldg(perm + f0 + lane) : 0u;
        const float* my_row = src.row(my_src);  // (a work-table search per lane, not per row)
        __syncwarp();
#pragma unroll 4
        for (int r = 0; r < rows_in; ++r) {
            const float* p = shfl_ptr(my_row, r);
            cp_async4(S.f + r * FZ_STRIDE + lane, p + lane);
            if (lane < NC - 32) cp_async4(S.f + r * FZ_STRIDE + 32 + lane, p + 32 + lane);
        }
        cp_async_wait_all();
        __syncwarp();
        // 2. this lane's fiber: screen values, key, length; the group's centre-point box
        const float* a = S.f + lane * FZ_STRIDE;
        bool finite = lane < rows_in;  // every centred coordinate finite, as in the other modes
#pragma unroll
        for (int k = 0; k < NC; k += 3)
            finite &= isfinite(a[k] - at.c0x) & isfinite(a[k + 1] - at.c0y) &
                      isfinite(a[k + 2] - at.c0z);
        float x = 0.f, y = 0.f, z = 0.f, h = NAN;  // NaN never passes test1
        if (finite) {
            x = a[3 * CENTRE] - at.c0x;
            y = a[3 * CENTRE + 1] - at.c0y;
            z = a[3 * CENTRE + 2] - at.c0z;
            const float r2 = fmaf(x, x, fmaf(y, y, z * z));
            h = 0.5f * r2 - 1e-5f * r2 - 1e-3f;
        }
        S.key[lane] = finite ? ~0ull : NAN_KEY;
        S.f[lane * FZ_STRIDE + NC] = at.cls != CLS_EQ2 && finite ? poly_length(a) : 0.0f;
        {   // (kept in shared memory: it is read once per 32 chunks)
            float lo[3], hi[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const float c = finite ? a[3 * CENTRE + r] : 0.0f;
                lo[r] = warp_min(finite ? c : INFINITY);
                hi[r] = warp_max(finite ? c : -INFINITY);
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                if (lane == r) S.box[r] = lo[r];
                if (lane == r + 3) S.box[r + 3] = hi[r];
            }
        }
        __syncwarp();
        unsigned surv = 0, blocks = 0;  // this group's test1 survivors (lane), chunks tested
        // 3. the chunks in reach
        const bool any_finite = S.box[0] <= S.box[3];
        for (int k0 = 0; any_finite && k0 < n_chunks; k0 += 32) {
            const int cq = k0 + lane;
            const UnitBox box{S.box[0], S.box[1], S.box[2], S.box[3], S.box[4], S.box[5]};
            if (!block_active(box, wbox, k0 / 32)) continue;  // the whole window out of reach
            unsigned act = __ballot_sync(0xffffffffu, cq < n_chunks && block_active(box, tbox, cq));
            while (act) {
                const int cc = k0 + __ffs(act) - 1;
                act &= act - 1;
                S.q[lane] = __ldg(scr_sp + 32 * (size_t)cc + lane);  // padded to whole chunks
                // test1 against min(theta^2, the fiber's best so far): the dot-product form's
                // threshold h rises by half of (theta^2 - best) where that is positive; with the
                // chunk's smallest theta^2 in place of each centroid's and a margin far above
                // the rounding of the difference and of the sum, the rise never drops a pair
                // the exact test could accept (its bound is the same minimum)
                float he = h;
                if (!at.multi) {
                    const float tmin = __ldg(&tbox[2 * cc + 1].w);
                    const float bb = key_bound2(fz_best(S, lane), at.cls);
                    he = h + fmaxf(0.0f, fmaf(0.5f, tmin - bb,
                                              -(1e-5f * (tmin + fabsf(h)) + 1e-4f)));
                }
                __syncwarp();
                unsigned m = 0u;  // test1 (dot-product form with its slack) of this lane's fiber
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float4 q = S.q[i];  // the same row for every lane: a broadcast
                    const float t = fmaf(z, q.z, fmaf(y, q.y, fmaf(x, q.x, q.w)));
                    m |= (t >= he ? 1u : 0u) << i;
                }
                ++blocks;
                __syncwarp();
                if (!__any_sync(0xffffffffu, m != 0u)) continue;
                surv += __popc(m);
                // the chunk's survivors join the warp's list column by column (a ballot per
                // column that any fiber passed); each full 32 is one round of test2
                unsigned cols = __reduce_or_sync(0xffffffffu, m);
                while (cols) {
                    const int b = __ffs(cols) - 1;
                    cols &= cols - 1;
                    const unsigned v = __ballot_sync(0xffffffffu, (m >> b) & 1u);
                    if ((m >> b) & 1u)
                        S.al[na + __popc(v & ((1u << lane) - 1u))] =
                            (unsigned)lane | ((unsigned)(32 * cc + b) << 5);
                    na += __popc(v);
                    if (na >= 32) {
                        __syncwarp();
                        na -= 32;
                        test2_round(S.al[na + lane], true);
                    }
                }
                __syncwarp();
            }
        }
        if (na > 0) {  // the group's last test1 survivors
            __syncwarp();
            test2_round(S.al[lane < na ? lane : 0], lane < na);
            na = 0;
        }
        if (qn > 0) {  // the group's last queued pairs
            if (lane < qn) fz_phase_b<EXT>(S, lane, at, g, perm, f0, npd);
            qn = 0;
        }
        __syncwarp();
        long long next = 0;
        surv = __reduce_add_sync(0xffffffffu, surv);
        if (lane == 0) {
            next = (long long)atomicAdd(g.cnt + 4, 1ull);
            if (surv) atomicAdd(g.cnt + 2, (unsigned long long)surv);
            if (blocks) atomicAdd(g.cnt + 3, 1024ull * blocks);
        }
        // 4. results in the caller's order
        if (lane < rows_in) {
            const unsigned long long k = S.key[lane];
            long long o2 = my_src;
            int* lab = labels;
            float* dst = dist;
            int* ci = cidx;
            unsigned char* ori = orient;
            if (src.table) {
                const BatchEntry& e = src.table[src.subject(o2)];
                lab = e.labels;
                dst = e.dist;
                ci = nullptr;
                ori = nullptr;
                o2 -= e.first;
            }
            if (k == NAN_KEY || k == ~0ull) {
                lab[o2] = -1;
                if (dst) dst[o2] = k == NAN_KEY ? NAN : INFINITY;
                if (ci) ci[o2] = -1;
                if (ori) ori[o2] = 0;
            } else {
                const int sidx = (int)((k & 0xffffffffull) >> 1);
                const float kf = __uint_as_float((unsigned)(k >> 32));
                lab[o2] = at.bundle[sidx];
                if (dst) dst[o2] = at.cls != CLS_EQ2 ? kf : sqrtf(kf);
                if (ci) ci[o2] = at.perm[sidx];
                if (ori) ori[o2] = (unsigned char)(k & 1ull);
            }
        }
        grp = __shfl_sync(0xffffffffu, next, 0);
    }
    unsigned long long tot = npd;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, off);
    if (lane == 0 && tot) atomicAdd(g.cnt + 5, tot);
}

__global__ void k_gemm_stats(const unsigned long long* __restrict__ cnt, long long pairs,
                             long long* __restrict__ stats) {
    stats[0] = pairs;
    stats[1] = (long long)cnt[2];
    stats[2] = (long long)cnt[1];
    stats[3] = (long long)cnt[3];
    stats[4] = (long long)cnt[5];
}

constexpr unsigned DONE_ENTRY = 0xFFFFFFFFu;  // queue entry already tested

// test3 and test4 of one queued pair (its live orientations and partial maxima from phase A),
// against min(theta^2, the fiber's best so far); a pass is merged into the fiber's packed key
// and its best. A tighter bound than phase A's discards only pairs strictly worse than a pair
// already merged.
template <bool INV>
__device__ __forceinline__ void exact_entry(unsigned ent, float2 mm, const float* s_fib,
                                            const float4* s_cen, const float* s_thr,
                                            const int* s_sidx, unsigned* s_best,
                                            unsigned long long* key, unsigned& npd,
                                            const AtlasView& at, const unsigned* perm) {
    const int cls = at.cls;
    const int lo = (int)(ent & 31u), bit = (int)((ent >> 5) & 31u);
    const int j = INV ? bit : bit >> 1;
    const float* a = s_fib + lo * FS_STRIDE;
    const float4* b = s_cen + j * CROW4;
    const float bound =
        pair_bound2(at, s_thr[j], key_bound2(__uint_as_float(s_best[lo]), cls));
    float md = mm.x, mr = mm.y, d2;
    int o;
    bool pass;
    if (INV) {
        bool ad = ((ent >> 10) & 1u) && md <= bound;
        bool ar = ((ent >> 11) & 1u) && mr <= bound;
        if (ad) { md = mid4<0>(a, b, md); ad = md <= bound; npd += 4; }
        if (ar) { mr = mid4<1>(a, b, mr); ar = mr <= bound; npd += 4; }
        if (ad) { md = rest17<0>(a, b, md); ad = md <= bound; npd += 14; }
        if (ar) { mr = rest17<1>(a, b, mr); ar = mr <= bound; npd += 14; }
        pass = ad || ar;
        if (ad && (!ar || md <= mr)) { d2 = md; o = 0; } else { d2 = mr; o = 1; }
    } else {
        o = bit & 1;
        pass = md <= bound;
        if (pass) { md = o ? mid4<1>(a, b, md) : mid4<0>(a, b, md); pass = md <= bound; npd += 4; }
        if (pass) { md = o ? rest17<1>(a, b, md) : rest17<0>(a, b, md); pass = md <= bound; npd += 14; }
        d2 = md;
    }
    float kf;
    // a[63]: the fiber's length, b[0].w: the centroid's (the TN term)
    if (pass && key_value(cls, d2, s_thr[j], a[NC], b[0].w, kf)) {
        atomicMin(key + lo, pack_key(kf, s_sidx[j], o));
        if (at.multi) multi_mark(at, perm[lo], at.bundle[s_sidx[j]]);
        atomicMin(s_best + lo, __float_as_uint(kf));
    }
}

// EXT: the classification is not plain Eq. 2 or every passing bundle is wanted; without it the
// kernel's view is fixed to Eq. 2 and no multi-label output, which the compiler folds away.
template <bool INV, bool EXT>
__global__ void __launch_bounds__(EX_THREADS, 9)
k_exact_blocks(AtlasView at_in, GemmScratch g) {
    AtlasView at = at_in;
    if (!EXT) {
        at.cls = CLS_EQ2;
        at.multi = nullptr;
    }
    __shared__ __align__(16) float s_fib[32 * FS_STRIDE];
    __shared__ __align__(16) float4 s_cen[CenRows<INV>::ROWS * CROW4];
    __shared__ float s_thr[32];              // theta^2 of each centroid row
    __shared__ unsigned s_pre[32], s_best[32];
    __shared__ int s_sidx[32];               // sorted (bundle-major) index of each centroid row
    __shared__ unsigned s_q[EX_QLEN];        // fiber | bit << 5 | direct alive << 10 | rev << 11
    __shared__ float2 s_qm[EX_QLEN];         // partial maxima of the queued pairs
    __shared__ unsigned s_nq;
    // per fiber: its most promising queued pair, as the partial maximum's bits with the low
    // nine replaced by the queue index (the order only guides which pair goes first)
    __shared__ unsigned s_first[32];
    __shared__ unsigned short s_pair[EX_QCAP];  // the block's pairs: fiber | bit << 5
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const long long cnt = min((long long)*g.cnt, g.cap);
    __shared__ long long s_run;
    // Records are taken in runs of EX_RUN consecutive ones: an epilogue warp writes its records
    // for the same 32 fibers one after another, so consecutive records usually share their
    // fiber rows (kept in shared memory) and each fiber's best so far.
    long long blk = 0, blk_end = 0;
    unsigned cur = EMPTY_SLOT;  // first fiber of the rows in s_fib
    unsigned npd = 0;           // point distances this thread evaluated (statistics)
    uint2 hn = make_uint2(EMPTY_SLOT, 0u);  // the next record's header and masks, loaded one
    unsigned mn = 0u;                       // record ahead
    for (;;) {
        if (blk == blk_end) {
            __syncthreads();
            if (tid == 0) s_run = (long long)atomicAdd(g.cnt + 4, (unsigned long long)EX_RUN);
            __syncthreads();
            blk = s_run;
            if (blk >= cnt) break;
            blk_end = min(blk + EX_RUN, cnt);
            hn = g.hdr[blk];
            mn = g.mask[blk * 32 + lane];
        }
        const uint2 h = hn;
        const unsigned m = mn;
        ++blk;
        if (blk < blk_end) {
            hn = g.hdr[blk];
            mn = g.mask[blk * 32 + lane];
        }
        if (h.x == EMPTY_SLOT) continue;
        const unsigned s0 = INV ? h.y : h.y >> 1;
        const bool same = h.x == cur;
        // the 32 sorted fiber rows (16-byte copies; kept from the previous record when it had
        // the same fibers) and the chunk's centroid rows (4-byte copies into conflict-free
        // rows), theta^2 beside each centroid
        const float* fsrc = g.fs + (size_t)h.x * CROW;
        if (!same) {
#pragma unroll
            for (int c = tid; c < 32 * (CROW / 4); c += EX_THREADS)
                cp_async16(s_fib + (c >> 4) * FS_STRIDE + 4 * (c & 15), fsrc + 4 * c);
        }
        cur = h.x;
        const int ncen = min(CenRows<INV>::ROWS, at.M - (int)s0);
        const float4* csrc = g.cen_sp + (size_t)s0 * CROW4;
        for (int c = tid; c < ncen * CROW4; c += EX_THREADS)
            cp_async16(reinterpret_cast<float*>(s_cen + c), reinterpret_cast<const float*>(csrc + c));
        if (tid < ncen) {
            s_thr[tid] = __ldg(g.thr2_sp + s0 + tid);
            s_sidx[tid] = __ldg(g.sp_s + s0 + tid);
        }
        if (w == 0) {
            unsigned incl = __popc(m);
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            s_pre[lane] = incl;
            // this fiber's pairs, numbered after the previous fibers'
            unsigned k = incl - __popc(m);
            for (unsigned mm = m; mm; mm &= mm - 1, ++k)
                s_pair[k] = (unsigned short)(lane | ((__ffs(mm) - 1) << 5));
            const unsigned kb = (unsigned)(g.key[h.x + lane] >> 32);
            s_best[lane] = same ? min(s_best[lane], kb) : kb;
            s_first[lane] = ~0u;
            if (lane == 0) s_nq = 0;
        }
        cp_async_wait_all();
        __syncthreads();
        const unsigned total = s_pre[31];
        // phase A: test1 and test2 on every pair
        for (unsigned p0 = 0; p0 < total; p0 += EX_THREADS) {
            const unsigned p = p0 + (unsigned)tid;
            bool push = false;
            unsigned ent = 0;
            float md = 0.0f, mr = 0.0f;
            if (p < total) {
                const unsigned pr = s_pair[p];
                const int lo = (int)(pr & 31u), bit = (int)(pr >> 5);
                const float* a = s_fib + lo * FS_STRIDE;
                const int j = INV ? bit : bit >> 1;
                const float4* b = s_cen + j * CROW4;
                const float bound =
                    pair_bound2(at, s_thr[j],
                                key_bound2(__uint_as_float(s_best[lo]), at.cls));
                const float c = pd2v(a, CENTRE, b, CENTRE);
                npd += 1;
                if (c <= bound) {
                    bool ad, ar = false;
                    if (INV) {
                        md = fmaxf(c, ends2<0>(a, b));
                        npd += 4;
                        mr = fmaxf(c, ends2<1>(a, b));
                        ad = md <= bound;
                        ar = mr <= bound;
                        if (at.cls == CLS_PAPER) {  // direction inferred from the end points
                            const bool direct = md <= mr;
                            ad = ad && direct;
                            ar = ar && !direct;
                        }
                    } else {
                        md = fmaxf(c, (bit & 1) ? ends2<1>(a, b) : ends2<0>(a, b));
                        npd += 2;
                        ad = md <= bound;
                        if (at.cls == CLS_PAPER) {  // this column's orientation must be the
                            // one the end points infer (the other column, if it survived the
                            // screen, carries the other)
                            const float other = fmaxf(c, (bit & 1) ? ends2<0>(a, b)
                                                                   : ends2<1>(a, b));
                            npd += 2;
                            const float dmax = (bit & 1) ? other : md;  // direct
                            const float rmax = (bit & 1) ? md : other;  // reversed
                            ad = ad && (((bit & 1) == 0) == (dmax <= rmax));
                        }
                    }
                    push = ad || ar;
                    ent = (unsigned)lo | ((unsigned)bit << 5) | ((unsigned)ad << 10) |
                          ((unsigned)ar << 11);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, push);
            unsigned base = 0;
            if (lane == 0 && bal) base = atomicAdd(&s_nq, (unsigned)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (push && base + __popc(bal & lt) >= EX_QLEN) {
                exact_entry<INV>(ent, make_float2(md, mr), s_fib, s_cen, s_thr, s_sidx, s_best,
                                 g.key + h.x, npd, at, g.perm + h.x);
                push = false;
            }
            if (push) {
                const unsigned q = base + __popc(bal & lt);
                s_q[q] = ent;
                s_qm[q] = make_float2(md, mr);
                // the fiber's most promising pair: smallest partial maximum of a live
                // orientation (non-negative floats order as their bit patterns)
                const float pm = (ent >> 10) & 1u ? ((ent >> 11) & 1u ? fminf(md, mr) : md) : mr;
                atomicMin(s_first + (ent & 31u), (__float_as_uint(pm) & ~511u) | q);
            }
        }
        __syncthreads();
        // phase B1: each fiber's most promising pair first, so that the others meet a tight
        // bound; phase B2: the rest of the queue
        if (tid < 32 && s_first[tid] != ~0u) {
            const unsigned q = s_first[tid] & 511u;
            exact_entry<INV>(s_q[q], s_qm[q], s_fib, s_cen, s_thr, s_sidx, s_best, g.key + h.x,
                             npd, at, g.perm + h.x);
            s_q[q] = DONE_ENTRY;
        }
        __syncthreads();
        const unsigned nq = min(s_nq, (unsigned)EX_QLEN);
        for (unsigned q = tid; q < nq; q += EX_THREADS) {
            const unsigned ent = s_q[q];
            if (ent != DONE_ENTRY)
                exact_entry<INV>(ent, s_qm[q], s_fib, s_cen, s_thr, s_sidx, s_best, g.key + h.x,
                                 npd, at, g.perm + h.x);
        }
        __syncthreads();  // the buffers are refilled for the next record
    }
    unsigned long long tot = npd;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, off);
    if (lane == 0 && tot) atomicAdd(g.cnt + 5, tot);
}

// Fibers whose survivors did not fit the record list: exact scan against the whole atlas (the
// kernel returns at once when no fiber was flagged).
__device__ __noinline__ void rescan_fiber(long long f, const AtlasView& at, const GemmScratch& g) {
    const float* src = g.fs + (size_t)f * CROW;
    float a[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) a[k] = __ldg(src + k);
    const float ls = __ldg(src + NC);  // the fiber's length (TN term)
    for (int s = 0; s < at.M; ++s) {
        const float t2 = __ldg(at.thr2 + s);
        const float bound =
            pair_bound2(at, t2,
                        key_bound2(__uint_as_float((unsigned)(g.key[f] >> 32)), at.cls));
        float d2, kf;
        int o;
        if (exact_pair(a, at.cen + (size_t)s * CROW, bound, d2, o, at.cls) &&
            key_value(at.cls, d2, t2, ls, __ldg(at.cen + (size_t)s * CROW + NC), kf)) {
            atomicMin(g.key + f, pack_key(kf, s, o));
            multi_mark(at, g.perm[f], at.bundle[s]);
        }
    }
}

__global__ void k_overflow_rescan(long long n, AtlasView at, GemmScratch g) {
    if (*(volatile unsigned long long*)(g.cnt + 1) == 0) return;
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < n;
         f += (long long)gridDim.x * blockDim.x)
        if (g.flag[f]) rescan_fiber(f, at, g);
}

// Labels and distances in the caller's order (for several subjects: into each subject's
// arrays; cidx and orient are not written then).
__global__ void k_finalize(long long n, AtlasView at, GemmScratch g, FiberSrc src, int* labels,
                           float* dist, int* __restrict__ cidx,
                           unsigned char* __restrict__ orient, long long pairs,
                           long long* __restrict__ stats) {
    const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (f == 0 && stats) {
        stats[0] = pairs;
        stats[1] = (long long)g.cnt[2];
        stats[2] = (long long)g.cnt[1];
        stats[3] = (long long)g.cnt[3];
        stats[4] = (long long)g.cnt[5];
    }
    if (f >= n) return;
    const unsigned long long k = g.key[f];
    long long o = g.perm[f];  // results go to the caller's order
    if (src.table) {
        const BatchEntry& e = src.table[src.subject(o)];
        labels = e.labels;
        dist = e.dist;
        cidx = nullptr;
        orient = nullptr;
        o -= e.first;
    }
    if (k == NAN_KEY || k == ~0ull) {
        labels[o] = -1;
        if (dist) dist[o] = k == NAN_KEY ? NAN : INFINITY;
        if (cidx) cidx[o] = -1;
        if (orient) orient[o] = 0;
        return;
    }
    const int s = (int)((k & 0xffffffffull) >> 1);
    labels[o] = at.bundle[s];
    const float kf = __uint_as_float((unsigned)(k >> 32));
    if (dist) dist[o] = at.cls != 0 ? kf : sqrtf(kf);  // D, or sqrt(d^2)
    if (cidx) cidx[o] = at.perm[s];
    if (orient) orient[o] = (unsigned char)(k & 1ull);
}

// Diagnostic output of the screen (seg_gemm_screen_bits): every surviving (fiber, column) of the
// block records as one bit per (caller fiber, caller centroid [, orientation]); one warp per
// record, lanes over its 32 fibers.
__global__ void k_survivor_bits(long long n, AtlasView at, GemmScratch g, int inv,
                                unsigned* __restrict__ bits, long long words,
                                long long pairs, long long* __restrict__ stats) {
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w0 == 0 && lane == 0 && stats) {
        stats[0] = pairs;
        stats[1] = (long long)g.cnt[2];
        stats[2] = (long long)g.cnt[1];
        stats[3] = (long long)g.cnt[3];
        stats[4] = 0;
    }
    const long long cnt = min((long long)g.cnt[0], g.cap);
    for (long long b = w0; b < cnt; b += nw) {
        const uint2 h = g.hdr[b];
        if (h.x == EMPTY_SLOT) continue;
        const long long f = (long long)h.x + lane;
        unsigned m = g.mask[b * 32 + lane];
        if (f >= n) continue;
        const long long fo = g.perm[f];
        for (; m; m &= m - 1) {
            const unsigned col = h.y + (unsigned)(__ffs(m) - 1);
            const int sp = inv ? (int)col : (int)(col >> 1);
            const long long c = at.perm[g.sp_s[sp]];
            const long long bit = inv ? c : 2 * c + (col & 1u);
            atomicOr(bits + fo * words + (bit >> 5), 1u << (bit & 31));
        }
    }
}

// ---- host side ---------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// rows x ke operand, K-major, box of box_rows rows and one K region (128 bytes, swizzled at
// 128, or a whole 64-byte row, swizzled at 64).
bool make_tmap(CUtensorMap* m, const void* ptr, long long rows, int fmt, int ke, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int elem = fmt == 1 ? 2 : 4;
    const int regb = ke * elem < 128 ? ke * elem : 128;
    cuuint64_t dims[2] = {(cuuint64_t)ke, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ke * elem)};
    cuuint32_t box[2] = {(cuuint32_t)(regb / elem), (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_TFLOAT32, 2,
              const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              regb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct GemmShape {
    int fmt, ke, R, N, S, ABUF;
};

// Tile shapes per mode; entry 0 is the default.
// Narrower tiles leave room in TMEM for more accumulators (512 / (R N)), so the MMAs can run
// further ahead of the epilogue.
const GemmShape kDirBf16Shapes[] = {{1, 64, 1, 256, 3, 2}, {1, 64, 1, 128, 6, 2}, {1, 64, 1, 64, 8, 2}};
const GemmShape kDirTf32Shapes[] = {{2, 64, 1, 256, 2, 2}, {2, 64, 1, 128, 4, 2}, {2, 64, 1, 64, 6, 2}};
const GemmShape kInvBf16Shapes[] = {{1, 32, 1, 256, 6, 2}, {1, 32, 1, 128, 12, 2}, {1, 32, 1, 64, 16, 2}};
const GemmShape kInvTf32Shapes[] = {{2, 32, 1, 256, 3, 2}, {2, 32, 1, 128, 8, 2}, {2, 32, 1, 64, 12, 2}};
constexpr int kNumShapes = 3;

template <int FMT, int KE, int R, int N, int S, int ABUF>
cudaError_t launch_screen(const CUtensorMap& ta, const CUtensorMap& tb, long long n_units,
                          int n_tiles, int cols, const GemmScratch& g, unsigned* status, int sms,
                          cudaStream_t st) {
    using C = GemmCfg<FMT, KE, R, N, S, ABUF>;
    auto kern = k_gemm_screen<FMT, KE, R, N, S, ABUF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e) return e;
    const long long grid = n_units < sms ? n_units : sms;
    kern<<<(unsigned)grid, GEMM_THREADS, C::SMEM, st>>>(ta, tb, n_units, n_tiles, cols, g, status);
    return cudaGetLastError();
}

cudaError_t dispatch_screen(const GemmShape& sh, const CUtensorMap& ta, const CUtensorMap& tb,
                            long long n_units, int n_tiles, int cols, const GemmScratch& g,
                            unsigned* status, int sms, cudaStream_t st) {
#define SEG_SHAPE(F, KE, R_, N_, S_, AB)                                                     \
    if (sh.fmt == F && sh.ke == KE && sh.R == R_ && sh.N == N_ && sh.S == S_ && sh.ABUF == AB) \
        return launch_screen<F, KE, R_, N_, S_, AB>(ta, tb, n_units, n_tiles, cols, g, status, \
                                                    sms, st);
    SEG_SHAPE(1, 64, 1, 256, 3, 2)
    SEG_SHAPE(1, 64, 1, 128, 6, 2)
    SEG_SHAPE(1, 64, 1, 64, 8, 2)
    SEG_SHAPE(2, 64, 1, 256, 2, 2)
    SEG_SHAPE(2, 64, 1, 128, 4, 2)
    SEG_SHAPE(2, 64, 1, 64, 6, 2)
    SEG_SHAPE(1, 32, 1, 256, 6, 2)
    SEG_SHAPE(1, 32, 1, 128, 12, 2)
    SEG_SHAPE(1, 32, 1, 64, 16, 2)
    SEG_SHAPE(2, 32, 1, 256, 3, 2)
    SEG_SHAPE(2, 32, 1, 128, 8, 2)
    SEG_SHAPE(2, 32, 1, 64, 12, 2)
#undef SEG_SHAPE
    return cudaErrorInvalidValue;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

int gemm_num_configs() { return kNumShapes; }

seg_status prep_gemm_atlas(const AtlasView& at, const int* sp_host, int max_per_bundle,
                           GemmAtlas* g, cudaStream_t st) {
    cudaError_t e;
    // A 32-fiber group inside a bundle keeps most of that bundle's centroids in both
    // orientations: about 2 * max_per_bundle / 32 directional chunks, contiguous in the spatial
    // order; twice that plus slack, and never less than 16 (atlases shaped like the paper's
    // 20-centroid bundles need about 3.4).
    g->rec_per_group = std::max(16, 2 * ((2 * max_per_bundle + 31) / 32) + 8);
    if ((e = cudaMalloc(&g->stats, 5 * sizeof(long long))) ||
        (e = cudaMemsetAsync(g->stats, 0, 5 * sizeof(long long), st)))
        return cuda_fail(e, "gemm stats");
    if ((e = cudaMalloc(&g->sp_s, (size_t)at.M * sizeof(int))) ||
        (e = cudaMalloc(&g->cen_sp, (size_t)at.M * CROW4 * sizeof(float4))) ||
        (e = cudaMalloc(&g->thr2_sp, (size_t)at.M * sizeof(float))) ||
        (e = cudaMalloc(&g->ctr_sp, (size_t)at.M * sizeof(float4))) ||
        (e = cudaMalloc(&g->scr_sp, (size_t)(at.M + 31) / 32 * 32 * sizeof(float4))) ||
        (e = cudaMalloc(&g->end_sp, (size_t)at.M * 3 * sizeof(float4))))
        return cuda_fail(e, "gemm spatial order");
    // the host array lives until the caller synchronizes the stream
    if ((e = cudaMemcpyAsync(g->sp_s, sp_host, (size_t)at.M * sizeof(int), cudaMemcpyHostToDevice,
                             st)))
        return cuda_fail(e, "gemm spatial order");
    k_prep_spatial<<<((at.M + 31) / 32 * 32 + 7) / 8, dim3(32, 8), 0, st>>>(at, g->sp_s, g->cen_sp, g->thr2_sp,
                                                          g->ctr_sp, g->scr_sp, g->end_sp);
    g->cols = 2 * at.M;
    g->cols_pad = (g->cols + COL_ALIGN - 1) / COL_ALIGN * COL_ALIGN;
    if ((e = cudaMalloc(&g->b_bf16, (size_t)g->cols_pad * 64 * 2)) ||
        (e = cudaMalloc(&g->b_tf32, (size_t)g->cols_pad * 64 * 4)))
        return cuda_fail(e, "gemm operands");
    const int threads = 128, blocks = (g->cols_pad + threads - 1) / threads;
    k_prep_b<<<blocks, threads, 0, st>>>(at, g->sp_s, 1, g->cols, g->cols_pad, g->b_bf16);
    k_prep_b<<<blocks, threads, 0, st>>>(at, g->sp_s, 2, g->cols, g->cols_pad, g->b_tf32);
    if ((e = cudaGetLastError())) return cuda_fail(e, "gemm operand prep");
    g->cols_inv = at.M;
    g->cols_inv_pad = (at.M + COL_ALIGN - 1) / COL_ALIGN * COL_ALIGN;
    if ((e = cudaMalloc(&g->bi_bf16, (size_t)g->cols_inv_pad * KE_INV * 2)) ||
        (e = cudaMalloc(&g->bi_tf32, (size_t)g->cols_inv_pad * KE_INV * 4)))
        return cuda_fail(e, "gemm operands");
    const int bi = (g->cols_inv_pad + threads - 1) / threads;
    k_prep_b_inv<<<bi, threads, 0, st>>>(at, g->sp_s, 1, g->cols_inv, g->cols_inv_pad, g->bi_bf16);
    k_prep_b_inv<<<bi, threads, 0, st>>>(at, g->sp_s, 2, g->cols_inv, g->cols_inv_pad, g->bi_tf32);
    if ((e = cudaGetLastError())) return cuda_fail(e, "gemm operand prep");
    // the fused mode's chunk boxes (orientation-free chunks of 32 centroids) and window boxes
    const int nc = g->cols_inv_pad / 32, nw = (nc + 31) / 32;
    if ((e = cudaMalloc(&g->tbox32, (size_t)nc * 2 * sizeof(float4))) ||
        (e = cudaMalloc(&g->wbox32, (size_t)nw * 2 * sizeof(float4))))
        return cuda_fail(e, "gemm chunk boxes");
    k_tile_box<<<(nc + 127) / 128, 128, 0, st>>>(g->ctr_sp, at.M, 32, nc, g->tbox32);
    k_window_box<<<(nw + 127) / 128, 128, 0, st>>>(g->tbox32, nc, nw, g->wbox32);
    if ((e = cudaGetLastError())) return cuda_fail(e, "gemm chunk boxes");
    return SEG_OK;
}

void free_gemm_atlas(GemmAtlas* g) {
    cudaFree(g->b_bf16);
    cudaFree(g->b_tf32);
    cudaFree(g->bi_bf16);
    cudaFree(g->bi_tf32);
    cudaFree(g->sp_s);
    cudaFree(g->cen_sp);
    cudaFree(g->thr2_sp);
    cudaFree(g->ctr_sp);
    cudaFree(g->scr_sp);
    cudaFree(g->end_sp);
    cudaFree(g->tbox32);
    cudaFree(g->wbox32);
    cudaFree(g->stats);
    *g = GemmAtlas{};
}

// One GEMM-mode call over n fibers: sizes, the scratch layout and the tensor maps.
struct GemmCall {
    bool culled, fused, tf32, inv;
    GemmShape sh;
    long long n, n_pad, n_units;
    int cols, n_tiles, n_chunks, awords, sms;
    GemmScratch g;
    unsigned *perm, *bin, *hist, *top;
    float4 *ubox, *tbox;
    unsigned long long* amask;
    CUtensorMap ta, tb;
};

// Sizes the call, takes the atlas's scratch (the caller holds the atlas mutex and releases the
// scratch on `st` once the call's work is enqueued) and encodes the tensor maps.
seg_status gemm_setup(const AtlasView& at, GemmAtlas* ga, ScratchArena* scratch, long long n,
                      int mode, int config, cudaStream_t st, GemmCall* c) {
    c->fused = mode == SEG_MODE_CULLED_FUSED;  // one kernel after the sort, no record list
    c->culled = c->fused || mode == SEG_MODE_PLAIN_CULLED;  // test1 on CUDA cores, no operand
    c->tf32 = mode == SEG_MODE_GEMM_TF32 || mode == SEG_MODE_GEMM_INV_TF32;
    c->inv = c->culled || mode == SEG_MODE_GEMM_INV_BF16 || mode == SEG_MODE_GEMM_INV_TF32;
    const bool culled = c->culled, tf32 = c->tf32, inv = c->inv;
    const int fmt = tf32 ? 2 : 1;
    const int cols = inv ? ga->cols_inv : ga->cols;
    const int cols_pad = inv ? ga->cols_inv_pad : ga->cols_pad;
    const void* bop = inv ? (tf32 ? ga->bi_tf32 : ga->bi_bf16) : (tf32 ? ga->b_tf32 : ga->b_bf16);
    if (config < 0 || config >= kNumShapes) config = 0;
    const GemmShape sh = inv ? (tf32 ? kInvTf32Shapes[config] : kInvBf16Shapes[config])
                             : (tf32 ? kDirTf32Shapes[config] : kDirBf16Shapes[config]);
    const long long rows_per_unit = 128LL * sh.R;
    const long long n_units = (n + rows_per_unit - 1) / rows_per_unit;
    const long long n_pad = n_units * rows_per_unit;
    if (n_pad >= (1LL << 32))
        return fail(SEG_ERR_INVALID_ARG, "seg_label: n=%lld too large for the GEMM modes", n);
    const int n_chunks = cols_pad / 32;
    const int awords = (n_chunks + 63) / 64;
    if (!culled && awords > MAXW)
        return fail(SEG_ERR_UNSUPPORTED,
                    "seg_label: %d operand columns exceed the GEMM modes' limit of %d", cols_pad,
                    32 * 64 * MAXW);
    // block records: about 3.4 per 32 fibers on atlases shaped like the paper's; room for
    // rec_per_group per 32 fibers + slack (fibers past the room are rescanned exactly)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // every warp that writes records reserves SLOT_GRAB slots at a time and may leave up to
    // that many unused: room for that waste comes on top of the records themselves
    const long long writers =
        culled ? std::min<long long>((n_pad / 32 + CS_WARPS - 1) / CS_WARPS, (long long)sms * 8) *
                     CS_WARPS
               : (long long)sms * EPI_WARPS;
    long long cap = n_pad / 32 * ga->rec_per_group + 65536 + writers * SLOT_GRAB;
    if (ga->cap_limit > 0 && ga->cap_limit < cap) cap = ga->cap_limit;
    if (c->fused) cap = 0;  // keys, flags and the sorted rows are not used either
    if (c->fused && at.M >= FZ_MAX_M)
        return fail(SEG_ERR_UNSUPPORTED, "seg_label: %d centroids exceed the fused mode's %d",
                    at.M, FZ_MAX_M);
    const size_t elem = culled ? 0 : tf32 ? 4 : 2;
    const size_t off_alpha = align256((size_t)n_pad * sh.ke * elem);
    // (the fused mode uses the count words, the order, the bins and the chunk boxes only)
    const size_t off_key = off_alpha + align256((size_t)n_pad * 4);
    const size_t off_flag = off_key + align256(c->fused ? 0 : (size_t)n * 8);
    const size_t off_cnt = off_flag + align256(c->fused ? 0 : (size_t)n);
    const size_t off_perm = off_cnt + 256;
    const size_t off_bin = off_perm + align256((size_t)n * 4);
    const size_t off_hist = off_bin + align256((size_t)n * 4);
    const size_t off_top = off_hist + (size_t)NBINS * 4;
    const size_t off_fs = off_top + (size_t)NTOP * 4;
    const size_t off_ubox = off_fs + (c->fused ? 0 : (size_t)n_pad * CROW * 4);
    const size_t off_tbox = off_ubox + align256((size_t)(n_pad / 32) * 32);
    const size_t off_amask = off_tbox + align256((size_t)n_chunks * 32);
    const size_t off_hdr = off_amask + align256((size_t)n_units * awords * 8);
    const size_t off_mask = off_hdr + align256((size_t)cap * 8);
    const size_t bytes = off_mask + (size_t)cap * 128;

    c->sms = sms;
    void* base = nullptr;
    seg_status s = scratch_acquire(scratch, bytes, st, &base);
    if (s != SEG_OK) return s;
    unsigned char* b8 = static_cast<unsigned char*>(base);
    GemmScratch& g = c->g;
    g.a = b8;
    g.alpha = reinterpret_cast<float*>(b8 + off_alpha);
    g.key = reinterpret_cast<unsigned long long*>(b8 + off_key);
    g.flag = b8 + off_flag;
    g.cnt = reinterpret_cast<unsigned long long*>(b8 + off_cnt);
    g.hdr = reinterpret_cast<uint2*>(b8 + off_hdr);
    g.mask = reinterpret_cast<unsigned*>(b8 + off_mask);
    c->perm = reinterpret_cast<unsigned*>(b8 + off_perm);
    c->bin = reinterpret_cast<unsigned*>(b8 + off_bin);
    c->hist = reinterpret_cast<unsigned*>(b8 + off_hist);
    c->top = reinterpret_cast<unsigned*>(b8 + off_top);
    g.perm = c->perm;
    g.fs = reinterpret_cast<float*>(b8 + off_fs);
    c->ubox = reinterpret_cast<float4*>(b8 + off_ubox);
    c->tbox = reinterpret_cast<float4*>(b8 + off_tbox);
    c->amask = reinterpret_cast<unsigned long long*>(b8 + off_amask);
    g.amask = c->amask;
    g.awords = awords;
    g.cen_sp = ga->cen_sp;
    g.end_sp = ga->end_sp;
    g.thr2_sp = ga->thr2_sp;
    g.sp_s = ga->sp_s;
    g.cap = cap;
    g.wait_ns = at.wait_ns;
    c->sh = sh;
    c->n = n;
    c->n_pad = n_pad;
    c->n_units = n_units;
    c->cols = cols;
    c->n_tiles = cols_pad / sh.N;
    c->n_chunks = n_chunks;
    c->awords = awords;
    if (!culled && (!make_tmap(&c->ta, g.a, n_pad, fmt, sh.ke, 128) ||
                    !make_tmap(&c->tb, bop, cols_pad, fmt, sh.ke, sh.N))) {
        scratch_release(scratch, st);
        return fail(SEG_ERR_CUDA, "seg_label: cuTensorMapEncodeTiled failed");
    }
    return SEG_OK;
}

// The call's kernels on `st` (no host synchronisation, no allocation: capturable in a graph).
// dbg_bits: the screen's survivors instead of labels (seg_gemm_screen_bits).
cudaError_t gemm_enqueue(const GemmCall& c, const AtlasView& at, GemmAtlas* ga, FiberSrc src,
                         int* labels, float* dist, int* cidx, unsigned char* orient,
                         cudaStream_t st, Profiler* prof, unsigned* dbg_bits, long long dbg_words) {
    const GemmScratch& g = c.g;
    const long long n = c.n;
    const int sms = c.sms;
    cudaError_t e = cudaMemsetAsync(g.cnt, 0, 256, st);
    if (!e && !c.fused) e = cudaMemsetAsync(g.flag, 0, (size_t)n, st);
    if (!e) {
        ProfScope ps(prof, PROF_GEMM_SORT, st);
        const unsigned nb = (unsigned)((n + 255) / 256);
        e = cudaMemsetAsync(c.hist, 0, (size_t)NBINS * 4, st);
        if (!e) k_bin_count<<<nb, 256, 0, st>>>(src, n, at, c.bin, c.hist);
        if (!e) k_bin_scan<<<NTOP, SCAN_BLOCK, 0, st>>>(c.hist, c.top);
        if (!e) k_bin_scan_top<<<1, 32, 0, st>>>(c.top);
        if (!e) k_bin_scatter<<<nb, 256, 0, st>>>(c.bin, n, c.hist, c.top, c.perm);
        if (!e) e = cudaGetLastError();
    }
    if (!e && c.fused) {
        ProfScope ps(prof, PROF_FUSED, st);
        const long long n_groups = (n + 31) / 32;
        const bool ext = at.cls != CLS_EQ2 || at.multi != nullptr;
        auto kern = ext ? k_fused<true> : k_fused<false>;
        const int smem = FZ_WARPS * (int)sizeof(FzWarp);
        if (smem > 48 * 1024)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e) return e;
        kern<<<(unsigned)std::min<long long>((n_groups + FZ_WARPS - 1) / FZ_WARPS,
                                             (long long)sms * FZ_CTAS),
               FZ_WARPS * 32, FZ_WARPS * sizeof(FzWarp), st>>>(
            src, c.perm, n, n_groups, at, g, ga->scr_sp, ga->tbox32, ga->wbox32, c.n_chunks,
            labels, dist, cidx, orient);
        if (!dbg_bits) k_gemm_stats<<<1, 1, 0, st>>>(g.cnt, n * (long long)c.cols, ga->stats);
        return cudaGetLastError();
    }
    if (!e) {
        ProfScope ps(prof, PROF_GEMM_PREP, st);
        const long long rows_per_block = 32LL * PREP_WARPS;
        const unsigned pb = (unsigned)((c.n_pad + rows_per_block - 1) / rows_per_block);
        auto prep = c.culled ? k_prep_a<0, false>
                    : c.tf32 ? (c.inv ? k_prep_a<2, true> : k_prep_a<2, false>)
                             : (c.inv ? k_prep_a<1, true> : k_prep_a<1, false>);
        prep<<<pb, PREP_WARPS * 32, 0, st>>>(src, c.perm, n, c.n_pad, at, g.a, g.alpha, g.key,
                                             g.fs, c.ubox);
        // centroids per 32-column chunk: 32 (orientation-free) or 16 (directional)
        e = cudaGetLastError();
        if (!e)
            k_tile_box<<<(c.n_chunks + 127) / 128, 128, 0, st>>>(ga->ctr_sp, at.M,
                                                                c.inv ? 32 : 16, c.n_chunks,
                                                                c.tbox);
        if (!e && !c.culled)
            k_block_mask<<<(unsigned)((c.n_units + 3) / 4), 128, 0, st>>>(
                c.ubox, c.tbox, c.n_units, c.sh.R, c.n_chunks, c.awords, c.amask);
        if (!e) e = cudaGetLastError();
    }
    if (!e) {
        ProfScope ps(prof, c.culled ? PROF_CULL_SCREEN : PROF_GEMM_SCREEN, st);
        if (c.culled) {
            const long long n_groups = c.n_pad / 32;
            k_culled_screen<<<(unsigned)std::min<long long>((n_groups + CS_WARPS - 1) / CS_WARPS,
                                                            (long long)sms * 8),
                              CS_WARPS * 32, 0, st>>>(n, n_groups, at, g, ga->scr_sp, c.ubox,
                                                      c.tbox, c.n_chunks);
            e = cudaGetLastError();
        } else {
            e = dispatch_screen(c.sh, c.ta, c.tb, c.n_units, c.n_tiles, c.cols, g, at.status, sms,
                                st);
        }
    }
    if (!e && dbg_bits) {  // diagnostic: the screen's survivors instead of labels
        e = cudaMemsetAsync(dbg_bits, 0, (size_t)n * dbg_words * 4, st);
        if (!e)
            k_survivor_bits<<<sms * 8, 256, 0, st>>>(n, at, g, c.inv ? 1 : 0, dbg_bits, dbg_words,
                                                     n * (long long)c.cols, ga->stats);
        if (!e) e = cudaGetLastError();
        return e;
    }
    if (!e) {
        ProfScope ps(prof, PROF_GEMM_EXACT, st);
        const bool ext = at.cls != CLS_EQ2 || at.multi != nullptr;
        auto kern = c.inv ? (ext ? k_exact_blocks<true, true> : k_exact_blocks<true, false>)
                          : (ext ? k_exact_blocks<false, true> : k_exact_blocks<false, false>);
        kern<<<sms * (c.inv ? 8 : 9), EX_THREADS, 0, st>>>(at, g);
        e = cudaGetLastError();
    }
    if (!e) {
        ProfScope ps(prof, PROF_GEMM_FINAL, st);
        k_overflow_rescan<<<sms * 4, 256, 0, st>>>(n, at, g);
        k_finalize<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            n, at, g, src, labels, dist, cidx, orient, n * (long long)c.cols, ga->stats);
        e = cudaGetLastError();
    }
    return e;
}

seg_status label_gemm(const AtlasView& at, GemmAtlas* ga, ScratchArena* scratch, std::mutex* mu,
                      const float* fib, long long n, int mode, int* labels, float* dist,
                      int* cidx, unsigned char* orient, cudaStream_t st, int config,
                      Profiler* prof, unsigned* dbg_bits, long long dbg_words) {
    std::lock_guard<std::mutex> lock(*mu);
    GemmCall c;
    seg_status s = gemm_setup(at, ga, scratch, n, mode, config, st, &c);
    if (s != SEG_OK) return s;
    const FiberSrc src{fib, nullptr, 0};
    const cudaError_t e = gemm_enqueue(c, at, ga, src, labels, dist, cidx, orient, st, prof,
                                       dbg_bits, dbg_words);
    const seg_status r = scratch_release(scratch, st);
    if (e) return cuda_fail(e, dbg_bits ? "seg_gemm_screen_bits" : "seg_label: GEMM mode");
    return r;
}

// seg_label_batch in the GEMM modes: the subjects are one virtual array of `total` fibers
// (FiberSrc over the device work table), sorted and screened together, and the whole sequence
// of kernels is captured once into a CUDA graph per (mode, tile shape, subject count, total,
// scratch buffer) and replayed. Stream order on `st`: the scratch's previous user, then the
// table upload (from the pinned host table; `copied_event` is recorded after it), then the
// graph. The caller holds the atlas mutex.
seg_status gemm_batch_launch(const AtlasView& at, GemmAtlas* ga, ScratchArena* scratch,
                             BatchState* b, int nsubj, long long total, int mode, int config,
                             const void* host_table, size_t table_bytes, void* copied_event,
                             cudaStream_t st) {
    GemmCall c;
    seg_status s = gemm_setup(at, ga, scratch, total, mode, config, st, &c);
    if (s != SEG_OK) return s;
    cudaError_t e = cudaSuccess;
    if (!b->graph_exec || b->mode != mode || b->config != config || b->nsubj != nsubj ||
        b->total != total || b->scratch_ptr != c.g.a || b->cls != at.cls ||
        b->wait_ns != at.wait_ns) {
        if (b->graph_exec) {
            cudaGraphExecDestroy((cudaGraphExec_t)b->graph_exec);
            b->graph_exec = nullptr;
        }
        cudaStream_t cs = (cudaStream_t)b->cap_stream;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (!e) {
            const FiberSrc src{nullptr, (const BatchEntry*)b->table, nsubj};
            const cudaError_t e1 = gemm_enqueue(c, at, ga, src, nullptr, nullptr, nullptr, nullptr,
                                                cs, nullptr, nullptr, 0);
            e = cudaStreamEndCapture(cs, &graph);
            if (!e) e = e1;
        }
        cudaGraphExec_t exec = nullptr;
        if (!e) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e) {
            scratch_release(scratch, st);
            return cuda_fail(e, "seg_label_batch: capture of the GEMM-mode sequence");
        }
        b->graph_exec = exec;
        b->mode = mode;
        b->config = config;
        b->nsubj = nsubj;
        b->total = total;
        b->scratch_ptr = c.g.a;
        b->cls = at.cls;
        b->wait_ns = at.wait_ns;
    }
    e = cudaMemcpyAsync(b->table, host_table, table_bytes, cudaMemcpyHostToDevice, st);
    if (!e) e = cudaEventRecord((cudaEvent_t)copied_event, st);
    if (!e) e = cudaGraphLaunch((cudaGraphExec_t)b->graph_exec, st);
    const seg_status r = scratch_release(scratch, st);
    if (e) return cuda_fail(e, "seg_label_batch: graph launch");
    return r;
}

}  // namespace seg
