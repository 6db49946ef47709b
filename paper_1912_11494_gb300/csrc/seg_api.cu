// C ABI entry points of libseg (declared in include/seg.h): argument checks, the atlas handle
// and its preparation kernel, dispatch to the labelling kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "seg_internal.cuh"

namespace seg {

thread_local std::string g_last_error;

seg_status fail(seg_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

seg_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? SEG_ERR_OOM : SEG_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

void Profiler::begin(int slot, cudaStream_t st, cudaEvent_t* end_out) {
    if (used == pool.size()) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) || cudaEventCreate(&b)) {
            if (a) cudaEventDestroy(a);
            *end_out = nullptr;
            return;
        }
        pool.emplace_back(a, b);
    }
    cudaEventRecord(pool[used].first, st);
    *end_out = pool[used].second;
    slot_of.push_back(slot);
    ++used;
}

void Profiler::clear() {
    used = 0;
    slot_of.clear();
}

Profiler::~Profiler() {
    for (auto& pr : pool) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
}

namespace {

// float and int32 buffers are read and written as 4-byte words
bool unaligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) != 0; }

// Sorted copy of the atlas: row s of the output is caller centroid perm[s].
__global__ void k_prep_atlas(const float* __restrict__ cen, const int* __restrict__ bundle_of,
                             const float* __restrict__ thr, const int* __restrict__ perm, int M,
                             int M_pad, float c0x, float c0y, float c0z, float* __restrict__ cs,
                             float4* __restrict__ scr, float4* __restrict__ scr2,
                             float* __restrict__ thr2, int* __restrict__ bundle) {
    const int s = blockIdx.x * blockDim.y + threadIdx.y;
    if (s >= M_pad) return;
    if (s >= M) {
        if (threadIdx.x == 0) scr2[s] = make_float4(0.f, 0.f, 0.f, -INFINITY);
        return;
    }
    const int c = perm[s];
    const float* src = cen + (size_t)c * NC;
    float* dst = cs + (size_t)s * CROW;
    for (int k = threadIdx.x; k < NC; k += blockDim.x) dst[k] = src[k];
    if (threadIdx.x == 0) {
        float len = 0.0f;  // the centroid's polyline length (Eq. 3's l_C) in the free slot
        for (int i = 0; i + 1 < NPTS; ++i) {
            const float dx = src[3 * i] - src[3 * i + 3], dy = src[3 * i + 1] - src[3 * i + 4],
                        dz = src[3 * i + 2] - src[3 * i + 5];
            len += sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
        dst[CROW - 1] = len;
        const int b = bundle_of[c];
        const float t = thr[b];
        const float t2 = t * t;
        bundle[s] = b;
        thr2[s] = t2;
        scr[s] = make_float4(src[3 * CENTRE], src[3 * CENTRE + 1], src[3 * CENTRE + 2], t2);
        // test1 in dot-product form (see k_plain.cu); the slack only keeps more pairs
        const float x = src[3 * CENTRE] - c0x, y = src[3 * CENTRE + 1] - c0y,
                    z = src[3 * CENTRE + 2] - c0z;
        const float r2 = fmaf(x, x, fmaf(y, y, z * z));
        scr2[s] = make_float4(x, y, z, 0.5f * (t2 - r2) + 1e-5f * (r2 + t2) + 1e-3f);
    }
}

bool device_is_sm103(int* dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (dev_out) *dev_out = dev;
    return major == 10 && minor == 3;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

}  // namespace
}  // namespace seg

using namespace seg;

namespace {
// An NVTX range around one C ABI call, so profilers show each call and the kernels it launched
// (a no-op unless a tool is attached).
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
};
}  // namespace

struct seg_atlas {
    AtlasView view{};
    int device = 0;
    float* cen = nullptr;
    float4* scr = nullptr;
    float4* scr2 = nullptr;
    float* thr2 = nullptr;
    int* bundle = nullptr;
    int* perm = nullptr;
    int* inv_perm = nullptr;
    unsigned* status = nullptr;
    GemmAtlas gemm{};
    ScratchArena scratch{};
    ScratchArena rs_scratch{};  // seg_label_streamlines: the resampled fibers (guarded by rs_mu)
    std::mutex rs_mu;
    ScratchArena ref_scratch{};  // seg_refine_affine's buffers (guarded by ref_mu)
    std::mutex ref_mu;
    float max_thr = 0.0f;        // the largest bundle threshold
    // seg_label_host: two device copies of the caller's host buffers, used by alternate calls
    // (so that a call's upload overlaps the previous call's labelling), an internal copy
    // stream, one event per chunk and one per buffer marking its last use (guarded by
    // host_mu)
    void* hbuf[2] = {nullptr, nullptr};
    size_t hbuf_bytes[2] = {0, 0};
    int hnext = 0;
    cudaStream_t hcopy = nullptr;
    cudaEvent_t hev[SEG_HOST_CHUNKS + 2] = {};
    std::mutex host_mu;
    BatchState batch{};
    int config[7] = {0, 0, 0, 0, 0, 0, 0};  // tile-shape selection per seg_mode
    Profiler prof;
    std::mutex mu;  // guards scratch growth and the batch graph cache
};

extern "C" {

const char* seg_status_string(seg_status s) {
    switch (s) {
        case SEG_OK: return "SEG_OK";
        case SEG_ERR_INVALID_ARG: return "SEG_ERR_INVALID_ARG";
        case SEG_ERR_CUDA: return "SEG_ERR_CUDA";
        case SEG_ERR_OOM: return "SEG_ERR_OOM";
        case SEG_ERR_UNSUPPORTED: return "SEG_ERR_UNSUPPORTED";
        case SEG_ERR_TIMEOUT: return "SEG_ERR_TIMEOUT";
        case SEG_ERR_OVERFLOW: return "SEG_ERR_OVERFLOW";
    }
    return "SEG_ERR_UNKNOWN";
}

const char* seg_last_error(void) { return g_last_error.c_str(); }

static void free_atlas(seg_atlas* a) {
    if (!a) return;
    cudaFree(a->cen);
    cudaFree(a->scr);
    cudaFree(a->scr2);
    cudaFree(a->thr2);
    cudaFree(a->bundle);
    cudaFree(a->perm);
    cudaFree(a->inv_perm);
    cudaFree(a->status);
    free_gemm_atlas(&a->gemm);
    free_scratch(&a->scratch);
    free_scratch(&a->rs_scratch);
    free_scratch(&a->ref_scratch);
    if (a->hcopy) cudaStreamSynchronize(a->hcopy);
    for (cudaEvent_t ev : a->hev)
        if (ev) cudaEventDestroy(ev);
    if (a->hcopy) cudaStreamDestroy(a->hcopy);
    cudaFree(a->hbuf[0]);
    cudaFree(a->hbuf[1]);
    free_batch(&a->batch);
    delete a;
}

seg_status seg_create_atlas(const float* d_centroids, const int32_t* d_bundle_of,
                            const float* d_thresholds, int32_t M, int32_t B, int32_t npts,
                            void* stream, seg_atlas** out) {
    const CallRange range("seg_create_atlas");
    g_last_error.clear();
    if (!out) return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: out is NULL");
    *out = nullptr;
    if (!d_centroids || !d_bundle_of || !d_thresholds)
        return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: NULL input buffer");
    if (M < 1 || B < 1) return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: M=%d B=%d", M, B);
    if (M > (1 << 28)) return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: M=%d too large", M);
    if (npts != SEG_NPTS)
        return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: npts=%d, must be %d", npts, SEG_NPTS);
    int dev = 0;
    if (!device_is_sm103(&dev))
        return fail(SEG_ERR_UNSUPPORTED, "seg_create_atlas: device is not compute capability 10.3");
    cudaStream_t st = (cudaStream_t)stream;

    std::vector<int32_t> hb(M);
    std::vector<float> ht(B);
    std::vector<float> hc((size_t)M * NC);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(hb.data(), d_bundle_of, M * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(ht.data(), d_thresholds, B * sizeof(float), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(hc.data(), d_centroids, hc.size() * sizeof(float), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "seg_create_atlas: reading the atlas");
    for (int b = 0; b < B; ++b)
        if (!(std::isfinite(ht[b]) && ht[b] > 0.0f))
            return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: threshold[%d]=%g must be finite and > 0", b, (double)ht[b]);
    for (size_t k = 0; k < hc.size(); ++k)
        if (!std::isfinite(hc[k]))
            return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: centroid %zu has a non-finite coordinate", k / NC);
    // Stable counting sort by bundle: the visiting order of Algorithm 1.
    std::vector<int32_t> cnt(B + 1, 0), perm(M);
    for (int c = 0; c < M; ++c) {
        if (hb[c] < 0 || hb[c] >= B)
            return fail(SEG_ERR_INVALID_ARG, "seg_create_atlas: bundle_of[%d]=%d outside [0,%d)", c, hb[c], B);
        cnt[hb[c] + 1]++;
    }
    for (int b = 0; b < B; ++b) cnt[b + 1] += cnt[b];
    for (int c = 0; c < M; ++c) perm[cnt[hb[c]]++] = c;
    std::vector<int32_t> inv(M);
    for (int sp = 0; sp < M; ++sp) inv[perm[sp]] = sp;
    const int M_pad = (M + MPAD - 1) / MPAD * MPAD;
    double c0[3] = {0.0, 0.0, 0.0};  // centring offset: mean centroid centre point
    for (int c = 0; c < M; ++c)
        for (int r = 0; r < 3; ++r) c0[r] += hc[(size_t)c * NC + 3 * CENTRE + r];
    for (int r = 0; r < 3; ++r) c0[r] = std::round(c0[r] / M);
    // Spatial order of the sorted centroids for the tensor-core prune: the Hilbert-curve
    // position of the centre point's cell (the grid the GEMM modes also sort fibers on), so
    // that a tile of consecutive columns covers a compact region. sp[c] = sorted index at
    // spatial position c.
    std::vector<int32_t> sp(M);
    {
        std::vector<std::pair<uint32_t, int32_t>> key(M);
        for (int s = 0; s < M; ++s) {
            uint32_t cell[3];
            for (int r = 0; r < 3; ++r) {
                const double v = hc[(size_t)perm[s] * NC + 3 * CENTRE + r];
                const double t = std::floor((v - c0[r]) / LOC_CELL_MM) + (1 << (LOC_BITS - 1));
                const double top = (1 << LOC_BITS) - 1;
                cell[r] = t >= 0.0 ? (uint32_t)(t < top ? t : top) : 0u;  // NaN -> 0
            }
            key[s] = {hilbert_index3(cell[0], cell[1], cell[2]), s};
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const auto& x, const auto& y) { return x.first < y.first; });
        for (int c = 0; c < M; ++c) sp[c] = key[c].second;
    }

    seg_atlas* a = new seg_atlas();
    a->device = dev;
    for (int b = 0; b < B; ++b) a->max_thr = std::max(a->max_thr, ht[b]);
    if ((e = dalloc(&a->cen, (size_t)M * CROW)) || (e = dalloc(&a->scr, M)) || (e = dalloc(&a->scr2, M_pad)) ||
        (e = dalloc(&a->thr2, M)) || (e = dalloc(&a->bundle, M)) || (e = dalloc(&a->perm, M)) ||
        (e = dalloc(&a->inv_perm, M)) || (e = dalloc(&a->status, 4))) {
        free_atlas(a);
        return cuda_fail(e, "seg_create_atlas: allocation");
    }
    if ((e = cudaMemcpyAsync(a->perm, perm.data(), M * sizeof(int32_t), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(a->inv_perm, inv.data(), M * sizeof(int32_t), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemsetAsync(a->status, 0, 4 * sizeof(unsigned), st))) {
        free_atlas(a);
        return cuda_fail(e, "seg_create_atlas: upload");
    }
    dim3 blk(32, 8);
    k_prep_atlas<<<(M_pad + 7) / 8, blk, 0, st>>>(d_centroids, d_bundle_of, d_thresholds,
                                                  a->perm, M, M_pad, (float)c0[0], (float)c0[1],
                                                  (float)c0[2], a->cen, a->scr, a->scr2, a->thr2,
                                                  a->bundle);
    if ((e = cudaGetLastError())) {
        free_atlas(a);
        return cuda_fail(e, "seg_create_atlas: prep kernel");
    }
    a->view.M = M;
    a->view.B = B;
    a->view.M_pad = M_pad;
    a->view.c0x = (float)c0[0];
    a->view.c0y = (float)c0[1];
    a->view.c0z = (float)c0[2];
    a->view.scr2 = a->scr2;
    a->view.cen = a->cen;
    a->view.scr = a->scr;
    a->view.thr2 = a->thr2;
    a->view.bundle = a->bundle;
    a->view.perm = a->perm;
    a->view.status = a->status;
    a->view.wait_ns = 2000000000ull;
    int max_per_bundle = 0;  // (cnt[b] now ends bundle b: the sort advanced it)
    for (int b = 0; b < B; ++b)
        max_per_bundle = std::max(max_per_bundle, cnt[b] - (b ? cnt[b - 1] : 0));
    seg_status s = prep_gemm_atlas(a->view, sp.data(), max_per_bundle, &a->gemm, st);
    if (s != SEG_OK) {
        free_atlas(a);
        return s;
    }
    if ((e = cudaStreamSynchronize(st))) {
        free_atlas(a);
        return cuda_fail(e, "seg_create_atlas: synchronize");
    }
    *out = a;
    return SEG_OK;
}

seg_status seg_destroy_atlas(seg_atlas* atlas) {
    const CallRange range("seg_destroy_atlas");
    g_last_error.clear();
    if (!atlas) return SEG_OK;
    cudaDeviceSynchronize();
    free_atlas(atlas);
    return SEG_OK;
}

seg_status seg_atlas_info(const seg_atlas* atlas, int32_t* M, int32_t* B) {
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_atlas_info: atlas is NULL");
    if (M) *M = atlas->view.M;
    if (B) *B = atlas->view.B;
    return SEG_OK;
}

seg_status seg_label(const seg_atlas* atlas, const float* d_fibers, int64_t n, seg_mode mode,
                     int32_t* d_labels, float* d_dist, int32_t* d_cidx, uint8_t* d_orient,
                     void* stream) {
    const CallRange range("seg_label");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_label: atlas is NULL");
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_label: n=%lld < 0", (long long)n);
    if (n > 0 && (!d_fibers || !d_labels))
        return fail(SEG_ERR_INVALID_ARG, "seg_label: NULL fibers or labels");
    if (unaligned4(d_fibers) || unaligned4(d_labels) || unaligned4(d_dist) || unaligned4(d_cidx))
        return fail(SEG_ERR_INVALID_ARG, "seg_label: a buffer is not 4-byte aligned");
    if ((int)mode < SEG_MODE_PLAIN || (int)mode > SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_INVALID_ARG, "seg_label: unknown mode %d", (int)mode);
    if (n == 0) return SEG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    if (mode == SEG_MODE_PLAIN) {
        ProfScope ps(&a->prof, PROF_PLAIN, st);
        cudaError_t e = launch_label_plain(atlas->view, d_fibers, n, d_labels, d_dist, d_cidx,
                                           d_orient, st, atlas->config[0]);
        return e ? cuda_fail(e, "seg_label: plain kernel") : SEG_OK;
    }
    return label_gemm(a->view, &a->gemm, &a->scratch, &a->mu, d_fibers, n, (int)mode, d_labels,
                      d_dist, d_cidx, d_orient, st, a->config[(int)mode], &a->prof);
}

seg_status seg_label_multi(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                           seg_mode mode, uint32_t* d_bundle_bits, int64_t words_per_fiber,
                           int32_t* d_labels, float* d_dist, void* stream) {
    const CallRange range("seg_label_multi");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_label_multi: atlas is NULL");
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_label_multi: n=%lld < 0", (long long)n);
    if ((int)mode < SEG_MODE_PLAIN || (int)mode > SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_multi: unknown mode %d", (int)mode);
    const int64_t need = ((int64_t)atlas->view.B + 31) / 32;
    if (words_per_fiber < need)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_multi: words_per_fiber=%lld < %lld",
                    (long long)words_per_fiber, (long long)need);
    if (n == 0) return SEG_OK;
    if (!d_fibers || !d_bundle_bits || !d_labels)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_multi: NULL fibers, bits or labels");
    if (unaligned4(d_fibers) || unaligned4(d_bundle_bits) || unaligned4(d_labels) ||
        unaligned4(d_dist))
        return fail(SEG_ERR_INVALID_ARG, "seg_label_multi: a buffer is not 4-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_bundle_bits, 0, (size_t)n * words_per_fiber * 4, st);
    if (e) return cuda_fail(e, "seg_label_multi: clearing the bundle bits");
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    AtlasView view = atlas->view;  // this call's copy, with the multi-label output
    view.multi = d_bundle_bits;
    view.multi_words = words_per_fiber;
    if (mode == SEG_MODE_PLAIN) {
        ProfScope ps(&a->prof, PROF_PLAIN, st);
        e = launch_label_plain(view, d_fibers, n, d_labels, d_dist, nullptr, nullptr, st,
                               atlas->config[0]);
        return e ? cuda_fail(e, "seg_label_multi: plain kernel") : SEG_OK;
    }
    return label_gemm(view, &a->gemm, &a->scratch, &a->mu, d_fibers, n, (int)mode, d_labels,
                      d_dist, nullptr, nullptr, st, a->config[(int)mode], &a->prof);
}

seg_status seg_label_host(const seg_atlas* atlas, const float* h_fibers, int64_t n,
                          seg_mode mode, int32_t* h_labels, float* h_dist, void* stream) {
    const CallRange range("seg_label_host");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_label_host: atlas is NULL");
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_label_host: n=%lld < 0", (long long)n);
    if (n > 0 && (!h_fibers || !h_labels))
        return fail(SEG_ERR_INVALID_ARG, "seg_label_host: NULL fibers or labels");
    if ((int)mode < SEG_MODE_PLAIN || (int)mode > SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_host: unknown mode %d", (int)mode);
    if (n == 0) return SEG_OK;
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(a->host_mu);
    cudaError_t e;
    if (!a->hcopy) {
        if ((e = cudaStreamCreateWithFlags(&a->hcopy, cudaStreamNonBlocking)))
            return cuda_fail(e, "seg_label_host: stream");
        for (cudaEvent_t& ev : a->hev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)))
                return cuda_fail(e, "seg_label_host: event");
    }
    const int bi = a->hnext;
    a->hnext ^= 1;
    cudaEvent_t ev_done = a->hev[SEG_HOST_CHUNKS + bi];
    const size_t fb = ((size_t)n * NC * 4 + 255) / 256 * 256, lb = ((size_t)n * 4 + 255) / 256 * 256;
    const size_t need = fb + 2 * lb;
    if (need > a->hbuf_bytes[bi]) {
        // the call before the previous one may still use the old buffer
        if ((e = cudaEventSynchronize(ev_done)) || (e = cudaFree(a->hbuf[bi])))
            return cuda_fail(e, "seg_label_host: buffer");
        a->hbuf[bi] = nullptr;
        a->hbuf_bytes[bi] = 0;
        if ((e = cudaMalloc(&a->hbuf[bi], need))) return cuda_fail(e, "seg_label_host: buffer");
        a->hbuf_bytes[bi] = need;
    }
    float* d_fib = static_cast<float*>(a->hbuf[bi]);
    int32_t* d_lab = reinterpret_cast<int32_t*>(static_cast<char*>(a->hbuf[bi]) + fb);
    float* d_dst = reinterpret_cast<float*>(static_cast<char*>(a->hbuf[bi]) + fb + lb);
    // the upload starts as soon as this buffer's previous use (two calls ago) has finished,
    // which lets it overlap the previous call's labelling
    if ((e = cudaStreamWaitEvent(a->hcopy, ev_done, 0)))
        return cuda_fail(e, "seg_label_host: ordering");
    const int chunks = n >= (1 << 21) ? SEG_HOST_CHUNKS : n >= (1 << 19) ? 2 : 1;
    const int64_t per = (n + chunks - 1) / chunks;
    for (int c = 0; c < chunks; ++c) {
        const int64_t off = c * per, len = std::min<int64_t>(per, n - off);
        if (len <= 0) break;
        if ((e = cudaMemcpyAsync(d_fib + off * NC, h_fibers + off * NC, (size_t)len * NC * 4,
                                 cudaMemcpyHostToDevice, a->hcopy)) ||
            (e = cudaEventRecord(a->hev[c], a->hcopy)) ||
            (e = cudaStreamWaitEvent(st, a->hev[c], 0)))
            return cuda_fail(e, "seg_label_host: upload");
        seg_status s = seg_label(atlas, d_fib + off * NC, len, mode, d_lab + off,
                                 h_dist ? d_dst + off : nullptr, nullptr, nullptr, stream);
        if (s != SEG_OK) return s;
        if ((e = cudaMemcpyAsync(h_labels + off, d_lab + off, (size_t)len * 4,
                                 cudaMemcpyDeviceToHost, st)) ||
            (h_dist && (e = cudaMemcpyAsync(h_dist + off, d_dst + off, (size_t)len * 4,
                                            cudaMemcpyDeviceToHost, st))))
            return cuda_fail(e, "seg_label_host: download");
    }
    if ((e = cudaEventRecord(ev_done, st))) return cuda_fail(e, "seg_label_host: event");
    return SEG_OK;
}

seg_status seg_resample(const float* d_points, const int64_t* d_offsets, int64_t n, float* d_out,
                        void* stream) {
    const CallRange range("seg_resample");
    g_last_error.clear();
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_resample: n=%lld < 0", (long long)n);
    if (n == 0) return SEG_OK;
    if (!d_offsets || !d_out)
        return fail(SEG_ERR_INVALID_ARG, "seg_resample: NULL offsets or output");
    if (unaligned4(d_points) || unaligned4(d_out) ||
        (reinterpret_cast<uintptr_t>(d_offsets) & 7u))
        return fail(SEG_ERR_INVALID_ARG, "seg_resample: a buffer is not aligned");
    return resample_launch(d_points, reinterpret_cast<const long long*>(d_offsets), n, d_out,
                           (cudaStream_t)stream);
}

seg_status seg_label_streamlines(const seg_atlas* atlas, const float* d_points,
                                 const int64_t* d_offsets, int64_t n, seg_mode mode,
                                 int32_t* d_labels, float* d_dist, int32_t* d_cidx,
                                 uint8_t* d_orient, void* stream) {
    const CallRange range("seg_label_streamlines");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_label_streamlines: atlas is NULL");
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_label_streamlines: n < 0");
    if ((int)mode < SEG_MODE_PLAIN || (int)mode > SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_streamlines: unknown mode %d", (int)mode);
    if (n == 0) return SEG_OK;
    if (!d_offsets || !d_labels)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_streamlines: NULL offsets or labels");
    if (unaligned4(d_points) || unaligned4(d_labels) || unaligned4(d_dist) ||
        unaligned4(d_cidx) || (reinterpret_cast<uintptr_t>(d_offsets) & 7u))
        return fail(SEG_ERR_INVALID_ARG, "seg_label_streamlines: a buffer is not aligned");
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lock(a->rs_mu);  // one user of rs_scratch at a time
    void* buf = nullptr;
    seg_status s = scratch_acquire(&a->rs_scratch, (size_t)n * NC * sizeof(float), st, &buf);
    if (s != SEG_OK) return s;
    float* fib = static_cast<float*>(buf);
    s = resample_launch(d_points, reinterpret_cast<const long long*>(d_offsets), n, fib, st);
    if (s == SEG_OK)
        s = seg_label(atlas, fib, n, mode, d_labels, d_dist, d_cidx, d_orient, stream);
    const seg_status r = scratch_release(&a->rs_scratch, st);
    return s != SEG_OK ? s : r;
}

seg_status seg_label_batch(const seg_atlas* atlas, int32_t nsubj, const float* const* h_fibers,
                           const int64_t* h_counts, seg_mode mode, int32_t* const* h_labels,
                           float* const* h_dist, void* stream) {
    const CallRange range("seg_label_batch");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_label_batch: atlas is NULL");
    if (nsubj < 0) return fail(SEG_ERR_INVALID_ARG, "seg_label_batch: nsubj=%d < 0", nsubj);
    if (nsubj == 0) return SEG_OK;
    if (!h_fibers || !h_counts || !h_labels)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_batch: NULL pointer array");
    if ((int)mode < SEG_MODE_PLAIN || (int)mode > SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_INVALID_ARG, "seg_label_batch: unknown mode %d", (int)mode);
    for (int s = 0; s < nsubj; ++s) {
        if (h_counts[s] < 0)
            return fail(SEG_ERR_INVALID_ARG, "seg_label_batch: count[%d] < 0", s);
        if (h_counts[s] > 0 && (!h_fibers[s] || !h_labels[s]))
            return fail(SEG_ERR_INVALID_ARG, "seg_label_batch: NULL buffer for subject %d", s);
        if (unaligned4(h_fibers[s]) || unaligned4(h_labels[s]) ||
            (h_dist && unaligned4(h_dist[s])))
            return fail(SEG_ERR_INVALID_ARG,
                        "seg_label_batch: a buffer of subject %d is not 4-byte aligned", s);
    }
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    ProfScope ps(&a->prof, PROF_BATCH, (cudaStream_t)stream);
    return batch_launch(a->view, &a->gemm, &a->batch, &a->scratch, &a->mu, nsubj, h_fibers,
                        reinterpret_cast<const long long*>(h_counts), (int)mode, h_labels,
                        h_dist, (cudaStream_t)stream, a->config[(int)mode]);
}

seg_status seg_apply_affine(const float* d_in, int64_t n, const double* h_affine12, float* d_out,
                            void* stream) {
    const CallRange range("seg_apply_affine");
    g_last_error.clear();
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_apply_affine: n < 0");
    if (!h_affine12) return fail(SEG_ERR_INVALID_ARG, "seg_apply_affine: NULL affine");
    if (n == 0) return SEG_OK;
    if (!d_in || !d_out) return fail(SEG_ERR_INVALID_ARG, "seg_apply_affine: NULL buffer");
    if (unaligned4(d_in) || unaligned4(d_out))
        return fail(SEG_ERR_INVALID_ARG, "seg_apply_affine: buffer not 4-byte aligned");
    return apply_affine_launch(d_in, n, h_affine12, d_out, (cudaStream_t)stream);
}

seg_status seg_grad(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                    const double* h_affine12, const int32_t* d_cidx, const uint8_t* d_orient,
                    double* d_grad_affine12, float* d_grad_centroids, double* d_cost,
                    void* stream) {
    const CallRange range("seg_grad");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_grad: atlas is NULL");
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_grad: n < 0");
    if (!h_affine12 || !d_grad_affine12)
        return fail(SEG_ERR_INVALID_ARG, "seg_grad: NULL affine or gradient buffer");
    if (n > 0 && (!d_fibers || !d_cidx || !d_orient))
        return fail(SEG_ERR_INVALID_ARG, "seg_grad: NULL fibers, cidx or orient");
    if (unaligned4(d_fibers) || unaligned4(d_cidx))
        return fail(SEG_ERR_INVALID_ARG, "seg_grad: fibers or cidx not 4-byte aligned");
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    ProfScope ps(&a->prof, PROF_GRAD, (cudaStream_t)stream);
    return grad_launch(a->view, a->inv_perm, &a->scratch, &a->mu, d_fibers, n, h_affine12,
                       d_cidx, d_orient, d_grad_affine12, d_grad_centroids, d_cost,
                       (cudaStream_t)stream);
}

int32_t seg_num_configs(seg_mode mode) {
    switch (mode) {
        case SEG_MODE_PLAIN: return kNumPlainConfigs;
        case SEG_MODE_GEMM_BF16:
        case SEG_MODE_GEMM_TF32:
        case SEG_MODE_GEMM_INV_BF16:
        case SEG_MODE_GEMM_INV_TF32: return gemm_num_configs();
        case SEG_MODE_PLAIN_CULLED:
        case SEG_MODE_CULLED_FUSED: return 1;
    }
    return 0;
}

seg_status seg_set_config(seg_atlas* atlas, seg_mode mode, int32_t config) {
    const CallRange range("seg_set_config");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_set_config: atlas is NULL");
    const int nc = seg_num_configs(mode);
    if (nc <= 0) return fail(SEG_ERR_INVALID_ARG, "seg_set_config: unknown mode %d", (int)mode);
    if (config < 0 || config >= nc)
        return fail(SEG_ERR_INVALID_ARG, "seg_set_config: config %d outside [0,%d)", config, nc);
    atlas->config[(int)mode] = config;
    return SEG_OK;
}

seg_status seg_set_classification(seg_atlas* atlas, seg_classification cls) {
    const CallRange range("seg_set_classification");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_set_classification: atlas is NULL");
    if ((int)cls < SEG_CLASS_EQ2 || (int)cls > SEG_CLASS_PAPER)
        return fail(SEG_ERR_INVALID_ARG, "seg_set_classification: unknown classification %d",
                    (int)cls);
    std::lock_guard<std::mutex> lock(atlas->mu);
    atlas->view.cls = (int)cls;
    return SEG_OK;
}

seg_status seg_set_wait_limit(seg_atlas* atlas, uint64_t ns) {
    const CallRange range("seg_set_wait_limit");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_set_wait_limit: atlas is NULL");
    std::lock_guard<std::mutex> lock(atlas->mu);
    atlas->view.wait_ns = ns;
    return SEG_OK;
}

seg_status seg_set_scratch_limit(seg_atlas* atlas, int64_t bytes) {
    const CallRange range("seg_set_scratch_limit");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_set_scratch_limit: atlas is NULL");
    if (bytes < 0) return fail(SEG_ERR_INVALID_ARG, "seg_set_scratch_limit: bytes < 0");
    std::lock_guard<std::mutex> lock(atlas->mu);
    for (ScratchArena* sa : {&atlas->scratch, &atlas->rs_scratch, &atlas->ref_scratch})
        sa->limit = (size_t)bytes;
    return SEG_OK;
}

seg_status seg_get_classification(const seg_atlas* atlas, seg_classification* cls) {
    const CallRange range("seg_get_classification");
    g_last_error.clear();
    if (!atlas || !cls) return fail(SEG_ERR_INVALID_ARG, "seg_get_classification: NULL argument");
    *cls = (seg_classification)atlas->view.cls;
    return SEG_OK;
}

seg_status seg_get_config(const seg_atlas* atlas, seg_mode mode, int32_t* config) {
    const CallRange range("seg_get_config");
    g_last_error.clear();
    if (!atlas || !config) return fail(SEG_ERR_INVALID_ARG, "seg_get_config: NULL argument");
    if (seg_num_configs(mode) <= 0)
        return fail(SEG_ERR_INVALID_ARG, "seg_get_config: unknown mode %d", (int)mode);
    *config = atlas->config[(int)mode];
    return SEG_OK;
}

seg_status seg_refine_affine(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                             seg_mode mode, double* h_affine12, int32_t iters, double step_mm,
                             double* h_cost, int32_t* h_iters_done, void* stream) {
    const CallRange range("seg_refine_affine");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_refine_affine: atlas is NULL");
    if (n <= 0 || !d_fibers || !h_affine12)
        return fail(SEG_ERR_INVALID_ARG, "seg_refine_affine: no fibers or NULL affine");
    if ((int)mode < SEG_MODE_PLAIN || (int)mode > SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_INVALID_ARG, "seg_refine_affine: unknown mode %d", (int)mode);
    if (iters < 0 || !(step_mm > 0.0) || !std::isfinite(step_mm))
        return fail(SEG_ERR_INVALID_ARG, "seg_refine_affine: iters=%d step=%g", iters, step_mm);
    for (int k = 0; k < 12; ++k)
        if (!std::isfinite(h_affine12[k]))
            return fail(SEG_ERR_INVALID_ARG, "seg_refine_affine: non-finite affine");
    if (unaligned4(d_fibers))
        return fail(SEG_ERR_INVALID_ARG, "seg_refine_affine: fibers not 4-byte aligned");
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    int done = 0;
    const seg_status s = refine_launch(atlas, atlas->view, &a->ref_scratch, &a->ref_mu, d_fibers,
                                       n, (int)mode, h_affine12, iters, step_mm,
                                       (double)atlas->max_thr, h_cost, &done,
                                       (cudaStream_t)stream);
    if (h_iters_done) *h_iters_done = done;
    return s;
}

seg_status seg_grad_noalloc(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                            const double* h_affine12, const int32_t* d_cidx,
                            const uint8_t* d_orient, double* d_grad_affine12,
                            float* d_grad_centroids, double* d_cost, void* stream) {
    const CallRange range("seg_grad_noalloc");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_grad_noalloc: atlas is NULL");
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_grad_noalloc: n < 0");
    if (!h_affine12 || !d_grad_affine12)
        return fail(SEG_ERR_INVALID_ARG, "seg_grad_noalloc: NULL affine or gradient buffer");
    if (n > 0 && (!d_fibers || !d_cidx || !d_orient))
        return fail(SEG_ERR_INVALID_ARG, "seg_grad_noalloc: NULL fibers, cidx or orient");
    if (unaligned4(d_fibers) || unaligned4(d_cidx))
        return fail(SEG_ERR_INVALID_ARG, "seg_grad_noalloc: fibers or cidx not 4-byte aligned");
    return grad_noalloc_launch(atlas->view, atlas->inv_perm, d_fibers, n, h_affine12, d_cidx,
                               d_orient, d_grad_affine12, d_grad_centroids, d_cost,
                               (cudaStream_t)stream);
}

seg_status seg_gemm_screen_bits(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                                seg_mode mode, uint32_t* d_bits, int64_t words_per_fiber,
                                void* stream) {
    const CallRange range("seg_gemm_screen_bits");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_gemm_screen_bits: atlas is NULL");
    if (n < 0) return fail(SEG_ERR_INVALID_ARG, "seg_gemm_screen_bits: n < 0");
    if ((int)mode < SEG_MODE_GEMM_BF16 || (int)mode > SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_INVALID_ARG, "seg_gemm_screen_bits: mode %d has no screen",
                    (int)mode);
    if (mode == SEG_MODE_CULLED_FUSED)
        return fail(SEG_ERR_UNSUPPORTED, "seg_gemm_screen_bits: mode %d has no separate screen",
                    (int)mode);
    const bool inv = mode == SEG_MODE_GEMM_INV_BF16 || mode == SEG_MODE_GEMM_INV_TF32 ||
                     mode == SEG_MODE_PLAIN_CULLED;
    const int64_t need = ((inv ? 1 : 2) * (int64_t)atlas->view.M + 31) / 32;
    if (words_per_fiber < need)
        return fail(SEG_ERR_INVALID_ARG,
                    "seg_gemm_screen_bits: words_per_fiber=%lld < %lld", (long long)words_per_fiber,
                    (long long)need);
    if (n > 0 && (!d_fibers || !d_bits))
        return fail(SEG_ERR_INVALID_ARG, "seg_gemm_screen_bits: NULL fibers or bits");
    if (unaligned4(d_fibers) || unaligned4(d_bits))
        return fail(SEG_ERR_INVALID_ARG, "seg_gemm_screen_bits: a buffer is not 4-byte aligned");
    if (n == 0) return SEG_OK;
    seg_atlas* a = const_cast<seg_atlas*>(atlas);
    return label_gemm(a->view, &a->gemm, &a->scratch, &a->mu, d_fibers, n, (int)mode, nullptr,
                      nullptr, nullptr, nullptr, (cudaStream_t)stream, a->config[(int)mode],
                      nullptr, d_bits, words_per_fiber);
}

seg_status seg_profile_enable(seg_atlas* atlas, int32_t enable) {
    const CallRange range("seg_profile_enable");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_profile_enable: atlas is NULL");
    std::lock_guard<std::mutex> lock(atlas->mu);
    cudaError_t e = cudaDeviceSynchronize();
    if (e) return cuda_fail(e, "seg_profile_enable");
    atlas->prof.clear();
    atlas->prof.enabled = enable != 0;
    return SEG_OK;
}

seg_status seg_profile_read(seg_atlas* atlas, const char* kernel, int64_t* launches,
                            double* total_ms) {
    const CallRange range("seg_profile_read");
    g_last_error.clear();
    if (!atlas || !kernel) return fail(SEG_ERR_INVALID_ARG, "seg_profile_read: NULL argument");
    static const char* names[PROF_SLOTS] = {"plain",         "batch", "gemm_prep",
                                            "gemm_screen",   "gemm_exact", "gemm_finalize",
                                            "grad",          "gemm_sort", "cull_screen",
                                            "culled_fused"};
    int slot = -1;
    for (int k = 0; k < PROF_SLOTS; ++k)
        if (strcmp(kernel, names[k]) == 0) slot = k;
    if (slot < 0) return fail(SEG_ERR_INVALID_ARG, "seg_profile_read: unknown kernel '%s'", kernel);
    long long cnt = 0;
    double ms = 0.0;
    Profiler& p = atlas->prof;
    for (size_t i = 0; i < p.used; ++i) {
        if (p.slot_of[i] != slot) continue;
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(p.pool[i].second);
        if (!e) e = cudaEventElapsedTime(&t, p.pool[i].first, p.pool[i].second);
        if (e) return cuda_fail(e, "seg_profile_read");
        ++cnt;
        ms += t;
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = ms;
    return SEG_OK;
}

seg_status seg_sync_status(const seg_atlas* atlas, void* stream) {
    const CallRange range("seg_sync_status");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_sync_status: atlas is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(st)) ||
        (e = cudaMemcpy(&h, atlas->status, sizeof(unsigned), cudaMemcpyDeviceToHost)) ||
        (e = cudaMemset(atlas->status, 0, sizeof(unsigned))))
        return cuda_fail(e, "seg_sync_status");
    if (h & ST_TIMEOUT) return fail(SEG_ERR_TIMEOUT, "a bounded device wait timed out");
    if (h & ST_OVERFLOW) return fail(SEG_ERR_OVERFLOW, "a device list overflowed");
    return SEG_OK;
}

seg_status seg_set_gemm_record_cap(seg_atlas* atlas, int64_t records) {
    const CallRange range("seg_set_gemm_record_cap");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_set_gemm_record_cap: atlas is NULL");
    if (records < 0)
        return fail(SEG_ERR_INVALID_ARG, "seg_set_gemm_record_cap: records=%lld < 0",
                    (long long)records);
    std::lock_guard<std::mutex> lock(atlas->mu);
    atlas->gemm.cap_limit = records;
    return SEG_OK;
}

seg_status seg_gemm_stats(const seg_atlas* atlas, int64_t* pairs, int64_t* survivors,
                          int64_t* overflow_fibers, int64_t* screened,
                          int64_t* point_distances) {
    const CallRange range("seg_gemm_stats");
    g_last_error.clear();
    if (!atlas) return fail(SEG_ERR_INVALID_ARG, "seg_gemm_stats: atlas is NULL");
    long long h[5] = {0, 0, 0, 0, 0};
    if (atlas->gemm.stats) {
        cudaError_t e = cudaMemcpy(h, atlas->gemm.stats, sizeof(h), cudaMemcpyDeviceToHost);
        if (e) return cuda_fail(e, "seg_gemm_stats");
    }
    if (pairs) *pairs = h[0];
    if (survivors) *survivors = h[1];
    if (overflow_fibers) *overflow_fibers = h[2];
    if (screened) *screened = h[3];
    if (point_distances) *point_distances = h[4];
    return SEG_OK;
}

}  // extern "C"
