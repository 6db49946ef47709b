// Host-side internals shared by the libseg sources: atlas-owned scratch, the tensor-core
// prune's operands, the batch graph cache and the launchers.
#pragma once

#include <cstdarg>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "seg_common.cuh"

namespace seg {

seg_status fail(seg_status s, const char* fmt, ...);
seg_status cuda_fail(cudaError_t e, const char* what);

// Event-pair timing of the library's kernels (seg_profile_enable / seg_profile_read).
enum ProfSlot { PROF_PLAIN = 0, PROF_BATCH, PROF_GEMM_PREP, PROF_GEMM_SCREEN, PROF_GEMM_EXACT,
                PROF_GEMM_FINAL, PROF_GRAD, PROF_GEMM_SORT, PROF_CULL_SCREEN, PROF_FUSED,
                PROF_SLOTS };
struct Profiler {
    bool enabled = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;  // reusable events
    size_t used = 0;
    std::vector<int> slot_of;                                // slot of each used pair
    void begin(int slot, cudaStream_t st, cudaEvent_t* end_out);
    void clear();
    ~Profiler();
};
// RAII helper: records the start event now and the end event when it goes out of scope.
struct ProfScope {
    Profiler* p;
    cudaStream_t st;
    cudaEvent_t end = nullptr;
    ProfScope(Profiler* prof, int slot, cudaStream_t s) : p(prof), st(s) {
        if (p && p->enabled) p->begin(slot, st, &end);
    }
    ~ProfScope() {
        if (end) cudaEventRecord(end, st);
    }
};

// A growable device buffer owned by an atlas. Users lock the atlas mutex on the host and order
// themselves on the device through `last_use`, so calls from different streams never overlap
// on it.
struct ScratchArena {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaEvent_t last_use = nullptr;
    size_t limit = 0;  // the caller's cap on this arena's size (0: none); above it SEG_ERR_OOM
};
seg_status scratch_acquire(ScratchArena* s, size_t bytes, cudaStream_t st, void** out);
seg_status scratch_release(ScratchArena* s, cudaStream_t st);
void free_scratch(ScratchArena* s);

// Operands of the tensor-core prune (SEG_MODE_GEMM_*), built with the atlas.
struct GemmAtlas {
    int cols = 0;             // 2M columns: centroid at spatial position c direct at 2c,
                              // reversed at 2c+1
    int cols_pad = 0;         // cols rounded up to the N tile
    void* b_bf16 = nullptr;   // [cols_pad][64] bf16, centred, K-major
    void* b_tf32 = nullptr;   // [cols_pad][64] fp32 holding TF32-rounded values
    int cols_inv = 0;         // M columns of orientation-free features (spatial position c at c)
    int cols_inv_pad = 0;
    void* bi_bf16 = nullptr;  // [cols_inv_pad][32]
    void* bi_tf32 = nullptr;
    // Columns follow the spatial order of the centroids (Hilbert-curve order of the centre
    // point's cell): spatial position c holds sorted centroid sp_s[c]; directional columns
    // 2c, 2c+1.
    int* sp_s = nullptr;      // [M]
    float4* cen_sp = nullptr; // [M][21] centroid rows in spatial order, point-major
    float* thr2_sp = nullptr; // [M] theta^2 in spatial order
    float4* ctr_sp = nullptr; // [M] centre point and theta^2 in spatial order
    float4* scr_sp = nullptr; // [M rounded up to 32] the test1 screen row (AtlasView::scr2) in
                              // spatial order; the pad (0, 0, 0, -inf) passes no fiber
    float4* tbox32 = nullptr; // [cols_inv_pad / 32][2] boxes of the 32-centroid chunks (lo, hi;
                              // lo.w the largest theta^2, hi.w the smallest)
    float4* wbox32 = nullptr; // [ceil(chunks / 32)][2] boxes of 32 consecutive chunks
    float4* end_sp = nullptr; // [M][3] points 0, 10, 20 in spatial order (w: the length,
                              // theta^2, 0): what test1 and test2 read, 48 bytes a centroid
    long long* stats = nullptr;  // [5] pairs, survivors, overflow fibers, screened pairs,
                                 // point distances of the exact re-check
    long long cap_limit = 0;     // caller's limit on survivor block records (0: none)
    int rec_per_group = 16;      // default room for block records per 32 fibers (from the
                                 // atlas's largest bundle)
};
seg_status prep_gemm_atlas(const AtlasView& at, const int* sp_host, int max_per_bundle,
                           GemmAtlas* g, cudaStream_t st);
void free_gemm_atlas(GemmAtlas* g);
int gemm_num_configs();
seg_status label_gemm(const AtlasView& at, GemmAtlas* g, ScratchArena* scratch, std::mutex* mu,
                      const float* fib, long long n, int mode, int* labels, float* dist,
                      int* cidx, unsigned char* orient, cudaStream_t st, int config,
                      Profiler* prof = nullptr, unsigned* dbg_bits = nullptr,
                      long long dbg_words = 0);

// Cached CUDA graph of the batched launch. The work table goes to the device with one copy on
// the caller's stream before each replay, from one of two pinned host buffers used by
// alternate calls (a buffer is rewritten only after the copy of two calls ago has run), so
// back-to-back calls do not wait for each other on the host.
struct BatchState {
    void* graph_exec = nullptr;   // cudaGraphExec_t
    int mode = -1, nsubj = -1, config = -1, cls = -1;
    unsigned long long wait_ns = 0;
    long long total = -1;         // fibers of all subjects (GEMM modes: sizes the graph)
    void* scratch_ptr = nullptr;  // the scratch the GEMM graph was captured on
    void* table = nullptr;        // device BatchEntry[table_cap]
    void* table_host[2] = {nullptr, nullptr};  // pinned copies
    void* copied[2] = {nullptr, nullptr};      // cudaEvent_t after each buffer's last copy
    int next = 0;                 // host buffer of the next call
    size_t table_cap = 0;         // entries allocated
    void* counter = nullptr;      // device work counter (plain mode)
    void* cap_stream = nullptr;   // cudaStream_t used for capture
    void* done = nullptr;         // cudaEvent_t recorded after each replay
};
void free_batch(BatchState* b);
seg_status batch_launch(const AtlasView& at, GemmAtlas* g, BatchState* b, ScratchArena* scratch,
                        std::mutex* mu, int nsubj, const float* const* fib,
                        const long long* counts, int mode, int* const* labels,
                        float* const* dist, cudaStream_t st, int config);
// GEMM modes: every subject in one virtual array through one captured launch sequence (table
// already uploaded to b->table by the caller's stream order, see batch_launch).
seg_status gemm_batch_launch(const AtlasView& at, GemmAtlas* ga, ScratchArena* scratch,
                             BatchState* b, int nsubj, long long total, int mode, int config,
                             const void* host_table, size_t table_bytes, void* copied_event,
                             cudaStream_t st);

seg_status grad_launch(const AtlasView& at, const int* inv_perm, ScratchArena* scratch,
                       std::mutex* mu, const float* fib, long long n, const double* h_aff,
                       const int* cidx, const unsigned char* orient, double* grad_aff,
                       float* grad_cen, double* cost, cudaStream_t st);
seg_status grad_noalloc_launch(const AtlasView& at, const int* inv_perm, const float* fib,
                               long long n, const double* h_aff, const int* cidx,
                               const unsigned char* orient, double* grad_aff, float* grad_cen,
                               double* cost, cudaStream_t st);
seg_status refine_launch(const seg_atlas* atlas, const AtlasView& at, ScratchArena* scratch,
                         std::mutex* mu, const float* fib, long long n, int mode, double* aff,
                         int iters, double step_mm, double penalty, double* cost_out,
                         int* iters_done, cudaStream_t st);
seg_status resample_launch(const float* pts, const long long* off, long long n, float* out,
                           cudaStream_t st);
seg_status apply_affine_launch(const float* in, long long n, const double* h_aff, float* out,
                               cudaStream_t st);

}  // namespace seg
