/*
 * seg.h - C ABI of libseg, GB300 (sm_103a) atlas-based fiber bundle segmentation.
 *
 * Method (arXiv:1912.11494, Section 2.3-2.4): every subject fiber, resampled to 21 points, is
 * compared with every atlas centroid by the maximum point-pair Euclidean distance
 *     d_ME(a, b) = min( max_i |a_i - b_i|, max_i |a_i - b_(20-i)| )          (Eq. 1, Eq. 2)
 * and labelled with the bundle of the closest centroid whose bundle threshold it passes
 * (d_ME <= theta), or -1 (Algorithm 1, closest-bundle classification).
 *
 * Conventions shared by every entry point:
 *  - Coordinates are float32 millimetres, fibers and centroids laid out [count][21][3]
 *    (point-major, xyz innermost), C-contiguous, 4-byte aligned (a float or int32 buffer
 *    that is not returns SEG_ERR_INVALID_ARG).
 *  - Pointers named d_* are device memory owned by the caller; h_* are host memory owned by
 *    the caller. The library keeps no pointer to caller memory after a call returns, except
 *    that asynchronous work queued on `stream` reads and writes it until the stream reaches it.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Unless a
 *    function says otherwise it only enqueues work on `stream` and returns without waiting.
 *  - Argument errors are detected synchronously and returned before anything is enqueued.
 *    Errors found on the device (a bounded wait that timed out, a full survivor list that could
 *    not be recovered) are recorded in the atlas's device status word; seg_sync_status() waits
 *    for the stream and reports them. No C++ exception crosses this boundary.
 *  - Labels are bundle indices in the caller's numbering; centroid indices (cidx) are positions
 *    in the caller's centroid array.
 *  - Tie rule (Algorithm 1 visits bundles in increasing index, the centroids of a bundle in
 *    their given order, and replaces the best only on a strict decrease): among centroids at the
 *    same float32 squared distance the lowest bundle wins, then the lowest centroid index.
 *  - A fiber with any non-finite coordinate gets label -1 and distance NaN.
 *  - Every entry point is safe to call from several host threads; calls on one atlas from
 *    different streams may overlap, because per-call scratch is stream-ordered.
 *  - Every entry point opens an NVTX range named after it for the duration of the call.
 */
#ifndef SEG_H_
#define SEG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEG_NPTS 21 /* points per fiber and per centroid (Section 2.2, 2.3) */

typedef enum {
    SEG_OK = 0,
    SEG_ERR_INVALID_ARG = 1, /* bad size, NULL where a buffer is required, bad bundle id ... */
    SEG_ERR_CUDA = 2,        /* a CUDA runtime call failed; seg_last_error() has the text */
    SEG_ERR_OOM = 3,         /* device allocation failed */
    SEG_ERR_UNSUPPORTED = 4, /* mode or device not supported (needs sm_103a), or an atlas too
                              * large for a GEMM mode (more than 131,072 operand columns) */
    SEG_ERR_TIMEOUT = 5,     /* a bounded device wait gave up; results of that call invalid */
    SEG_ERR_OVERFLOW = 6     /* a fixed-capacity device list overflowed and was not recovered */
} seg_status;

typedef enum {
    /* Exact FP32 kernel: test1 (centre point) then test2 (end points), test3 (four
     * intermediate points), test4 (all points), each with early exit (Section 2.3-2.4). */
    SEG_MODE_PLAIN = 0,
    /* Tensor-core prune, then the exact test on survivors. The prune is a conservative lower
     * bound d_ME^2 >= (|A|^2 + |B|^2 - 2 A.B) / 21 over the 63 coordinates, for the direct and
     * the reversed centroid, from a BF16 (or TF32) GEMM with FP32 accumulation and a rounding
     * margin. Labels and distances equal SEG_MODE_PLAIN's. Not in the paper. */
    SEG_MODE_GEMM_BF16 = 1,
    SEG_MODE_GEMM_TF32 = 2,
    /* Tensor-core prune with an orientation-free bound, then the exact test (both
     * orientations) on survivors. With c = a_10 and s_i = (a_i + a_(20-i))/2 (i < 10),
     * I(a,b) = |c_a - c_b|^2 + 2 sum_i |s_i(a) - s_i(b)|^2 <= min over orientations of the
     * 21-point sum <= 21 d_ME^2; c and s_9 merge into g = c/sqrt(2) + s_9 (a lower bound of
     * their two terms), so one column per centroid holds 30 features + bias (K = 32). Labels
     * and distances equal SEG_MODE_PLAIN's. Not in the paper.
     * All GEMM modes sort the fibers by the 2 mm cell of their centre point (cells along a
     * Hilbert curve; the centroid columns follow the same order) and skip the
     * (128-fiber, 32-column) blocks whose centre-point boxes are farther apart than every
     * threshold of the block (d_ME >= the centre points' distance); they take at most 131,072
     * operand columns (2M directional, M orientation-free). */
    SEG_MODE_GEMM_INV_BF16 = 3,
    SEG_MODE_GEMM_INV_TF32 = 4,
    /* Spatial culling without the tensor cores: the GEMM modes' locality sort and centre-point
     * block culling (32-fiber groups x 32-centroid chunks), then test1 (the centre point,
     * Section 2.3) on CUDA cores for every pair of the remaining blocks, then the same exact
     * test (both orientations) on the pairs that pass. Labels and distances equal
     * SEG_MODE_PLAIN's. The culling is not in the paper (its Section 2.4 data-locality argument
     * is about caches); it is reported as its own algorithmic mode. */
    SEG_MODE_PLAIN_CULLED = 5,
    /* SEG_MODE_PLAIN_CULLED's work in one kernel after the locality sort: a warp takes a
     * 32-fiber group, stages its rows once, culls the 32-centroid chunks by centre-point box,
     * runs test1 on the chunks in reach and the exact test (both orientations) on their
     * survivors at once, and keeps each fiber's best in on-chip memory. No survivor list, so
     * no list capacity and no overflow path. Labels and distances equal SEG_MODE_PLAIN's. Not
     * in the paper. seg_gemm_screen_bits does not take this mode (it has no separate screen). */
    SEG_MODE_CULLED_FUSED = 6
} seg_mode;

typedef struct seg_atlas seg_atlas; /* opaque; owns its device copies of the atlas */

/* How a fiber is classified once its distances are known (seg_set_classification). */
typedef enum {
    /* d_ME of Eq. 2 (both orientations exactly), a pair passes when d_ME <= theta; the default. */
    SEG_CLASS_EQ2 = 0,
    /* The classification distance D = d_ME + TN (Eq. 3, TN = (|l_S - l_C| / max(l_S, l_C) +
     * 1)^2 - 1, l the polyline arc length of the 21 points); a pair passes when D <= theta and
     * the fiber takes the passing centroid with the smallest D. TN is computed only for pairs
     * whose d_ME passes (Section 2.4; exact, since TN >= 0). Outputs: dist = D. */
    SEG_CLASS_EQ2_TN = 1,
    /* The paper's new algorithm (Section 2.4): the orientation is inferred from test2's end
     * points (the smaller partial maximum; ties direct) and tests 3-4 run in that orientation
     * only, then D = that orientation's maximum + TN as above. It can miss a centroid that
     * Eq. 2 accepts in the other orientation. Outputs: dist = D, orient = the inferred one. */
    SEG_CLASS_PAPER = 2
} seg_classification;

/* Human-readable name of a status code (static string). */
const char* seg_status_string(seg_status s);

/* Text of the last error raised by a seg_* call on this host thread ("" if none). */
const char* seg_last_error(void);

/*
 * Build an atlas handle (the atlasData of Algorithm 1; 21-point centroids grouped in bundles,
 * Section 2.2; per-bundle thresholds, Section 2.3).
 *   d_centroids  device float32 [M][21][3], finite.
 *   d_bundle_of  device int32 [M], values in [0, B).
 *   d_thresholds device float32 [B], finite and > 0, millimetres.
 *   M >= 1, B >= 1, npts must equal SEG_NPTS.
 *   out          receives the handle; release it with seg_destroy_atlas().
 * The handle holds sorted bundle-major copies of the centroids, a spatially ordered copy and
 * the operands of the tensor-core prune (about 1.5 KB per centroid). This call copies the bundle ids and thresholds to
 * the host to validate them and SYNCHRONIZES `stream` before returning.
 */
seg_status seg_create_atlas(const float* d_centroids, const int32_t* d_bundle_of,
                            const float* d_thresholds, int32_t M, int32_t B, int32_t npts,
                            void* stream, seg_atlas** out);

/* Release a handle (NULL is accepted). Waits for the device to finish using it. */
seg_status seg_destroy_atlas(seg_atlas* atlas);

/* Number of centroids M and bundles B of a handle. */
seg_status seg_atlas_info(const seg_atlas* atlas, int32_t* M, int32_t* B);

/*
 * Label n fibers (Algorithm 1 with progressive discarding, Section 2.3; closest bundle only,
 * Section 2.4).
 *   d_fibers  device float32 [n][21][3]; n >= 0 (n = 0 does nothing).
 *   mode      a seg_mode.
 *   d_labels  device int32 [n]: bundle index, or -1 if no centroid passes (required).
 *   d_dist    device float32 [n] or NULL: d_ME to the chosen centroid, +inf if none.
 *   d_cidx    device int32 [n] or NULL: chosen centroid (caller's index), -1 if none.
 *   d_orient  device uint8 [n] or NULL: 0 direct, 1 reversed (ties go to direct).
 * Output buffers must not overlap the input. Scratch (GEMM modes) is allocated stream-ordered
 * on `stream` and released before the call's work completes.
 */
seg_status seg_label(const seg_atlas* atlas, const float* d_fibers, int64_t n, seg_mode mode,
                     int32_t* d_labels, float* d_dist, int32_t* d_cidx, uint8_t* d_orient,
                     void* stream);

/*
 * Every bundle each fiber passes, besides the closest one (Section 2.4, on classifying fibers:
 * the paper's earlier algorithm could give a fiber several bundles; its new one keeps the
 * closest). d_bundle_bits is device uint32 [n][words_per_fiber], overwritten: bit b
 * of fiber f's row (word b / 32, bit b % 32) is set when some centroid of bundle b passes its
 * threshold for f under the atlas's classification (d_ME <= theta, or D <= theta with TN).
 * words_per_fiber >= ceil(B / 32). d_labels (required) and d_dist (or NULL) receive seg_label's
 * closest-bundle result. Every passing pair is evaluated in full (no pruning by the best so far),
 * so this costs more than seg_label on atlases whose bundles overlap.
 */
seg_status seg_label_multi(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                           seg_mode mode, uint32_t* d_bundle_bits, int64_t words_per_fiber,
                           int32_t* d_labels, float* d_dist, void* stream);

/*
 * seg_label on host buffers (not in the paper): h_fibers host float32 [n][21][3], h_labels host
 * int32 [n] (required), h_dist host float32 [n] or NULL. The subject is split into up to
 * SEG_HOST_CHUNKS chunks; chunk c+1 is uploaded on an internal stream while chunk c is labelled
 * (seg_label on `stream`, so the results equal seg_label's), and each chunk's results are
 * copied back on `stream`. Asynchronous: the host buffers must stay valid and unread until
 * `stream` completes. The upload is not ordered after earlier work on `stream`: h_fibers must
 * already hold the fibers when the call is made. The atlas owns two device copies used by
 * alternate calls, so a call's upload overlaps the previous call's labelling (grown on demand;
 * calls on one atlas are serialised on the host). Page-locked (cudaHostAlloc) buffers let the
 * copies overlap the labelling; pageable ones work but serialise.
 */
#define SEG_HOST_CHUNKS 4
seg_status seg_label_host(const seg_atlas* atlas, const float* h_fibers, int64_t n,
                          seg_mode mode, int32_t* h_labels, float* h_dist, void* stream);

/*
 * Resample raw streamlines to the 21 arc-length-equidistant points the labelling takes
 * (Section 2.3 works on fibers of 21 equidistant points; the paper's tractography steps
 * 0.2 mm, Section 2.1). Not tied to an atlas.
 *   d_points  device float32 [P][3]: the points of every streamline, one streamline after
 *             another (4-byte aligned).
 *   d_offsets device int64 [n + 1] (8-byte aligned): streamline f has the points
 *             d_offsets[f] .. d_offsets[f+1] - 1; non-decreasing from d_offsets[0] = 0 (read on
 *             the device and not validated: a decreasing entry gives an empty streamline).
 *   d_out     device float32 [n][21][3].
 * Output point k is the point at arc length k L / 20 along the polyline (L its length; linear
 * interpolation inside the segment that reaches it); points 0 and 20 are the end points. A
 * streamline with one point, or of zero length, gives 21 copies of its first point; one with
 * no point gives NaN coordinates (such a fiber is labelled -1 with distance NaN).
 */
seg_status seg_resample(const float* d_points, const int64_t* d_offsets, int64_t n, float* d_out,
                        void* stream);

/*
 * seg_resample, then seg_label on the 21-point fibers it produced (held in atlas-owned scratch,
 * grown on demand and released stream-ordered): raw tractography in, labels out. Outputs and
 * modes as seg_label.
 */
seg_status seg_label_streamlines(const seg_atlas* atlas, const float* d_points,
                                 const int64_t* d_offsets, int64_t n, seg_mode mode,
                                 int32_t* d_labels, float* d_dist, int32_t* d_cidx,
                                 uint8_t* d_orient, void* stream);

/*
 * Label nsubj subjects of uneven size together (not in the paper; the paper labels one subject
 * at a time, Section 3). Subject s has h_counts[s] >= 0 fibers at device pointer h_fibers[s]
 * and writes h_labels[s] (required) and h_dist[s] (array or entries may be NULL). The pointer
 * arrays are host memory read during the call. Results per subject equal seg_label's.
 *  - SEG_MODE_PLAIN: one persistent launch over (subject, 32-fiber tile) work items.
 *  - GEMM modes, SEG_MODE_PLAIN_CULLED and SEG_MODE_CULLED_FUSED: the subjects form one virtual array of fibers that
 *    goes through the mode's launch sequence once (sorted and screened together).
 * In every mode the launches are captured once into a CUDA graph and replayed; the graph is
 * captured again when the mode, tile shape or subject count changes (and, in the GEMM and
 * culled modes, the total fiber count or the atlas's scratch buffer). The work table is copied
 * to the device on `stream` before each replay from one of two pinned buffers used by
 * alternate calls, so a call waits on the host only for the table copy of two calls earlier.
 */
seg_status seg_label_batch(const seg_atlas* atlas, int32_t nsubj, const float* const* h_fibers,
                           const int64_t* h_counts, seg_mode mode, int32_t* const* h_labels,
                           float* const* h_dist, void* stream);

/*
 * y = A x + t for every point of n fibers (float32 in and out, FP32 arithmetic).
 * h_affine12: host float64 [12], A row-major (9) then t (3). d_out may equal d_in.
 * Not in the paper: the affine is the subject-to-atlas registration refined through seg_grad.
 */
seg_status seg_apply_affine(const float* d_in, int64_t n, const double* h_affine12, float* d_out,
                            void* stream);

/*
 * Gradient of C = sum over labelled fibers of d_ME(T f, c_sigma(f)), T f = A f + t applied to
 * every point, through the argmax point (subgradient; not in the paper).
 *   d_fibers        device float32 [n][21][3], the UNtransformed fibers.
 *   h_affine12      host float64 [12], the affine at which the forward ran.
 *   d_cidx, d_orient the forward's outputs for the transformed fibers (seg_label on
 *                   seg_apply_affine's result): chosen centroid (caller index, -1 = none) and
 *                   orientation.
 *   d_grad_affine12 device float64 [12] (required): dC/dA row-major, then dC/dt. Per-fiber
 *                   terms are FP32; the sum over fibers is FP64 with a fixed order, so the
 *                   result is deterministic.
 *   d_grad_centroids device float32 [M][21][3] or NULL: dC/dc (overwritten, not accumulated).
 *   d_cost          device float64 [1] or NULL: C.
 * The argmax point is recomputed from the fiber and centroid: the lowest point index attaining
 * the maximum point distance in the saved orientation (on FP32 transformed points, as
 * seg_apply_affine computes them). The residual at that point is recomputed exactly enough
 * that every per-fiber term is within a few FP32 ulps (error-free FP32 transformations over
 * the affine split into FP32 high and low parts). The centroid gradient is summed in 64-bit
 * fixed point (multiples of 2^-36), so it is deterministic and rounded to FP32 once. A zero
 * distance contributes zero. n may be at most 2^27 fibers per call (SEG_ERR_INVALID_ARG above).
 */
seg_status seg_grad(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                    const double* h_affine12, const int32_t* d_cidx, const uint8_t* d_orient,
                    double* d_grad_affine12, float* d_grad_centroids, double* d_cost,
                    void* stream);

/*
 * Subject-to-atlas affine refinement driven by seg_grad (not in the paper: its subjects are
 * registered to the atlas beforehand). Minimises
 *     J(T) = sum over labelled fibers of d_ME(T f, c_sigma(f)) + P * (unlabelled fibers),
 * P the atlas's largest threshold (so labelling more fibers never costs more), re-labelling
 * every iteration: seg_apply_affine, seg_label in `mode`, seg_grad, then an Adam step in
 * centred, radius-scaled coordinates with a learning rate of step_mm millimetres (a step
 * moves points by about that much), halved whenever J does not improve on the best so far.
 *   d_fibers     device float32 [n][21][3], the subject as given (n >= 1).
 *   h_affine12   host float64 [12] in: the starting affine (A row-major, then t); out: the best
 *                affine found.
 *   iters >= 0, step_mm > 0.
 *   h_cost       host float64 [iters + 1] or NULL: J at the start and after every iteration.
 *   h_iters_done host int32 or NULL: iterations run.
 * SYNCHRONIZES `stream` once per iteration (the 12 gradient values and J go to the host). The
 * atlas's classification applies to the labelling; the cost is the Eq. 2 distance.
 */
seg_status seg_refine_affine(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                             seg_mode mode, double* h_affine12, int32_t iters, double step_mm,
                             double* h_cost, int32_t* h_iters_done, void* stream);

/*
 * seg_grad without any device allocation, for callers that cannot allocate: code running
 * inside a host allocator callback or a plugin whose host framework owns all device memory,
 * or a process whose device memory is reserved up front. The paper has no counterpart.
 * Arguments, outputs and results are those of seg_grad, except that the FP64 sums use a
 * different fixed order and the centroid gradient is an FP32 atomic sum in no fixed order (so
 * results agree with seg_grad's to rounding, not bit for bit). The scratch is a fixed 1.7 MB
 * array inside the library, held by every GPU that loads it until the process exits:
 *  - n may be at most 4,194,304 fibers per call; larger n returns SEG_ERR_INVALID_ARG;
 *  - calls share that array, so calls whose work overlaps on the GPU race: serialize them;
 *  - every call looks up the array's device address (cudaGetSymbolAddress, with the caller's
 *    device current); the first call on a device may load the library's device code there,
 *    so make that first call before any stream capture.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 */
seg_status seg_grad_noalloc(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                            const double* h_affine12, const int32_t* d_cidx,
                            const uint8_t* d_orient, double* d_grad_affine12,
                            float* d_grad_centroids, double* d_cost, void* stream);

/*
 * Tile shapes of a mode's kernels (the autotuner's search space; not in the paper).
 * seg_num_configs returns how many shapes `mode` has (>= 1). seg_set_config selects shape
 * `config` in [0, seg_num_configs(mode)) for later calls on this atlas; 0 is the default. Every
 * shape gives identical results; only speed differs. seg_get_config reads the selection.
 */
int32_t seg_num_configs(seg_mode mode);
seg_status seg_set_config(seg_atlas* atlas, seg_mode mode, int32_t config);
seg_status seg_get_config(const seg_atlas* atlas, seg_mode mode, int32_t* config);

/*
 * Select the classification of later seg_label / seg_label_host / seg_label_batch calls on
 * this atlas (every mode supports every classification; the default is SEG_CLASS_EQ2). The
 * tensor-core prune and the culling stay exact: D >= d_ME >= their lower bounds. seg_grad
 * always differentiates the Eq. 2 cost.
 */
seg_status seg_set_classification(seg_atlas* atlas, seg_classification cls);
seg_status seg_get_classification(const seg_atlas* atlas, seg_classification* cls);

/*
 * Failure-path controls (for testing error handling; not in the paper).
 * seg_set_wait_limit: limit of the kernels' first bounded device waits, in nanoseconds (the
 *   default is 2 s). With 0, a wait that is not complete at its first try gives up at once:
 *   the kernel records SEG_ERR_TIMEOUT in the atlas's status word (seg_sync_status reports it),
 *   waits (2 s at most) for its own copies and tensor-core work in flight, frees its tensor
 *   memory and returns; the call's results are invalid, later calls are unaffected.
 * seg_set_scratch_limit: cap, in bytes, on each of the atlas's scratch buffers (0: none); a call
 *   that needs more returns SEG_ERR_OOM before any device work.
 */
seg_status seg_set_wait_limit(seg_atlas* atlas, uint64_t ns);
seg_status seg_set_scratch_limit(seg_atlas* atlas, int64_t bytes);

/*
 * Kernel timing (observability; not in the paper). While enabled on an atlas, every kernel the
 * library launches for it records a pair of CUDA events on its stream (no host synchronisation).
 * seg_profile_read waits for those events and returns, for one kernel name, the number of
 * launches and their summed duration in milliseconds since profiling was (re)enabled.
 * Kernel names: "plain", "batch", "gemm_sort", "gemm_prep" (their launches precede the
 * screen), "gemm_screen", "cull_screen" (SEG_MODE_PLAIN_CULLED's test1 screen), "culled_fused"
 * (SEG_MODE_CULLED_FUSED's one kernel after the sort), "gemm_exact",
 * "gemm_finalize", "grad". Enabling (or disabling) clears what was recorded.
 */
seg_status seg_profile_enable(seg_atlas* atlas, int32_t enable);
seg_status seg_profile_read(seg_atlas* atlas, const char* kernel, int64_t* launches,
                            double* total_ms);

/*
 * Wait for `stream`, then report and clear the atlas's device status word: SEG_OK, or the first
 * device-side error (SEG_ERR_TIMEOUT, SEG_ERR_OVERFLOW) recorded since the last call.
 */
seg_status seg_sync_status(const seg_atlas* atlas, void* stream);

/*
 * Limit the survivor list of the GEMM modes to `records` block records (each: 32 fibers x 32
 * columns, 136 bytes of scratch); 0 restores the default (16 per 32 fibers + 65,536). Fibers
 * whose survivors do not fit are rescanned exactly against the whole atlas, so results do not
 * change; only time and scratch memory do. Not in the paper.
 */
seg_status seg_set_gemm_record_cap(seg_atlas* atlas, int64_t records);

/*
 * Statistics of the last GEMM-mode seg_label on this atlas (read after the stream finished):
 * pairs = fibers x columns (2M directional, or M orientation-free) candidates, screened = the
 * candidates inside the (128-fiber x N-column) blocks the tensor cores computed (blocks whose
 * centre-point boxes lie farther apart than every threshold are skipped; padding included),
 * survivors = candidates kept by the tensor-core bound, overflow_fibers = fibers rescanned by
 * the exact kernel because the survivor list was full, point_distances = squared point
 * distances the exact re-check of the survivors evaluated (the rescan not included). Any
 * pointer may be NULL.
 */
seg_status seg_gemm_stats(const seg_atlas* atlas, int64_t* pairs, int64_t* survivors,
                          int64_t* overflow_fibers, int64_t* screened,
                          int64_t* point_distances);

/*
 * Diagnostic of the tensor-core prune (not in the paper): run the locality sort, the block
 * culling and the screen of a GEMM mode (or SEG_MODE_PLAIN_CULLED's test1 screen) on n fibers and return the pairs the screen keeps for
 * the exact test, instead of labels. d_bits is device uint32 [n][words_per_fiber], overwritten:
 * bit k of fiber f's row is set when the screen keeps column k for f, where k = 2 c + o for
 * the directional modes (c the caller's centroid index, o = 0 direct, 1 reversed) and k = c for
 * the orientation-free modes and SEG_MODE_PLAIN_CULLED. words_per_fiber >= ceil(2M / 32) (directional) or ceil(M / 32).
 * Every pair whose float32 exact test passes (d_o^2 <= theta^2) is kept; seg_gemm_stats reports
 * the screen's counters afterwards (overflow_fibers > 0 means survivors of those fibers were
 * dropped for lack of record space and the output is incomplete for them).
 */
seg_status seg_gemm_screen_bits(const seg_atlas* atlas, const float* d_fibers, int64_t n,
                                seg_mode mode, uint32_t* d_bits, int64_t words_per_fiber,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SEG_H_ */
