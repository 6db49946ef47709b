// SEG_MODE_GEMM_*: tensor-core lower-bound prune + exact re-check (placeholder until built).
#include "seg_internal.cuh"

namespace seg {

seg_status prep_gemm_atlas(const AtlasView& at, GemmAtlas* g, cudaStream_t st) {
    (void)at;
    (void)st;
    cudaError_t e = cudaMalloc(&g->stats, 3 * sizeof(long long));
    if (e) return cuda_fail(e, "gemm stats");
    return cudaMemsetAsync(g->stats, 0, 3 * sizeof(long long), st) ? SEG_ERR_CUDA : SEG_OK;
}

int gemm_num_configs() { return 1; }

void free_gemm_atlas(GemmAtlas* g) {
    cudaFree(g->b_bf16);
    cudaFree(g->b_tf32);
    cudaFree(g->stats);
    *g = GemmAtlas{};
}

seg_status label_gemm(const AtlasView&, GemmAtlas*, ScratchArena*, std::mutex*, const float*,
                      long long, bool, int*, float*, int*, unsigned char*, cudaStream_t) {
    return fail(SEG_ERR_UNSUPPORTED, "seg_label: GEMM modes are not built yet");
}

}  // namespace seg
