// Batched persistent launch over many subjects (placeholder until built).
#include "seg_internal.cuh"

namespace seg {

void free_batch(BatchState* b) {
    cudaFree(b->table);
    cudaFree(b->counter);
    *b = BatchState{};
}

seg_status batch_launch(const AtlasView&, GemmAtlas*, BatchState*, ScratchArena*, std::mutex*,
                        int, const float* const*, const long long*, int, int* const*,
                        float* const*, cudaStream_t) {
    return fail(SEG_ERR_UNSUPPORTED, "seg_label_batch: not built yet");
}

}  // namespace seg
