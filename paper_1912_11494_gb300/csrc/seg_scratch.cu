// Atlas-owned growable scratch buffer with stream ordering through an event.
#include "seg_internal.cuh"

namespace seg {

seg_status scratch_acquire(ScratchArena* s, size_t bytes, cudaStream_t st, void** out) {
    cudaError_t e;
    if (!s->last_use) {
        if ((e = cudaEventCreateWithFlags(&s->last_use, cudaEventDisableTiming)))
            return cuda_fail(e, "scratch event");
    } else if ((e = cudaStreamWaitEvent(st, s->last_use, 0))) {
        return cuda_fail(e, "scratch wait");
    }
    if (s->limit && bytes > s->limit)
        return fail(SEG_ERR_OOM, "scratch of %zu bytes exceeds the atlas's limit of %zu bytes",
                    bytes, s->limit);
    if (bytes > s->bytes) {
        // the previous owner may still be running on another stream
        if ((e = cudaEventSynchronize(s->last_use))) return cuda_fail(e, "scratch sync");
        cudaFree(s->ptr);
        s->ptr = nullptr;
        s->bytes = 0;
        if ((e = cudaMalloc(&s->ptr, bytes))) {
            s->ptr = nullptr;
            return cuda_fail(e, "scratch allocation");
        }
        s->bytes = bytes;
    }
    *out = s->ptr;
    return SEG_OK;
}

seg_status scratch_release(ScratchArena* s, cudaStream_t st) {
    cudaError_t e = cudaEventRecord(s->last_use, st);
    return e ? cuda_fail(e, "scratch record") : SEG_OK;
}

void free_scratch(ScratchArena* s) {
    if (s->last_use) cudaEventDestroy(s->last_use);
    cudaFree(s->ptr);
    *s = ScratchArena{};
}

}  // namespace seg
