// seg_label_batch: many subjects of uneven size (not in the paper; it labels one subject at a
// time, Section 3).
//
// SEG_MODE_PLAIN runs one persistent launch over a device work table of (subject, 32-fiber tile)
// items taken from an atomic counter; the counter reset, the table upload and the launch are
// captured once into a CUDA graph per (atlas, subject count, tile shape) and replayed with the
// new table (the graph's copy node reads a pinned host buffer rewritten before each replay).
// The GEMM modes label the subjects one after another on the caller's stream.
#include "seg_internal.cuh"

namespace seg {

void free_batch(BatchState* b) {
    if (b->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)b->graph_exec);
    if (b->done) cudaEventDestroy((cudaEvent_t)b->done);
    if (b->cap_stream) cudaStreamDestroy((cudaStream_t)b->cap_stream);
    cudaFree(b->table);
    cudaFreeHost(b->table_host);
    cudaFree(b->counter);
    *b = BatchState{};
}

static seg_status capture(const AtlasView& at, BatchState* b, int nsubj, int config) {
    if (b->graph_exec) {
        cudaGraphExecDestroy((cudaGraphExec_t)b->graph_exec);
        b->graph_exec = nullptr;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t cs = (cudaStream_t)b->cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e) return cuda_fail(e, "seg_label_batch: begin capture");
    cudaError_t e1 = cudaMemsetAsync(b->counter, 0, sizeof(unsigned long long), cs);
    cudaError_t e2 = cudaMemcpyAsync(b->table, b->table_host, sizeof(BatchEntry) * (nsubj + 1),
                                     cudaMemcpyHostToDevice, cs);
    cudaError_t e3 = launch_label_plain_batch((const BatchEntry*)b->table, nsubj,
                                              (unsigned long long*)b->counter, at, sms, cs,
                                              config);
    e = cudaStreamEndCapture(cs, &graph);
    if (e1 || e2 || e3 || e) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e1 ? e1 : e2 ? e2 : e3 ? e3 : e, "seg_label_batch: capture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) return cuda_fail(e, "seg_label_batch: instantiate");
    b->graph_exec = exec;
    b->nsubj = nsubj;
    b->config = config;
    return SEG_OK;
}

seg_status batch_launch(const AtlasView& at, GemmAtlas* g, BatchState* b, ScratchArena* scratch,
                        std::mutex* mu, int nsubj, const float* const* fib,
                        const long long* counts, int mode, int* const* labels,
                        float* const* dist, cudaStream_t st, int config) {
    if (mode != SEG_MODE_PLAIN) {
        for (int s = 0; s < nsubj; ++s) {
            if (counts[s] == 0) continue;
            seg_status r = label_gemm(at, g, scratch, mu, fib[s], counts[s], mode, labels[s],
                                      dist ? dist[s] : nullptr, nullptr, nullptr, st, config);
            if (r != SEG_OK) return r;
        }
        return SEG_OK;
    }
    std::lock_guard<std::mutex> lock(*mu);
    cudaError_t e;
    if (!b->cap_stream) {
        cudaStream_t cs;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))
            return cuda_fail(e, "seg_label_batch: stream");
        b->cap_stream = cs;
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)))
            return cuda_fail(e, "seg_label_batch: event");
        b->done = ev;
        if ((e = cudaMalloc(&b->counter, sizeof(unsigned long long))))
            return cuda_fail(e, "seg_label_batch: counter");
    }
    // the previous replay must have read the pinned table before it is rewritten
    if ((e = cudaEventSynchronize((cudaEvent_t)b->done)))
        return cuda_fail(e, "seg_label_batch: wait for the previous batch");
    if ((size_t)nsubj + 1 > b->table_cap) {
        cudaFree(b->table);
        cudaFreeHost(b->table_host);
        b->table = b->table_host = nullptr;
        b->table_cap = 0;
        if (b->graph_exec) {
            cudaGraphExecDestroy((cudaGraphExec_t)b->graph_exec);
            b->graph_exec = nullptr;
        }
        const size_t cap = (size_t)nsubj + 1;
        if ((e = cudaMalloc(&b->table, cap * sizeof(BatchEntry))) ||
            (e = cudaHostAlloc(&b->table_host, cap * sizeof(BatchEntry), cudaHostAllocDefault)))
            return cuda_fail(e, "seg_label_batch: work table");
        b->table_cap = cap;
    }
    BatchEntry* t = (BatchEntry*)b->table_host;
    long long tiles = 0;
    for (int s = 0; s < nsubj; ++s) {
        t[s].fib = fib[s];
        t[s].n = counts[s];
        t[s].labels = labels[s];
        t[s].dist = dist ? dist[s] : nullptr;
        t[s].tile0 = tiles;
        t[s].pad = 0;
        tiles += (counts[s] + PLAIN_TILE - 1) / PLAIN_TILE;
    }
    t[nsubj] = BatchEntry{nullptr, 0, nullptr, nullptr, tiles, 0};
    if (!b->graph_exec || b->nsubj != nsubj || b->config != config) {
        seg_status r = capture(at, b, nsubj, config);
        if (r != SEG_OK) return r;
    }
    if ((e = cudaGraphLaunch((cudaGraphExec_t)b->graph_exec, st)))
        return cuda_fail(e, "seg_label_batch: graph launch");
    if ((e = cudaEventRecord((cudaEvent_t)b->done, st)))
        return cuda_fail(e, "seg_label_batch: record");
    return SEG_OK;
}

}  // namespace seg
