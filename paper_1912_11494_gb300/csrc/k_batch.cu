// seg_label_batch: many subjects of uneven size (not in the paper; it labels one subject at a
// time, Section 3).
//
// SEG_MODE_PLAIN runs one persistent launch over a device work table of (subject, 32-fiber tile)
// items taken from an atomic counter; the counter reset and the launch are captured once into a
// CUDA graph per (atlas, subject count, tile shape) and replayed. The GEMM modes and
// SEG_MODE_PLAIN_CULLED treat the subjects as one virtual array of fibers and replay their
// whole captured sequence of kernels (gemm_batch_launch). In every mode the work table is
// copied to the device on the caller's stream just before the replay, from one of two pinned
// host buffers used by alternate calls.
#include "seg_internal.cuh"

namespace seg {

void free_batch(BatchState* b) {
    if (b->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)b->graph_exec);
    for (void* ev : {b->done, b->copied[0], b->copied[1]})
        if (ev) cudaEventDestroy((cudaEvent_t)ev);
    if (b->cap_stream) cudaStreamDestroy((cudaStream_t)b->cap_stream);
    cudaFree(b->table);
    cudaFreeHost(b->table_host[0]);
    cudaFreeHost(b->table_host[1]);
    cudaFree(b->counter);
    *b = BatchState{};
}

static seg_status capture_plain(const AtlasView& at, BatchState* b, int nsubj, int config) {
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
    cudaError_t e2 = launch_label_plain_batch((const BatchEntry*)b->table, nsubj,
                                              (unsigned long long*)b->counter, at, sms, cs,
                                              config);
    e = cudaStreamEndCapture(cs, &graph);
    if (e1 || e2 || e) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e1 ? e1 : e2 ? e2 : e, "seg_label_batch: capture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) return cuda_fail(e, "seg_label_batch: instantiate");
    b->graph_exec = exec;
    b->mode = SEG_MODE_PLAIN;
    b->nsubj = nsubj;
    b->config = config;
    b->total = -1;
    b->scratch_ptr = nullptr;
    b->cls = at.cls;
    b->wait_ns = at.wait_ns;
    return SEG_OK;
}

// Stream, events, counter and tables that hold at least `entries` entries.
static seg_status batch_resources(BatchState* b, size_t entries) {
    cudaError_t e;
    if (!b->cap_stream) {
        cudaStream_t cs;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)))
            return cuda_fail(e, "seg_label_batch: stream");
        b->cap_stream = cs;
        for (void** ev : {&b->done, &b->copied[0], &b->copied[1]}) {
            cudaEvent_t x;
            if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)))
                return cuda_fail(e, "seg_label_batch: event");
            *ev = x;
        }
        if ((e = cudaMalloc(&b->counter, sizeof(unsigned long long))))
            return cuda_fail(e, "seg_label_batch: counter");
    }
    if (entries > b->table_cap) {
        // every earlier replay and copy must be done with the old tables
        if ((e = cudaEventSynchronize((cudaEvent_t)b->done)) ||
            (e = cudaEventSynchronize((cudaEvent_t)b->copied[0])) ||
            (e = cudaEventSynchronize((cudaEvent_t)b->copied[1])))
            return cuda_fail(e, "seg_label_batch: wait for earlier batches");
        cudaFree(b->table);
        cudaFreeHost(b->table_host[0]);
        cudaFreeHost(b->table_host[1]);
        b->table = b->table_host[0] = b->table_host[1] = nullptr;
        b->table_cap = 0;
        if (b->graph_exec) {  // captured with the old table's address
            cudaGraphExecDestroy((cudaGraphExec_t)b->graph_exec);
            b->graph_exec = nullptr;
        }
        const size_t cap = entries < 64 ? 64 : entries;
        if ((e = cudaMalloc(&b->table, cap * sizeof(BatchEntry))) ||
            (e = cudaHostAlloc(&b->table_host[0], cap * sizeof(BatchEntry), cudaHostAllocDefault)) ||
            (e = cudaHostAlloc(&b->table_host[1], cap * sizeof(BatchEntry), cudaHostAllocDefault)))
            return cuda_fail(e, "seg_label_batch: work table");
        b->table_cap = cap;
    }
    return SEG_OK;
}

seg_status batch_launch(const AtlasView& at, GemmAtlas* g, BatchState* b, ScratchArena* scratch,
                        std::mutex* mu, int nsubj, const float* const* fib,
                        const long long* counts, int mode, int* const* labels,
                        float* const* dist, cudaStream_t st, int config) {
    long long total = 0;
    for (int s = 0; s < nsubj; ++s) total += counts[s];
    if (total == 0) return SEG_OK;
    std::lock_guard<std::mutex> lock(*mu);
    seg_status r = batch_resources(b, (size_t)nsubj + 1);
    if (r != SEG_OK) return r;
    cudaError_t e;
    // this call's host buffer: its copy of two calls ago must have run
    const int k = b->next;
    b->next ^= 1;
    if ((e = cudaEventSynchronize((cudaEvent_t)b->copied[k])))
        return cuda_fail(e, "seg_label_batch: wait for the table copy of two calls ago");
    BatchEntry* t = (BatchEntry*)b->table_host[k];
    long long tiles = 0, first = 0;
    for (int s = 0; s < nsubj; ++s) {
        t[s].fib = fib[s];
        t[s].n = counts[s];
        t[s].labels = labels[s];
        t[s].dist = dist ? dist[s] : nullptr;
        t[s].tile0 = tiles;
        t[s].first = first;
        tiles += (counts[s] + PLAIN_TILE - 1) / PLAIN_TILE;
        first += counts[s];
    }
    t[nsubj] = BatchEntry{nullptr, 0, nullptr, nullptr, tiles, first};
    const size_t bytes = sizeof(BatchEntry) * ((size_t)nsubj + 1);
    // the previous replay (on whatever stream) is done with the device table and counter
    if ((e = cudaStreamWaitEvent(st, (cudaEvent_t)b->done, 0)))
        return cuda_fail(e, "seg_label_batch: ordering");
    if (mode != SEG_MODE_PLAIN) {
        r = gemm_batch_launch(at, g, scratch, b, nsubj, total, mode, config, t, bytes,
                              b->copied[k], st);
        if (r != SEG_OK) return r;
    } else {
        if (!b->graph_exec || b->mode != SEG_MODE_PLAIN || b->nsubj != nsubj ||
            b->config != config || b->cls != at.cls || b->wait_ns != at.wait_ns) {
            r = capture_plain(at, b, nsubj, config);
            if (r != SEG_OK) return r;
        }
        if ((e = cudaMemcpyAsync(b->table, t, bytes, cudaMemcpyHostToDevice, st)) ||
            (e = cudaEventRecord((cudaEvent_t)b->copied[k], st)) ||
            (e = cudaGraphLaunch((cudaGraphExec_t)b->graph_exec, st)))
            return cuda_fail(e, "seg_label_batch: graph launch");
    }
    if ((e = cudaEventRecord((cudaEvent_t)b->done, st)))
        return cuda_fail(e, "seg_label_batch: record");
    return SEG_OK;
}

}  // namespace seg
