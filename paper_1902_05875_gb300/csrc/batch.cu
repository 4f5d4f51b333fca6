// Batched evaluation of many independent instances (each a medium with its own
// plan and its own particles), e.g. the many small layered-media problems of
// a parameter sweep.  Host worker threads, each driving its own stream, take
// instances from a shared counter and run tefmm_eval on them, so the
// instances' kernels overlap on the GPU and one instance's host-side waits
// (tree levels, list sizes) hide behind the others' work.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "internal.cuh"

extern "C" int tefmm_eval_batched(int n, tefmm_plan *plans, const tefmm_batch_item *items,
                                  int n_workers, void *stream, int *status) {
    if (n < 0 || (n > 0 && (!plans || !items))) return TEFMM_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return TEFMM_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return TEFMM_ERR_INVALID_ARG;   // a plan is not shared
    }
    if (n == 0) return TEFMM_OK;
    const int nw = std::max(1, std::min(n_workers > 0 ? n_workers : 8, n));
    cudaStream_t cs = (cudaStream_t)stream;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    cudaEvent_t ready;
    CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(ready, cs));          // the inputs are ready on the caller's stream
    std::vector<cudaStream_t> ws(nw, nullptr);
    std::vector<cudaEvent_t> done(nw, nullptr);
    int err = TEFMM_OK;
    for (int w = 0; w < nw && err == TEFMM_OK; ++w) {
        if (cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamWaitEvent(ws[w], ready, 0) != cudaSuccess)
            err = TEFMM_ERR_CUDA;
    }
    std::vector<int> st(n, TEFMM_OK);
    if (err == TEFMM_OK) {
        std::atomic<int> next(0);
        auto work = [&](int w) {
            cudaSetDevice(dev);
            for (;;) {
                const int i = next.fetch_add(1);
                if (i >= n) break;
                const tefmm_batch_item &it = items[i];
                const bool shared = it.tx == nullptr;
                st[i] = tefmm_eval(plans[i], it.ns, it.sx, it.sy, it.sz, it.q, shared ? it.ns : it.nt,
                                   shared ? it.sx : it.tx, shared ? it.sy : it.ty,
                                   shared ? it.sz : it.tz, it.phi, ws[w]);
            }
            cudaEventRecord(done[w], ws[w]);
        };
        std::vector<std::thread> th;
        for (int w = 0; w < nw; ++w) th.emplace_back(work, w);
        for (auto &t : th) t.join();
        for (int w = 0; w < nw; ++w)
            if (cudaStreamWaitEvent(cs, done[w], 0) != cudaSuccess) err = TEFMM_ERR_CUDA;
    }
    for (int w = 0; w < nw; ++w) {
        if (done[w]) cudaEventDestroy(done[w]);
        if (ws[w]) cudaStreamDestroy(ws[w]);
    }
    cudaEventDestroy(ready);
    for (int i = 0; i < n; ++i) {
        if (status) status[i] = st[i];
        if (err == TEFMM_OK && st[i] != TEFMM_OK) err = st[i];
    }
    return err;
}

// ---------------------------------------------------------------------------
// Batch graph: the charge phases (tefmm_apply) of many plans, each on the
// points of its last tefmm_set_points, captured once into one CUDA graph and
// then replayed by a single cudaGraphLaunch per batch.  Each plan's apply is
// its own branch of the graph (forked from and joined to the caller's
// stream), so the instances' kernels overlap on the GPU as one launch.
struct tefmm_batch_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t origin = nullptr;     // the capture's origin stream (the legacy stream cannot be captured)
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<tefmm_plan> plans;
};

static void batch_graph_free(tefmm_batch_graph_s *G) {
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    for (cudaEvent_t e : G->events) cudaEventDestroy(e);
    for (cudaStream_t s : G->streams) cudaStreamDestroy(s);
    if (G->origin) cudaStreamDestroy(G->origin);
    delete G;
}

extern "C" int tefmm_batch_graph_create(int n, tefmm_plan *plans, const double *const *q, double *const *phi,
                                        void *stream, tefmm_batch_graph *out) {
    if (!out || n <= 0 || !plans || !q || !phi) return TEFMM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !plans[i]->geom_ready || !q[i] || !phi[i]) return TEFMM_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return TEFMM_ERR_INVALID_ARG;   // a plan is not shared
    }
    // one apply per plan outside the capture: sizes its buffers (no allocation
    // may happen inside a capture) and checks that it runs
    for (int i = 0; i < n; ++i) TRY(tefmm_apply(plans[i], q[i], phi[i], stream));
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    tefmm_batch_graph_s *G = new tefmm_batch_graph_s();
    G->plans.assign(plans, plans + n);
    int err = TEFMM_OK;
    if (cudaStreamCreateWithFlags(&G->origin, cudaStreamNonBlocking) != cudaSuccess) err = TEFMM_ERR_CUDA;
    cudaStream_t cs = G->origin;
    G->streams.resize(n, nullptr);
    G->events.resize(n + 1, nullptr);
    for (int i = 0; i < n && err == TEFMM_OK; ++i)
        if (cudaStreamCreateWithFlags(&G->streams[i], cudaStreamNonBlocking) != cudaSuccess) err = TEFMM_ERR_CUDA;
    for (int i = 0; i <= n && err == TEFMM_OK; ++i)
        if (cudaEventCreateWithFlags(&G->events[i], cudaEventDisableTiming) != cudaSuccess) err = TEFMM_ERR_CUDA;
    if (err != TEFMM_OK) {
        batch_graph_free(G);
        return err;
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        fprintf(stderr, "tefmm: stream capture could not begin: %s\n", cudaGetErrorString(cudaGetLastError()));
        batch_graph_free(G);
        return TEFMM_ERR_CUDA;
    }
    if (cudaEventRecord(G->events[n], cs) != cudaSuccess) err = TEFMM_ERR_CUDA;
    for (int i = 0; i < n && err == TEFMM_OK; ++i) {
        if (cudaStreamWaitEvent(G->streams[i], G->events[n], 0) != cudaSuccess) err = TEFMM_ERR_CUDA;
        if (err == TEFMM_OK) err = tefmm_apply(plans[i], q[i], phi[i], G->streams[i]);
        if (err == TEFMM_OK && (cudaEventRecord(G->events[i], G->streams[i]) != cudaSuccess ||
                                cudaStreamWaitEvent(cs, G->events[i], 0) != cudaSuccess))
            err = TEFMM_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    G->graph = graph;
    if (err == TEFMM_OK && ec != cudaSuccess) err = TEFMM_ERR_CUDA;
    if (err == TEFMM_OK && cudaGraphInstantiate(&G->exec, G->graph, 0) != cudaSuccess) err = TEFMM_ERR_CUDA;
    if (err != TEFMM_OK) {
        fprintf(stderr, "tefmm: batch graph capture failed (status %d, end capture: %s)\n", err,
                cudaGetErrorString(ec));
        cudaGetLastError();
        batch_graph_free(G);
        return err;
    }
    *out = G;
    return TEFMM_OK;
}

extern "C" int tefmm_batch_graph_launch(tefmm_batch_graph G, void *stream) {
    if (!G || !G->exec) return TEFMM_ERR_INVALID_ARG;
    CUDA_TRY(cudaGraphLaunch(G->exec, (cudaStream_t)stream));
    return TEFMM_OK;
}

extern "C" int tefmm_batch_graph_destroy(tefmm_batch_graph G) {
    if (G) batch_graph_free(G);
    return TEFMM_OK;
}
