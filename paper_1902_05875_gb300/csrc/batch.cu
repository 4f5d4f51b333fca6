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
