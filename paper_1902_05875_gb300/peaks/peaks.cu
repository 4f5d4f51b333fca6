// Arithmetic peaks of the GPU for the roofline denominators of the SIMT
// kernels: FP64 and FP32 fused multiply-add throughput, measured with CUDA
// events on a kernel that keeps every lane busy with independent FMA chains.
// A measurement aid of the benchmark, not part of the matrix-vector product.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int CHAINS = 8;   // independent dependency chains per thread (hides FMA latency)

template <class T>
__global__ void k_fma(int iters, T a, T b, T *out) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == (T)1.2345) out[0] = s;   // practically never: keeps the chains alive
}

template <class T>
double run(int blocks, int threads, int iters, int reps) {
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma<T><<<blocks, threads>>>(iters, (T)0.999999, (T)1e-7, out);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        k_fma<T><<<blocks, threads>>>(iters, (T)0.999999, (T)1e-7, out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const bool ok = cudaGetLastError() == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (!ok) return -1.0;
    const double flops = 2.0 * CHAINS * (double)iters * blocks * (double)threads;
    return flops / (best * 1e-3);
}

}  // namespace

// FMA throughput in FLOP/s (2 per FMA) of `blocks` x `threads` threads, each
// running 8 independent chains of `iters` FMAs; best of `reps` launches.
// Returns a negative value if a CUDA call failed.
extern "C" double tefmm_peaks_fp64(int blocks, int threads, int iters, int reps) {
    return run<double>(blocks, threads, iters, reps);
}
extern "C" double tefmm_peaks_fp32(int blocks, int threads, int iters, int reps) {
    return run<float>(blocks, threads, iters, reps);
}
