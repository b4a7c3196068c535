// Pipe-throughput microbenchmarks: the FP32 and FP64 fused multiply-add
// rates of the current device, the denominators of the sweep kernel's
// per-pipe roofline (its contractions run on these pipes).  Every thread
// runs 8 independent FMA chains for a fixed number of iterations; the
// grid fills every SM with 4 blocks of 256 threads, so issue, not latency,
// bounds the rate.  Timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "ttn_launch.h"

namespace {

constexpr int kChains = 8;

template <class F>
__global__ void __launch_bounds__(256) fma_chains(F m, F c, int iters, F* sink) {
    F a[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = (F)(threadIdx.x + q) * (F)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < kChains; ++q) a[q] = a[q] * m + c;   // contracted to one FMA
    }
    F s = 0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += a[q];
    if (s == (F)-12345.0) sink[blockIdx.x] = s;            // never true: keeps the chains live
}

template <class F>
int time_pipe(int iters, double* tflops, double* ms_out, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int grid = 4 * sms, block = 256;
    F* sink = nullptr;
    e = cudaMallocAsync((void**)&sink, sizeof(F) * grid, s);
    if (e != cudaSuccess) return (int)e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const F m = (F)0.999999, c = (F)1e-7;
    fma_chains<F><<<grid, block, 0, s>>>(m, c, iters / 8, sink);     // warm-up
    cudaEventRecord(t0, s);
    fma_chains<F><<<grid, block, 0, s>>>(m, c, iters, sink);
    cudaEventRecord(t1, s);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(sink, s);
    if (e != cudaSuccess) return (int)e;
    const double flops = 2.0 * kChains * (double)iters * grid * block;
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return (int)cudaGetLastError();
}

}  // namespace

int ttn_pipe_peak_fp32(int iters, double* tflops, double* ms, cudaStream_t s) {
    return time_pipe<float>(iters, tflops, ms, s);
}

int ttn_pipe_peak_fp64(int iters, double* tflops, double* ms, cudaStream_t s) {
    return time_pipe<double>(iters, tflops, ms, s);
}
