// Kernel-level mode product of the complex64 bulk: on the tensor cores
// (tcgen05, 3xTF32) or by the sweep's FFMA routine, for testing and
// timing the contraction alone.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ttn_device.cuh"
#include "ttn_launch.h"
#include "ttn_tc.cuh"

namespace {

constexpr int kTcStage = 160 * 1024;

__global__ void __launch_bounds__(256, 1) tc_mode_kernel(float2* out, const float2* in, int64_t L, int n, int64_t R,
                                                         const float2* M, double2 w, int accumulate, int* status) {
    __shared__ uint64_t bar;
    __shared__ uint32_t taddr_s;
    if ((threadIdx.x >> 5) == 0) tc_alloc(&taddr_s, kTcCols);
    if (threadIdx.x == 0) {
        tc_mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = taddr_s;
    uint32_t phase = 0;
    const int err = tc_mode_prod<256>(out, in, L, n, R, M, w, accumulate != 0, dyn_smem, kTcStage, taddr, &bar, phase,
                                      blockIdx.x, gridDim.x);
    if (err && threadIdx.x == 0) atomicExch(status, 5);
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc_dealloc(taddr, kTcCols);
}

__global__ void __launch_bounds__(256, 1) ffma_mode_kernel(float2* out, const float2* in, int64_t L, int n,
                                                           int64_t R, const float2* M, double2 w, int accumulate) {
    if (threadIdx.x == 0) { s_flops = 0.0; s_flops64 = 0.0; s_count = 1; }
    for (int i = threadIdx.x; i <= TTN_MAXCHI; i += 256) s_mpv[i] = 0;
    __syncthreads();
    mode_prod(out, in, L, n, n, R, M, false, w, accumulate != 0, Solo<256>());
}

int tc_init() {
    static std::mutex mu;
    static bool done[256] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 256) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return 0;
    e = cudaFuncSetAttribute(tc_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcStage);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(ffma_mode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBytes);
    if (e != cudaSuccess) return (int)e;
    done[dev] = true;
    return 0;
}

}  // namespace

int ttn_launch_mode_product(int tensor_cores, int64_t L, int n, int64_t R, const void* M, const void* x, void* y,
                            double wr, double wi, int accumulate, int* d_status, cudaStream_t s) {
    int e = tc_init();
    if (e) return e;
    if (tensor_cores) {
        if (n < 1 || n > tc_max_dim()) return (int)cudaErrorInvalidValue;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t tiles = (L * R + kTcRows - 1) / kTcRows;
        const int grid = (int)(tiles < sms ? tiles : sms);
        tc_mode_kernel<<<grid, 256, kTcStage, s>>>((float2*)y, (const float2*)x, L, n, R, (const float2*)M,
                                                   make_double2(wr, wi), accumulate, d_status);
    } else {
        ffma_mode_kernel<<<1, 256, kStageBytes, s>>>((float2*)y, (const float2*)x, L, n, R, (const float2*)M,
                                                     make_double2(wr, wi), accumulate);
    }
    return (int)cudaGetLastError();
}
