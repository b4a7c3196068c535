// Launch code of one interpreter variant (included by the per-variant
// translation units, which compile in parallel).
#pragma once
#include <mutex>

#include "ttn_device.cuh"
#include "ttn_launch.h"

namespace {

// Kernel attributes are per device: set them once for each device, under a
// lock, and remember a device only after every call succeeded.
template <class TS, class TB, class TM>
int variant_init() {
    static std::mutex mu;
    static bool done[256] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 256) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return 0;
    auto k = program_kernel<TS, TB, TM>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, TM::wide ? kStageBytesClu : kStageBytes);
    if (e == cudaSuccess && TM::wide) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return (int)e;
    done[dev] = true;
    return 0;
}

template <class TS, class TB, class TM>
int variant_launch(const TtnVariantArgs& a) {
    if (a.n_inst <= 0) return 0;
    int e = variant_init<TS, TB, TM>();
    if (e) return e;
    auto k = program_kernel<TS, TB, TM>;
    if constexpr (!TM::wide) {
        k<<<a.n_inst, TM::NT, kStageBytes, a.stream>>>(a.insts, a.hdr, a.n_inst, a.dt, a.nrep, a.slice_ns, a.rep_out);
    } else {
        if (a.cluster < 1 || a.cluster > TTN_MAX_CLUSTER) return (int)cudaErrorInvalidValue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(a.n_inst * a.cluster), 1, 1);
        cfg.blockDim = dim3(TM::NT, 1, 1);
        cfg.dynamicSmemBytes = kStageBytesClu;
        cfg.stream = a.stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)a.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t r = cudaLaunchKernelEx(&cfg, k, a.insts, a.hdr, a.n_inst, a.dt, a.nrep, a.slice_ns, a.rep_out);
        if (r != cudaSuccess) return (int)r;
    }
    return (int)cudaGetLastError();
}

template <class TS, class TB>
int variant_capacity(int cluster, int* max_active) {
    *max_active = 0;
    if (cluster < 1 || cluster > TTN_MAX_CLUSTER) return (int)cudaErrorInvalidValue;
    int e = variant_init<TS, TB, Clu>();
    if (e) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3(Clu::NT, 1, 1);
    cfg.dynamicSmemBytes = kStageBytesClu;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return (int)cudaOccupancyMaxActiveClusters(max_active, program_kernel<TS, TB, Clu>, &cfg);
}

}  // namespace
