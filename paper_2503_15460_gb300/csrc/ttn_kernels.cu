// libttn launch dispatch, the kernel-level effective-Hamiltonian entry
// point and its allocation-free variant.  The sweep interpreter itself is in
// ttn_device.cuh, compiled once per variant (ttn_var_*.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ttn_device.cuh"
#include "ttn_launch.h"

namespace {

// One thread block applies a sum-of-products operator to one tensor (the
// same device routine the sweep runs inside its Krylov exponentials).
__global__ void __launch_bounds__(256, 1) heff_kernel(const TtnEntry* es, int ne, const TtnSlot* slots, Shape sh,
                                                      const double2* x, double2* y, double2* t1, double2* t2,
                                                      double2* t3) {
    if (threadIdx.x == 0) { s_flops = 0.0; s_flops64 = 0.0; s_count = 1; }
    for (int i = threadIdx.x; i <= TTN_MAXCHI; i += 256) s_mpv[i] = 0;
    __syncthreads();
    heff_apply(y, x, t1, t2, t3, sh, es, ne, slots, Solo<256>());
}

// The dynamic shared-memory attribute is per device: set once per device,
// under a lock, remembered only after it succeeded.
int heff_init() {
    static std::mutex mu;
    static bool done[256] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 256) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return 0;
    e = cudaFuncSetAttribute(heff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBytes);
    if (e != cudaSuccess) return (int)e;
    done[dev] = true;
    return 0;
}

}  // namespace

int ttn_launch_heff(const TtnEntry* d_entries, int ne, const TtnSlot* d_slots, int D, const int* dims,
                    const void* x, void* y, void* t1, void* t2, void* t3, cudaStream_t s) {
    int e = heff_init();
    if (e) return e;
    Shape sh;
    sh.D = D;
    for (int j = 0; j < TTN_MAXD; ++j) sh.d[j] = j < D ? dims[j] : 1;
    heff_kernel<<<1, 256, kStageBytes, s>>>(d_entries, ne, d_slots, sh, (const double2*)x, (double2*)y,
                                            (double2*)t1, (double2*)t2, (double2*)t3);
    return (int)cudaGetLastError();
}

int ttn_program_init() {
    int e = ttn_variant_f64_solo_init();
    if (!e) e = ttn_variant_mix_solo_init();
    if (!e) e = ttn_variant_f64_clu_init();
    if (!e) e = ttn_variant_mix_clu_init();
    if (!e) e = ttn_variant_mix_solo_tc_init();
    if (!e) e = ttn_variant_mix_clu_tc_init();
    return e;
}

int ttn_cluster_capacity(int precision, int cluster, int* max_active) {
    return precision == 0 ? ttn_variant_f64_clu_capacity(cluster, max_active)
                          : ttn_variant_mix_clu_capacity(cluster, max_active);
}

int ttn_launch_program(int precision, int cluster, const TtnInstance* d_insts, int n_inst, double dt, int nrep,
                       cudaStream_t s, int tc) {
    return ttn_launch_program_ex(precision, cluster, d_insts, nullptr, n_inst, dt, nrep, 0, nullptr, s, tc);
}

int ttn_launch_program_ex(int precision, int cluster, const TtnInstance* d_insts, const TtnLaunchHdr* d_hdr,
                          int n_inst, double dt, int nrep, long long slice_ns, TtnRepOut* d_rep_out, cudaStream_t s,
                          int tc) {
    if (n_inst <= 0) return 0;
    TtnVariantArgs a{d_insts, d_hdr, n_inst, cluster, dt, nrep, slice_ns, d_rep_out, s};
    if (precision == 0) return cluster <= 1 ? ttn_variant_f64_solo(a) : ttn_variant_f64_clu(a);
    if (tc) return cluster <= 1 ? ttn_variant_mix_solo_tc(a) : ttn_variant_mix_clu_tc(a);
    return cluster <= 1 ? ttn_variant_mix_solo(a) : ttn_variant_mix_clu(a);
}

// ---------------------------------------------------------------------------
// Allocation-free effective-Hamiltonian application.
//
// Some callers must not allocate device memory while they run -- for example
// a serving loop that has handed all of the GPU's memory to its own pool
// allocator, or code that must not trigger the device-wide synchronisation
// that cudaMalloc / cudaFree can imply.  For them the scratch of the
// effective-Hamiltonian kernel (three tensors plus the term tables) lives in
// one file-scope device array of fixed size instead of being allocated per
// call.  Every GPU that loads the library keeps this array for the life of
// the process.  All calls share it: calls whose work overlaps on the GPU
// (different streams, different host threads) race on it and must be
// serialised by the caller.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_heff_scratch[TTN_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mutex;
void* g_scratch_addr[64] = {nullptr};
}  // namespace

// Device address of the static scratch on the current device.  In host code
// g_heff_scratch only names a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.
int ttn_noalloc_scratch(void** ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* a = nullptr;
        e = cudaGetSymbolAddress(&a, g_heff_scratch);
        if (e != cudaSuccess) return (int)e;
        g_scratch_addr[dev] = a;
    }
    *ptr = g_scratch_addr[dev];
    return 0;
}

int ttn_launch_heff_noalloc(const TtnEntry* h_entries, int ne, const TtnSlot* h_slots, int n_slots, int D,
                            const int* dims, const void* x, void* y, cudaStream_t s) {
    void* base = nullptr;
    int rc = ttn_noalloc_scratch(&base);
    if (rc) return rc;
    char* b = (char*)base;
    // layout: [3 tensors][entries][slot table]
    char* t1 = b;
    char* t2 = t1 + TTN_NOALLOC_MAX_ELEMS * 16;
    char* t3 = t2 + TTN_NOALLOC_MAX_ELEMS * 16;
    char* de = t3 + TTN_NOALLOC_MAX_ELEMS * 16;
    char* ds = de + TTN_NOALLOC_MAX_TERMS * sizeof(TtnEntry);
    cudaError_t e = cudaMemcpyAsync(de, h_entries, (size_t)ne * sizeof(TtnEntry), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ds, h_slots, (size_t)n_slots * sizeof(TtnSlot), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return (int)e;
    return ttn_launch_heff((const TtnEntry*)de, ne, (const TtnSlot*)ds, D, dims, x, y, t1, t2, t3, s);
}
