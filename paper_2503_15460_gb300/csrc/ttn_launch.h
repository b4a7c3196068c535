// Launch wrappers exported by the device translation units to the host library.
#pragma once
#include <cuda_runtime.h>

#include "ttn_program.h"

// Largest thread-block cluster one instance may use (non-portable size,
// enabled per kernel).
#define TTN_MAX_CLUSTER 16

// Run the op list of each instance nrep times.  cluster <= 1: one thread
// block (256 threads) per instance; cluster = 2..16: one thread-block
// cluster of that many blocks (512 threads each) per instance.
// precision: 0 = complex128, 1 = complex64 bulk.  tc = 1 (complex64 only)
// launches the build that carries the tcgen05 mode product (instances whose
// variant table asks for tensor cores); with tc = 0 such dimensions take
// the staged FFMA routine.  Returns a cudaError_t code.
int ttn_launch_program(int precision, int cluster, const TtnInstance* d_insts, int n_inst, double dt, int nrep,
                       cudaStream_t stream, int tc = 0);

// General form: `n_inst` instances (grid n_inst x cluster blocks).  With
// d_hdr (device memory) the first d_hdr->n instances run and
// d_hdr->slice_ns replaces slice_ns; without it all `n_inst` run.  nrep < 0
// takes each instance's own step count and time step (TtnInstance::nrep,
// ::dt).  slice_ns > 0 ends an instance after the step that uses up its
// slice of device time.  d_rep_out (optional, `n_inst` entries) receives
// what each instance did.
int ttn_launch_program_ex(int precision, int cluster, const TtnInstance* d_insts, const TtnLaunchHdr* d_hdr,
                          int n_inst, double dt, int nrep, long long slice_ns, TtnRepOut* d_rep_out,
                          cudaStream_t stream, int tc = 0);

// Set the kernel attributes of every variant on the current device (call
// before capturing a launch into a CUDA graph).  Returns a cudaError_t code.
int ttn_program_init();

// How many clusters of `cluster` blocks the cluster kernel of `precision`
// can keep resident at once on the current device (0 if none).
int ttn_cluster_capacity(int precision, int cluster, int* max_active);

// Apply a sum-of-products operator (entries, factor slots) to the complex128
// tensor x (dims[0..D-1]) into y with one thread block; t1..t3 are scratch
// tensors of prod(dims) complex128 elements each.  Returns a cudaError_t code.
int ttn_launch_heff(const TtnEntry* d_entries, int ne, const TtnSlot* d_slots, int D, const int* dims,
                    const void* x, void* y, void* t1, void* t2, void* t3, cudaStream_t stream);

// Limits of the allocation-free effective-Hamiltonian entry point: tensor
// elements, terms and matrices, and the size of its static device scratch.
#define TTN_NOALLOC_MAX_ELEMS 32768
#define TTN_NOALLOC_MAX_TERMS 512
#define TTN_NOALLOC_MAX_MATS 512
#define TTN_NOALLOC_SCRATCH_BYTES \
    (3 * TTN_NOALLOC_MAX_ELEMS * 16 + TTN_NOALLOC_MAX_TERMS * sizeof(TtnEntry) + TTN_NOALLOC_MAX_MATS * sizeof(TtnSlot))

// Same as ttn_launch_heff with the scratch and the term tables in the static
// device array (host tables are copied into it on `stream`).
int ttn_launch_heff_noalloc(const TtnEntry* h_entries, int ne, const TtnSlot* h_slots, int n_slots, int D,
                            const int* dims, const void* x, void* y, cudaStream_t stream);

// FP32 / FP64 fused multiply-add throughput of the current device: `iters`
// iterations of 8 independent FMA chains per thread, 4 blocks of 256
// threads per SM; TFLOP/s and the kernel's time (CUDA events on stream).
int ttn_pipe_peak_fp32(int iters, double* tflops, double* ms, cudaStream_t stream);
int ttn_pipe_peak_fp64(int iters, double* tflops, double* ms, cudaStream_t stream);

// One complex64 mode product y[l, p, r] (+)= w sum_m M[p, m] x[l, m, r]
// (device pointers, interleaved float pairs): tensor_cores = 1 on tcgen05
// with 3xTF32 split products (n <= 64, one block per SM over the fibre
// tiles), 0 by the sweep's FFMA routine (one block).  d_status (device int)
// receives 5 if an MMA did not complete in time.
int ttn_launch_mode_product(int tensor_cores, int64_t L, int n, int64_t R, const void* M, const void* x, void* y,
                            double wr, double wi, int accumulate, int* d_status, cudaStream_t stream);

// ---- internal: one entry point per kernel variant (own translation unit) ----
struct TtnVariantArgs {
    const TtnInstance* insts;
    const TtnLaunchHdr* hdr;
    int n_inst;
    int cluster;
    double dt;
    int nrep;
    long long slice_ns;
    TtnRepOut* rep_out;
    cudaStream_t stream;
};
int ttn_variant_f64_solo(const TtnVariantArgs& a);
int ttn_variant_mix_solo(const TtnVariantArgs& a);
int ttn_variant_f64_clu(const TtnVariantArgs& a);
int ttn_variant_mix_clu(const TtnVariantArgs& a);
// attribute set-up (init) and cluster occupancy (capacity) of one variant
int ttn_variant_f64_solo_init();
int ttn_variant_mix_solo_init();
int ttn_variant_f64_clu_init();
int ttn_variant_mix_clu_init();
int ttn_variant_f64_clu_capacity(int cluster, int* max_active);
int ttn_variant_mix_clu_capacity(int cluster, int* max_active);
// the complex64 builds with the tcgen05 mode product
int ttn_variant_mix_solo_tc(const TtnVariantArgs& a);
int ttn_variant_mix_clu_tc(const TtnVariantArgs& a);
int ttn_variant_mix_solo_tc_init();
int ttn_variant_mix_clu_tc_init();
