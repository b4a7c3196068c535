// Launch wrappers exported by ttn_kernels.cu to the host library.
#pragma once
#include <cuda_runtime.h>

#include "ttn_program.h"

// Run the op list of each instance (one thread block per instance) nrep times.
// precision: 0 = complex128, 1 = complex64 bulk.  Returns a cudaError_t code.
int ttn_launch_program(int precision, const TtnInstance* d_insts, int n_inst, double dt, int nrep,
                       cudaStream_t stream);

// General form: `grid` blocks.  With d_hdr (device memory) the first
// d_hdr->n blocks run and d_hdr->slice_ns replaces slice_ns; without it all
// `grid` blocks run.  nrep < 0 takes each instance's own step count and
// time step (TtnInstance::nrep, ::dt).  slice_ns > 0 ends a block after the
// step that uses up its slice of device time.  d_rep_out (optional, `grid`
// entries) receives what each block did.
int ttn_launch_program_ex(int precision, const TtnInstance* d_insts, const TtnLaunchHdr* d_hdr, int grid, double dt,
                          int nrep, long long slice_ns, TtnRepOut* d_rep_out, cudaStream_t stream);

// Set the kernel attributes once per process (call before capturing a
// launch into a CUDA graph).  Returns a cudaError_t code.
int ttn_program_init();

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
