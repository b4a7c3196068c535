// Launch wrappers exported by ttn_kernels.cu to the host library.
#pragma once
#include <cuda_runtime.h>

#include "ttn_program.h"

// Run the op list of each instance (one thread block per instance) nrep times.
// precision: 0 = complex128, 1 = complex64 bulk.  Returns a cudaError_t code.
int ttn_launch_program(int precision, const TtnInstance* d_insts, int n_inst, double dt, int nrep,
                       cudaStream_t stream);

// Apply a sum-of-products operator (entries, factor slots) to the complex128
// tensor x (dims[0..D-1]) into y with one thread block; t1..t3 are scratch
// tensors of prod(dims) complex128 elements each.  Returns a cudaError_t code.
int ttn_launch_heff(const TtnEntry* d_entries, int ne, const TtnSlot* d_slots, int D, const int* dims,
                    const void* x, void* y, void* t1, void* t2, void* t3, cudaStream_t stream);
