// Launch wrappers exported by ttn_kernels.cu to the host library.
#pragma once
#include <cuda_runtime.h>

#include "ttn_program.h"

// Run the op list of each instance (one thread block per instance) nrep times.
// precision: 0 = complex128, 1 = complex64 bulk.  Returns a cudaError_t code.
int ttn_launch_program(int precision, const TtnInstance* d_insts, int n_inst, double dt, int nrep,
                       cudaStream_t stream);
