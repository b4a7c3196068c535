// Internal view of a context, shared by the C ABI (ttn_api.cpp) and the
// request server (ttn_server.cpp).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ttn.h"
#include "ttn_plan.hpp"

namespace ttn {

struct DevProgram {
    TtnOp* d_ops = nullptr;
    int n_ops = 0;
};

}  // namespace ttn

struct ttn_ctx {
    int precision = 0;
    ttn::Tree tree;
    ttn::Hamiltonian ham;
    bool has_h = false;
    ttn::Plan plan;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    bool failed = false;

    // Residency.  A resident context holds its arenas and tensors on the
    // device; a host-resident one keeps the tensors in host_A and holds no
    // device memory.  Pooled contexts take their arenas from the
    // stream-ordered allocator (cudaMallocAsync on `stream`).
    bool resident = true;
    bool pooled = false;
    std::vector<std::vector<ttn::cplx>> host_A;
    int64_t saved_steps = 0;
    double saved_flops = 0.0;
    double saved_flops64 = 0.0;

    char* d_state = nullptr;       // tensors, bond, workspace, status, scalars, stamps
    size_t state_bytes = 0;
    char* d_ops = nullptr;         // slot storage, slot table, entries, op lists, instances
    size_t ops_bytes = 0;
    TtnSlot* d_slots = nullptr;
    TtnEntry* d_entries = nullptr;
    ttn::DevProgram init_p, step_p, ne_p, spawn_p, ground_p, setpop_p;
    std::vector<ttn::DevProgram> rdm_p, vac_p, to_root_p;
    TtnInstance* d_inst = nullptr; // staging for single-instance launches
    TtnInstance* d_batch = nullptr;
    int batch_cap = 0;
    double ktol = 0.0;
    double qtol = 0.0;
    int kmax = TTN_KMAX;
    // The SOP as last given to ttn_set_sop_hamiltonian (ttn_set_coefficients
    // replays it with new coefficients).
    std::vector<ttn::cplx> sop_coeff, sop_mats;
    std::vector<int> sop_ptr, sop_leaf;
    std::vector<int64_t> sop_off;
    int sop_herm = 1;
    // multi-set operator as last given (ttn_set_multiset_hamiltonian)
    int sop_nsets = 1;
    std::vector<int> sop_bra, sop_ket;
    int64_t steps_total = 0;
    int64_t spawned = 0;            // single-particle functions added by expansion
    // Thread blocks per instance: 0 = chosen from the plan, 1 = one block,
    // 2..16 = a thread-block cluster of that size.
    int cluster_req = 0;
    // Mode-product routine per dimension (TtnInstance::mp_variant), and the
    // autotuner's record: step time of the chosen configuration and of the
    // default one (ms), candidates timed.
    unsigned char mp_variant[TTN_MAXCHI + 1] = {0};
    double tune_ms = 0.0, tune_default_ms = 0.0;
    int tune_trials = 0;
};

namespace ttn {

// Device descriptor of one of the context's programs (resident contexts).
TtnInstance make_instance(ttn_ctx* c, const DevProgram& p);
// Largest tensor index dimension one thread block handles (the Gram
// contraction keeps a 2 x 2 block of a dim x dim result per thread, twice).
constexpr int kSoloMaxDim = 45;
// Thread blocks one instance of c runs on: the caller's choice, else one
// block per 4096 elements of the largest node tensor (a power of two, at
// most 16); at least 2 when an index dimension exceeds kSoloMaxDim.
int ctx_cluster(const ttn_ctx* c);
// Some dimension of c's variant table asks for the tcgen05 mode product
// (complex64 only): its launches take the build that carries it.
bool ctx_uses_tc(const ttn_ctx* c);
// Record a failure on c (or, for c == NULL, for ttn_last_error(NULL)).
ttn_status ctx_fail(ttn_ctx* c, ttn_status s, const std::string& msg);
// Bytes ctx_materialize allocates for the current plan.
size_t ctx_footprint(const ttn_ctx* c);
// Allocate the arenas, upload operators and tensors, build environments.
ttn_status ctx_materialize(ttn_ctx* c);
// Copy the tensors and counters to the host and release the arenas.
ttn_status ctx_evict(ttn_ctx* c);

}  // namespace ttn
