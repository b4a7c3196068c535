// Host-side planning for libttn: tree bookkeeping, grouping of the
// sum-of-product Hamiltonian into per-node operator entries, the device
// arena layout and the sweep programs.  Plain C++, no CUDA types.
#pragma once
#include <complex>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "ttn_program.h"

namespace ttn {

using cplx = std::complex<double>;
using Key = std::vector<std::pair<int, int>>;   // sorted (leaf, matrix id) pairs

struct Tree {
    int n = 0;
    std::vector<int> parent, phys, bond;
    std::vector<std::vector<int>> ch;      // children in index order
    std::vector<std::vector<int>> dims;    // tensor mode dimensions per node
    std::vector<int64_t> size;             // elements per node tensor
    std::vector<int> tin, tout;            // Euler-tour interval of each subtree
    bool leaf(int z) const { return phys[z] > 0; }
    bool in_sub(int x, int c) const { return tin[c] <= tin[x] && tin[x] < tout[c]; }
    std::vector<int> preorder() const;
    std::vector<int> postorder() const;
};

// Validate and build; returns "" on success or an error message.
std::string build_tree(int n, const int* parent, const int* phys, const int* bond, Tree& t);

struct Hamiltonian {
    std::vector<cplx> coeff;
    std::vector<Key> terms;                 // per term, factors sorted by leaf
    std::vector<std::vector<cplx>> mats;    // distinct factor matrices (row-major d x d)
    std::vector<int> mat_dim;
    bool hermitian = true;
    // Multi-set operator (paper Sec. II.A, multi-set ansatz): term r is
    // c_r |bra[r]><ket[r]| (x) (its factors); n_sets = 1 (bra, ket empty)
    // for the single-set SOP.
    int n_sets = 1;
    std::vector<int> bra, ket;
};

std::string build_hamiltonian(const Tree& t, int n_terms, const cplx* coeff, const int* term_ptr,
                              const int* factor_leaf, const cplx* mats, const int64_t* mat_off,
                              int hermitian, Hamiltonian& h, int n_sets = 1, const int* bra = nullptr,
                              const int* ket = nullptr);

// Device-side storage kinds.  Offsets are in bytes from the arena base.
struct SlotInfo {
    int rows = 0, cols = 0;
    bool constant = false;          // uploaded once (physical factors)
    std::vector<cplx> data;         // constant contents
    int64_t off = 0;
};

// An operation before linking: a/b/out hold arena byte offsets, or -1.
struct OpSpec {
    TtnOp op;
    int64_t a_off = -1, b_off = -1, out_off = -1, c_off = -1;   // c_off: ENV ket tensor
};

struct Program {
    std::vector<OpSpec> ops;
};

struct Plan {
    // arena layout (bytes)
    size_t esz = 16;                 // bytes per complex element of the bulk type (slots, Krylov)
    size_t esz_state = 16;           // bytes per element of node tensors / bond buffer (complex128)
    // Set blocks per node tensor (multi-set state, paper Sec. II.A): node z
    // holds nset tensors of t.size[z] elements back to back at tensor_off[z]
    // (set 0 first); the bond buffer holds nset bond matrices of the bond
    // being moved, each bond x bond, back to back.
    int nset = 1;
    std::vector<int64_t> tensor_off;
    int64_t bond_off = 0, work_off = 0, status_off = 0, steps_off = 0, stamps_off = 0, scal_off = 0, flops_off = 0, cycles_off = 0;
    int64_t smax = 0;                // elements per workspace vector
    // Energy shift of the complex64 path: the Hermitian local operator of
    // every leaf is stored minus its smallest eigenvalue (Sum of them =
    // e_shift), so the bulk arithmetic works on excitation energies; the
    // step ends with the global phase exp(-i e_shift dt) and energies are
    // reported with e_shift added.  Zero in complex128 and for generators
    // that are not Hermitian.
    double e_shift = 0.0;
    // Channels crossing each bond (entries of the bond operator: pairs of
    // single-particle and mean-field operators), index = child node.
    std::vector<int> op_bond_dim;
    int max_stamps = 0;
    int64_t total_bytes = 0;
    int max_chi = 1;

    std::vector<SlotInfo> slots;
    std::vector<TtnEntry> entries;

    Program init_prog;               // environment build after a state / Hamiltonian change
    Program step_prog;               // one time step
    Program spawn_prog;              // subspace-expansion pass (stops at the first bond that grows)
    Program ground_prog;             // one ground-state sweep (one-site tree DMRG), Hermitian H only
    std::vector<Program> to_root_prog;   // per node: move the orthogonality centre from it to the root
    int64_t spawn_out_off = 0;       // bytes: spawn result area
    int64_t spawn_out_bytes = 0;
    int64_t spawn_ws_off = 0;        // bytes: FP64 spawn workspace (a tensor + 6 K x K matrices)
    int spawn_kmax = 0;
    // observables
    Program norm_energy_prog;        // out scalars 0: <A,A>, 1: <A,HA>
    Program setpop_prog;             // multi-set: <A^a, A^a> of every set's root block at setpop_off + 16 a
    int64_t setpop_off = 0;
    std::vector<Program> rdm_prog;   // per leaf: gram walk + reduced density (slot rdm_slot[leaf])
    std::vector<int> rdm_slot;
    std::vector<Program> vac_prog;   // per leaf kept: vacuum projection, result vector slot vac_slot[leaf]
    std::vector<int> vac_slot;
};

// Build the complete plan (layout + programs) for a tree and, if h != nullptr,
// a Hamiltonian.  precision: TTN_FP64 (0) or TTN_MIXED (1).
// With h->n_sets > 1 the plan is that of a multi-set state (nset = n_sets):
// no expansion, ground-state, reduced-density or vacuum programs.
std::string make_plan(const Tree& t, const Hamiltonian* h, int precision, Plan& plan);

// Deterministic product state tensors (row-major per node) for leaf vectors.
void product_state(const Tree& t, const std::vector<std::vector<cplx>>& leaf_vecs,
                   std::vector<std::vector<cplx>>& tensors);

}  // namespace ttn
