// Device program format shared by the host planner (ttn_plan.cpp) and the
// device interpreter (ttn_kernels.cu).
//
// A sweep is compiled on the host into a flat list of operations on one
// instance's device arena.  Every operand is an absolute device pointer, so
// the interpreter does no address arithmetic beyond tensor indexing.
//
// Operators are "sums of product entries": each entry carries a complex
// weight and, per tensor index ("mode"), the id of a square matrix slot or
// -1 for the identity.  The same format expresses
//   * the effective Hamiltonian of a node  sum_e w_e (x_j M_ej) A  (paper
//     Eq. psi_eom_1 after term grouping),
//   * the bond operator  sum_e w_e h_e C H_e^T  (a node with two modes),
//   * environment builds  out_e += w_e * Q^dag (x_{j != keep} M_ej) Q, and
//   * linear combinations of matrices (combos).
#pragma once
#include <stdint.h>

#define TTN_MAXD 8      // tensor modes per node (children + parent)
#define TTN_KMAX 32     // maximal Krylov dimension
#define TTN_MAXCHI 64   // largest bond / local dimension
#define TTN_MAX_SETS 64 // largest set count of a multi-set state

enum TtnOpType : int {
    TTN_OP_QR_DOWN = 1,      // A (a) = Q x_k R^T ;  bond buffer (b) <- R^T      (C[n_spf, m_shf])
    TTN_OP_QR_UP = 2,        // A (a) = Q x_last R;  bond buffer (b) <- R
    TTN_OP_ABSORB_CHILD = 3, // A (a) <- A x_last B^T   with B = bond buffer (b)
    TTN_OP_ABSORB_PARENT = 4,// A (a) <- B x_k A
    TTN_OP_ENV = 5,          // out slots of entries += w * Q^dag (x_{j!=k} M_j) P   (Q = a, P = c or a, keep mode k)
    TTN_OP_COMBO = 6,        // out slot of entries = sum w * M (slot[0] = -1: identity)
    TTN_OP_EVOLVE = 7,       // a <- exp(-i tau H) a, tau = tau_coef * dt, H = entries
    TTN_OP_DOT = 8,          // out scalar <- <a, H a> (ne > 0) or <a, a> (ne == 0)
    TTN_OP_TRACE = 9,        // out scalar <- sum_ab slot0[a,b] * slot1[b,a]   (k = dim)
    TTN_OP_CONTRACT_VEC = 10,// a' <- contraction of tensor a with matrices on modes (vacuum projection)
    TTN_OP_STEP_END = 11,    // end of one time step (timestamp, step counter)
    TTN_OP_SPAWN = 12,       // subspace expansion test of the bond to child k (centre at a)
    TTN_OP_EIGEN = 13,       // a <- lowest eigenvector of H (entries, Hermitian), normalised; out <- eigenvalue
    TTN_OP_PHASE = 14        // a <- exp(-i tau_coef dt) a   (global phase of an energy shift)
};

// Status word value left by a SPAWN op that accepted new single-particle
// functions: the program stops so that the host can grow the bond.
#define TTN_STATUS_SPAWN_HIT 100
// Status word value of a SPAWN op whose bond has more up channels (or a
// larger channel space K = channels x bond dimension) than its workspace.
#define TTN_STATUS_SPAWN_SPACE 7
// Functions one growth may add to a bond: every accepted one up to the cap
// chi_max (Sec. II.D), so at most the largest bond dimension.
#define TTN_SPAWN_MAX_NEW TTN_MAXCHI
// Largest channel count and channel space K of one bond in a SPAWN op.
#define TTN_SPAWN_MAX_CHANNELS 32
#define TTN_SPAWN_MAX_K 512

struct TtnEntry {
    double wr, wi;          // complex weight
    int out;                // output slot (ENV, COMBO) or -1
    int slot[TTN_MAXD];     // factor slot per mode, -1 = identity
    // Multi-set operators (EVOLVE / DOT with nset > 1): the entry reads set
    // block `src` of its input and adds into set block `dst` of its output
    // (the set pair |dst><src| of the term, paper Sec. II.A multi-set ansatz).
    int src, dst;
};

struct TtnSlot {
    void* ptr;              // device pointer to a dim x dim row-major complex matrix
                            // (rows x cols for CONTRACT_VEC factors)
    int rows, cols;
};

struct TtnOp {
    int type;
    int D;                  // number of modes of tensor a
    int dims[TTN_MAXD];     // mode dimensions of tensor a
    int k;                  // mode argument
    int e0, ne;             // entry range
    int hermitian;          // EVOLVE: Lanczos (1) or Arnoldi (0)
    int nset;               // EVOLVE / DOT / PHASE: set blocks of tensor a (0 or 1: one)
    double tau_coef;        // EVOLVE
    void* a;                // main operand
    void* b;                // bond buffer / second operand / output tensor
    double* out;            // DOT / TRACE: complex scalar output (2 doubles)
    // ENV: the ket tensor when it differs from the bra tensor a (multi-set
    // cross-set environments), else null.
    // SPAWN: the child tensor, its index dimensions (children / physical, then
    // the bond), and the entry ranges of the child's up channels (e0/ne), of
    // the down channels of the bond built at this node (e1/ne1) and of the
    // ungrouped bond terms (e2/ne2: slot[0] up channel, slot[1] down channel)
    void* c;
    int Dc;
    int dimsc[TTN_MAXD];
    int e1, ne1, e2, ne2;
    int node, child;
};

struct TtnInstance {
    const TtnOp* ops;
    int n_ops;              // ops of one time step (or of one observable program)
    int n_slots;
    const TtnEntry* entries;
    const TtnSlot* slots;
    void* work;             // workspace: (KMAX+1) Krylov vectors + 4 scratch tensors
    int64_t smax;           // length (complex elements) of each workspace vector
    int* status;            // device status word (0 = ok, else ttn_status code)
    int* steps_done;        // device step counter
    unsigned long long* stamps;  // optional per-step completion time stamps (ns)
    double* flops;          // algorithmic flop counters: [0] all, [1] the FP64 part (block thread 0)
    unsigned long long* op_cycles;  // SM clock cycles spent per op type (16 counters)
    double ktol;
    double qtol;            // QR rank threshold relative to ||M||_F
    int kmax;
    int chi_max;            // SPAWN: bond-dimension cap
    double spawn_eps;       // SPAWN: accept dt * sigma >= spawn_eps
    double spawn_dt;
    double* spawn_out;      // SPAWN result: [node, child, p, NJ, sigma_1..p] then p vectors of NJ complex128
    void* spawn_ws;         // SPAWN FP64 workspace: one tensor copy + 6 dense K x K matrices
    int spawn_kmax;         // largest K the workspace holds
    int nrep;               // steps this launch when the launch asks for per-instance counts
    double dt;              // time step for the same case
    // Mode-product routine per dimension n (index n, 0..TTN_MAXCHI):
    // 0 = default (register fibre up to 32 in complex64 / 16 in complex128,
    // staged above), 1 = staged, 2 = tensor cores (complex64 bulk, where the
    // operands fit the staging area; else staged).  Chosen by ttn_autotune.
    unsigned char mp_variant[TTN_MAXCHI + 1];
    int use_tc;             // some entry of mp_variant is 2: hold tensor memory
};

// Launch parameters read from device memory (so one captured launch can be
// replayed with a different instance count and time slice).
struct TtnLaunchHdr {
    int n;                  // instances in the table
    int pad;
    long long slice_ns;     // device time per block, 0 = unlimited
};

// What one block reports after a launch that asked for it: whole steps run,
// the instance's status word, and the block's device time (globaltimer ns).
struct TtnRepOut {
    int reps;
    int status;
    long long elapsed_ns;
};
