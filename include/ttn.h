/*
 * libttn -- tree tensor network (ML-MCTDH) time evolution on one GB300 GPU.
 *
 * C ABI.  Plain pointers and sizes only; no exceptions cross it.
 *
 * The state is a tree tensor network (paper Sec. II.A, Eqs.
 * wavefunction_expansion_spf, spf_recursion): one coefficient tensor per node,
 * stored row-major with shape [n_1, ..., n_d, N] -- the bond dimensions of the
 * node's children in child order (a leaf has a single physical index of
 * dimension d instead), then the bond to its parent N (the root's N is 1).
 * Complex numbers are interleaved (re, im) doubles.
 *
 * The Hamiltonian is a sum of products (Sec. II.B.1, Eq. sop_ham),
 *     H = sum_r c_r  prod_{f in term r}  M_f  (acting on leaf(f)),
 * with hbar = 1.  Time stepping is the one-site projector-splitting
 * integrator (Sec. II.C, Eq. psi_eom_1): every node tensor is propagated
 * under its effective Hamiltonian, bonds are propagated backwards between
 * node updates, QR factorisations move the orthogonality centre.  One step
 * of length dt is the symmetric composition of a forward and a reverse
 * sweep of length dt/2 each.
 *
 * Ownership: the caller owns every array passed in; the library copies what
 * it keeps before returning, so inputs may be freed on return.  Outputs go
 * to caller-allocated host buffers.  A context owns its device memory
 * (allocated with cudaMalloc on the current device at ttn_create, released
 * by ttn_destroy) and runs its work on the stream given by ttn_set_stream
 * (default: the legacy default stream).
 *
 * Errors: every call returns a ttn_status.  TTN_E_INVALID leaves the context
 * unchanged; a CUDA or device-side failure (TTN_E_CUDA, TTN_E_NOCONV,
 * TTN_E_TIMEOUT) marks the context as failed, after which only ttn_get_state,
 * ttn_last_error and ttn_destroy are meaningful (TTN_E_STATE otherwise).
 * ttn_last_error returns a message describing the most recent failure.
 */
#ifndef TTN_H
#define TTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttn_ctx ttn_ctx;
typedef struct { double re, im; } ttn_c128;

typedef enum {
    TTN_OK = 0,
    TTN_E_INVALID = 1,   /* bad argument; nothing changed                          */
    TTN_E_OOM = 2,       /* device or host allocation failed                       */
    TTN_E_CUDA = 3,      /* a CUDA runtime call failed                              */
    TTN_E_NOCONV = 4,    /* Krylov exponential did not converge after substepping   */
    TTN_E_TIMEOUT = 5,   /* a bounded device-side wait gave up                      */
    TTN_E_STATE = 6      /* call not valid in the context's current state           */
} ttn_status;

/* Arithmetic of the bulk contractions.  TTN_FP64: everything in complex128.
 * TTN_MIXED: effective-Hamiltonian and environment products, Krylov vectors
 * and environment matrices in complex64 with FP32 accumulation; node
 * tensors, the QR gauge steps, Krylov coefficients and Gram-Schmidt
 * reductions, norms and the small projected exponential in FP64. */
enum { TTN_FP64 = 0, TTN_MIXED = 1 };

typedef struct {
    double krylov_tol;   /* stop when Saad's a-posteriori error estimate of the
                            projected exponential is below krylov_tol * ||v||;
                            <= 0 selects 1e-13 (FP64) or 1e-10 (MIXED)           */
    int krylov_maxdim;   /* Krylov dimension before the interval is halved,
                            1..32; <= 0 selects 32                               */
    double eps_spawn;    /* subspace-expansion tolerance eps_S (Sec. II.D): a
                            new single-particle function is added when
                            dt * sqrt(lambda) >= eps_spawn                       */
    int chi_max;         /* bond-dimension cap for expansion (<= 64)             */
    int expand;          /* 0: fixed bond dimensions; 1: before every step, an
                            expansion pass visits the bonds in sweep order with
                            the orthogonality centre on the bond's parent and
                            adds to the child the dominant eigenvectors of the
                            two-site energy-variance operator (1-P) G (1-P_S)
                            that pass the criterion (every one that passes, up
                            to chi_max); after each growth the centre returns
                            to the root and the pass restarts, until a pass
                            adds nothing.  ttn_bond_dims reports the result.
                            A bond whose terms have more than 32 distinct
                            coupling channels, or a channel space (channels x
                            bond dimension) above 512, cannot be tested:
                            TTN_E_INVALID.                                       */
    double qr_rank_tol;  /* a QR column whose remainder has norm <= qr_rank_tol
                            * ||M||_F is treated as zero and completed by the
                            deterministic unit vector (unoccupied function);
                            <= 0 selects 1e-10 (both modes)                      */
} ttn_step_opts;

/* Create a context for a tree (Sec. II.A).
 *   n_nodes   number of nodes, 1..65535.
 *   parent    [n_nodes]; parent[0] = -1 (root), 0 <= parent[i] < i otherwise.
 *             Children of a node are ordered by their index; the sweep visits
 *             them in that order.
 *   phys_dim  [n_nodes]; > 0 for leaves (local dimension of the single
 *             physical mode), 0 for interior nodes.  Leaves have no children,
 *             interior nodes at least one.
 *   bond_dim  [n_nodes]; bond to the parent (ignored for the root).  Every
 *             matricisation used by the sweep must have at least as many rows
 *             as columns: a node's parent bond is at most the product of its
 *             other index dimensions, and so is each child bond.
 *   precision TTN_FP64 or TTN_MIXED.
 * Allocates the context's device memory on the current CUDA device.  The
 * state is the product state with every leaf in basis state 0 (see
 * ttn_set_product_state); there is no Hamiltonian until
 * ttn_set_sop_hamiltonian. */
ttn_status ttn_create(int n_nodes, const int* parent, const int* phys_dim,
                      const int* bond_dim, int precision, ttn_ctx** out);

/* Same as ttn_create, but the context holds no device memory yet: its
 * tensors, Hamiltonian and plan stay on the host until ttn_materialize (or
 * the first call that needs the device, which materialises it).  Device
 * memory of such a context comes from the stream-ordered allocator
 * (cudaMallocAsync on the context's stream).  This is how requests wait in
 * a ttn_server queue without holding device memory. */
ttn_status ttn_create_host(int n_nodes, const int* parent, const int* phys_dim,
                           const int* bond_dim, int precision, ttn_ctx** out);

/* Make the context resident: allocate its arenas (ttn_footprint bytes),
 * upload operators and tensors, and build the environments.  No-op when it
 * is resident.  TTN_E_OOM leaves it on the host, unchanged. */
ttn_status ttn_materialize(ttn_ctx* ctx);

/* Copy the tensors and the step counters to the host and release the
 * context's device memory; device time stamps and cycle counters are
 * dropped.  Any later call that needs the device materialises it again
 * (ttn_get_state, ttn_bond_dims and ttn_step_stats do not). */
ttn_status ttn_evict(ttn_ctx* ctx);

/* Device bytes the context holds when resident (its state arena: tensors,
 * bond buffer, Krylov workspace, counters; and its operator arena: SOP
 * matrices, environments, term tables, op lists), from its plan; valid
 * whether or not it is resident.  Admission by a ttn_server uses it. */
ttn_status ttn_footprint(const ttn_ctx* ctx, size_t* bytes);

/* Set every node tensor.  tensors holds the tensors back to back, node z at
 * tensors[offsets[z] .. offsets[z+1]) (offsets has n_nodes+1 entries; sizes
 * must match the node shapes).  The caller promises canonical gauge with
 * the orthogonality centre at the root: each non-root tensor, matricised as
 * [prod(child dims) x N], has orthonormal columns.  Environments are
 * rebuilt if a Hamiltonian is set. */
ttn_status ttn_set_state(ttn_ctx* ctx, const ttn_c128* tensors, const int64_t* offsets);

/* Product state prod_leaf |v_leaf> (Sec. IV.A: a product state carried with
 * unoccupied single-particle functions).  leaf_vecs[leaf_offsets[z] ..
 * +phys_dim[z]) is the (not necessarily normalised, nonzero) vector of leaf
 * z; leaf_offsets has n_nodes entries, entries of interior nodes are
 * ignored.  Unoccupied functions are fixed deterministically: a leaf's
 * column 0 is v/|v|, further columns are the lowest-index unit vectors made
 * orthogonal to the previous ones (two Gram-Schmidt passes; a remainder of
 * norm < 1/2 is skipped); an interior node's column i is the unit tensor at
 * the i-th child multi-index in row-major order; the root holds a single 1
 * at (0, ..., 0). */
ttn_status ttn_set_product_state(ttn_ctx* ctx, const ttn_c128* leaf_vecs,
                                 const int64_t* leaf_offsets);

/* Sum-of-product Hamiltonian (Sec. II.B.1, Eq. sop_ham).
 *   coeff         [n_terms] c_r.
 *   term_ptr      [n_terms+1] CSR: the factors of term r are
 *                 term_ptr[r] .. term_ptr[r+1]-1 (a term with no factors is
 *                 the constant c_r).
 *   factor_leaf   node id of each factor; must be a leaf, at most one factor
 *                 per leaf and term.
 *   factor_mats / factor_mat_off: the d x d row-major matrix of factor f
 *                 starts at factor_mats[factor_mat_off[f]].
 *   hermitian     1 if H is Hermitian (Lanczos), 0 otherwise (Arnoldi; e.g.
 *                 the HEOM generator of Sec. II.E.3, Eq. fpheom_op).
 * The library groups terms per node (identity factors skipped, terms acting
 * inside one subtree pre-summed, terms that differ in one factor only
 * combined), which is exact, and builds all environments. */
ttn_status ttn_set_sop_hamiltonian(ttn_ctx* ctx, int n_terms, const ttn_c128* coeff,
                                   const int* term_ptr, const int* factor_leaf,
                                   const ttn_c128* factor_mats, const int64_t* factor_mat_off,
                                   int hermitian);

/* Time-dependent coefficients c_r(t) (the paper's interaction-picture and
 * chain mappings of a bath make the SOP coefficients time dependent,
 * Sec. II.E): replace the coefficients of the Hamiltonian last set by
 * ttn_set_sop_hamiltonian, keeping its factors (n_terms must be the same;
 * coefficients may become or stop being zero).  Everything that depends on
 * them -- pre-summed local operators, term weights, environments -- is
 * rebuilt; the state is unchanged.  Holding c(t + dt/2) over a step of
 * ttn_step(dt) (midpoint rule) keeps the step second-order accurate for
 * smooth c(t).  The cost is one host re-plan and one environment build. */
ttn_status ttn_set_coefficients(ttn_ctx* ctx, int n_terms, const ttn_c128* coeff);

/* Multi-set states (Sec. II.A, multi-set ansatz): |Psi> = sum_alpha |alpha>
 * |Psi^alpha> with one TTN per set state alpha (the system state, e.g. an
 * electronic state), all on the context's tree with the same bond
 * dimensions.  The operator is
 *     H = sum_r c_r |bra[r]><ket[r]| (x) prod_{factors of r} M_f
 * given like ttn_set_sop_hamiltonian plus, per term, the set pair
 * bra[r], ket[r] in 0 .. n_sets-1 (1 <= n_sets <= 64).  Every step is the
 * single-set projector-splitting step with all sets' tensors of a node (or
 * bond) propagated together, cross-set environments between the sets'
 * functions (an operator that is the identity on a subtree becomes the
 * overlap of the two sets' functions there when bra != ket), and QR gauge
 * moves done set by set.  A single-set state becomes multi-set here: set 0
 * keeps it, every other set starts empty (set 0's isometries, zero top
 * tensor).  A state with another set count > 1 gives TTN_E_INVALID.
 * ttn_set_coefficients replays the set pairs.  Multi-set contexts support
 * ttn_step (no subspace expansion: the paper leaves it open for this
 * ansatz), ttn_step_batch, the request server, ttn_norm_energy (whole
 * state), ttn_set_populations and the state calls below; the single-set
 * state, density, vacuum-projection and ground-state calls return
 * TTN_E_INVALID.  ttn_save / ttn_load carry multi-set states too (the set
 * count and set pairs with the operator, every set's tensors). */
ttn_status ttn_set_multiset_hamiltonian(ttn_ctx* ctx, int n_sets, int n_terms, const ttn_c128* coeff,
                                        const int* term_ptr, const int* factor_leaf,
                                        const ttn_c128* factor_mats, const int64_t* factor_mat_off,
                                        const int* bra, const int* ket, int hermitian);

/* Set every set's node tensors (after ttn_set_multiset_hamiltonian; n_sets
 * must equal its set count).  The tensor of set alpha, node z is
 * tensors[offsets[alpha*n_nodes + z] .. offsets[alpha*n_nodes + z + 1]);
 * offsets has n_sets*n_nodes+1 entries.  Each set in canonical gauge with
 * its centre at the root (non-root tensors isometric; a set may be empty:
 * zero top tensor).  Environments are rebuilt. */
ttn_status ttn_set_multiset_state(ttn_ctx* ctx, int n_sets, const ttn_c128* tensors, const int64_t* offsets);

/* Copy set alpha's node tensors to the host in the layout of ttn_get_state. */
ttn_status ttn_get_multiset_state(ttn_ctx* ctx, int alpha, ttn_c128* tensors, int64_t* offsets);

/* Populations <Psi^alpha|Psi^alpha> of every set (the squared norm of each
 * set's top tensor, the centre being at the root between steps), computed
 * on the device; pops has n_sets entries (a single-set context gives its
 * squared norm). */
ttn_status ttn_set_populations(ttn_ctx* ctx, double* pops);

/* Set count of the context's state (1 for a single-set state). */
ttn_status ttn_n_sets(const ttn_ctx* ctx, int* n_sets);

/* Checkpoint / resume (the paper has no counterpart: long propagations
 * are resumed from saved states).  ttn_save writes the tree (with the
 * current bond dimensions, which subspace expansion may have grown), the
 * step and flop counters, the Hamiltonian as last given (coefficients,
 * factors, matrices, hermitian flag; for a multi-set state also the set
 * count and every term's set pair) and every node tensor (complex128,
 * centre at the root; all set blocks) into buf, a self-describing byte stream of *len
 * bytes; with buf == NULL it only stores the required size in *len, and a
 * too small *len gives TTN_E_INVALID with the size in *len.  ttn_load
 * replaces the tree, state, Hamiltonian and counters of ctx by those of a
 * checkpoint, keeping ctx's precision and residency (a resident context is
 * re-materialised, environments rebuilt).  Device time stamps and cycle
 * counters are not saved.  A stream that is not a checkpoint, is
 * truncated or inconsistent returns TTN_E_INVALID and leaves ctx
 * unchanged.  Resuming gives bit-identical results to not stopping. */
ttn_status ttn_save(ttn_ctx* ctx, void* buf, size_t* len);
ttn_status ttn_load(ttn_ctx* ctx, const void* buf, size_t len);

/* Advance by nsteps steps of length dt (Sec. II.C).  opts may be NULL
 * (defaults).  Blocks until the device work has finished. */
ttn_status ttn_step(ttn_ctx* ctx, double dt, int nsteps, const ttn_step_opts* opts);

/* Ground state by one-site tree DMRG sweeps (the paper names DMRG beside
 * the time evolution, Sec. I and Sec. II.C; same environments, effective
 * Hamiltonian and gauge moves as ttn_step).  One sweep visits the nodes in
 * the order of the step's forward sweep S: centre moved to each child by
 * QR, recursion, centre moved back, then the node tensor replaced by the
 * normalised lowest eigenvector of its effective Hamiltonian (restarted
 * Lanczos with full reorthogonalisation; residual below 1e-12 relative in
 * TTN_FP64, 1e-7 in TTN_MIXED).  Bond dimensions stay fixed, so the state
 * only explores the span of its current single-particle functions
 * (occupied and unoccupied).  energies[i] (may be NULL) receives the
 * root's eigenvalue after sweep i: the energy <Psi|H|Psi> of the
 * normalised state, non-increasing from sweep to sweep up to the
 * tolerance.  Hermitian Hamiltonians only (TTN_E_INVALID otherwise);
 * TTN_E_NOCONV if an eigen-solve fails to converge in 200 restarts. */
ttn_status ttn_ground_state(ttn_ctx* ctx, int nsweeps, double* energies);

/* Advance n independent contexts (same precision) by nsteps steps of dt in
 * one device launch, one thread block per context; the stream of ctxs[0]
 * is used.  Contexts may have different trees and Hamiltonians.  Fixed bond
 * dimensions only (opts->expand must be 0). */
ttn_status ttn_step_batch(ttn_ctx* const* ctxs, int n, double dt, int nsteps,
                          const ttn_step_opts* opts);

/* Reduced density matrix of a leaf's physical mode, normalised by <Psi|Psi>:
 * rho[a, a'] = <Psi| (|a'><a|) |Psi> / <Psi|Psi>, written row-major to
 * out[d*d]. */
ttn_status ttn_reduced_density(ttn_ctx* ctx, int leaf, ttn_c128* out);

/* <Psi|O|Psi>/<Psi|Psi> for n_obs single-leaf operators: O_i is the d x d
 * row-major matrix at ops[op_off[i]] acting on leaf[i]. */
ttn_status ttn_expect(ttn_ctx* ctx, int n_obs, const int* leaf, const ttn_c128* ops,
                      const int64_t* op_off, ttn_c128* out);

/* <Psi|Psi> and <Psi|H|Psi>/<Psi|Psi>. */
ttn_status ttn_norm_energy(ttn_ctx* ctx, double* norm2, ttn_c128* energy);

/* Contract every leaf except keep_leaf with its basis vector 0 and write the
 * remaining vector over keep_leaf's physical index to out[d] (for the HEOM
 * generator this is rho_S = <0_bath|rho), paper SI Sec. S2). */
ttn_status ttn_vacuum_projection(ttn_ctx* ctx, int keep_leaf, ttn_c128* out);

/* Copy all node tensors to the host, in the layout of ttn_set_state;
 * offsets (n_nodes+1 entries) receives the layout. */
ttn_status ttn_get_state(ttn_ctx* ctx, ttn_c128* tensors, int64_t* offsets);

/* The context's tree as it is now (ttn_load or subspace expansion may have
 * changed it since ttn_create): *n_nodes, and, for each non-NULL array of
 * n_nodes entries, parent (root: -1), phys_dim (0 for interior nodes) and
 * the current bond dimension to the parent (root: 1).  Call with NULL
 * arrays first to learn n_nodes. */
ttn_status ttn_tree(const ttn_ctx* ctx, int* n_nodes, int* parent, int* phys_dim, int* bond_dim);

/* Bond dimension of every node to its parent (root: 1), out[n_nodes]. */
ttn_status ttn_bond_dims(ttn_ctx* ctx, int* out);

/* Effective-Hamiltonian action on one node tensor (paper Sec. II.C, Eq.
 * psi_eom_1 without the factor -i), on caller-owned DEVICE buffers:
 *     y = sum_t coeff[t] (x_j M_{t,j}) x,
 * where M_{t,j} acts on index j of the row-major tensor x (dims[0..D-1],
 * 1 <= D <= 8, every dims[j] <= 64) as y[.., p, ..] = sum_m M[p, m] x[.., m, ..].
 *   factor[t*D + j]  index into mats of the dims[j] x dims[j] row-major
 *                    complex128 matrix of term t on index j, or -1 (identity).
 *   mats[i]          DEVICE pointer to matrix i (host array of n_mats pointers).
 *   x, y             DEVICE pointers to prod(dims) complex128 values; y must
 *                    not overlap x or any matrix.
 * This is the contraction the sweep evaluates inside its Krylov
 * exponentials, with environment matrices as the factors.  The call
 * allocates its device scratch (three tensors and the term tables) with
 * cudaMalloc, runs one thread block on `stream` (a cudaStream_t, NULL for
 * the legacy default stream), waits for it, and frees the scratch.  Errors
 * are reported through ttn_last_error(NULL). */
ttn_status ttn_heff_apply(void* stream, int D, const int* dims, int n_terms, const ttn_c128* coeff,
                          const int* factor, int n_mats, const void* const* mats, const ttn_c128* x,
                          ttn_c128* y);

/* Allocation-free variant of ttn_heff_apply: same arguments, same result.
 * The paper has no counterpart; this entry point exists for callers that
 * must not allocate device memory during the call (for instance a serving
 * loop whose device memory is owned by its own pool allocator, or code that
 * cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
 * cause).  It calls no cudaMalloc, cudaFree or other allocating routine: its
 * scratch (three tensors and the term tables, 1.6 MB) is a static array in
 * device memory that every GPU loading the library holds until the process
 * exits.  Limits: prod(dims) <= 32768 elements, n_terms <= 512,
 * n_mats <= 512; larger requests return TTN_E_INVALID with a message.
 * The first call on a device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream
 * capture.  All calls share the one array, and it keeps the contents of the
 * last call: calls whose work can overlap on the GPU (several streams or
 * host threads) race on it -- on the term tables copied into it at the
 * start of a call as well as on the three scratch tensors -- and must be
 * serialised by the caller.  Runs one
 * thread block on `stream` and waits for it; errors through
 * ttn_last_error(NULL). */
ttn_status ttn_heff_apply_noalloc(void* stream, int D, const int* dims, int n_terms, const ttn_c128* coeff,
                                  const int* factor, int n_mats, const void* const* mats,
                                  const ttn_c128* x, ttn_c128* y);

/* Make `device` the CUDA device on which the calling thread's subsequent
 * ttn_create calls allocate (the library carries its own CUDA runtime, so
 * a device selected through another runtime, e.g. PyTorch's, is not seen). */
ttn_status ttn_set_device(int device);

/* Autotuning (no counterpart in the paper): pick the launch shape and the
 * contraction routines for ctx's own problem by timing them on the device.
 * Every trial restores a snapshot of everything a step modifies (node
 * tensors, bond buffer, Krylov workspace, counters, environment and
 * channel matrices), runs `steps` steps of length dt and times them with
 * CUDA events on the context's stream; the fastest configuration is kept
 * and the context is left exactly as it was before the call (the same
 * bits).  flags (bitwise or):
 *   1  thread blocks per instance (1, 2, 4, 8, 16; see ttn_set_cluster);
 *   2  mode-product routine per tensor-index dimension n, largest first:
 *      the register-fibre product (n <= 32 complex64 / 16 complex128) or
 *      the shared-memory-staged one;
 *   4  with 2, in TTN_MIXED also the tcgen05 tensor-core product (3xTF32)
 *      for n <= 48.  Contexts with such a dimension launch a separate
 *      build of the sweep kernel that carries the tcgen05 code (the default
 *      build has none: it keeps two blocks per SM overlapping); the request
 *      server always runs the default build, where those dimensions take
 *      the staged routine.
 * tuned_ms (may be NULL) receives the time of `steps` steps with the chosen
 * configuration.  The choice changes results only through rounding.
 * Errors: TTN_E_INVALID (steps outside 1..1000), TTN_E_STATE (no
 * Hamiltonian), device failures as for ttn_step. */
ttn_status ttn_autotune(ttn_ctx* ctx, double dt, int steps, int flags, double* tuned_ms);

/* The configuration in use: thread blocks per instance, the mode-product
 * routine per dimension (variants[0..64]: 0 default, 1 staged, 2 tensor
 * cores), and the last ttn_autotune's record: time of its steps with the
 * chosen and with the initial configuration (ms) and the trials run.  Any
 * output pointer may be NULL. */
ttn_status ttn_tuning(const ttn_ctx* ctx, int* blocks, unsigned char* variants, double* tuned_ms,
                      double* default_ms, int* trials);

/* Operator bond dimensions of the hierarchical sum-of-products form the
 * library built from the Hamiltonian (Sec. II.B.2): out[c] = the number of
 * (single-particle operator, mean-field operator) pairs crossing the bond
 * between node c and its parent -- one for the terms acting only inside the
 * subtree of c, one for those acting only outside, and, for the terms acting
 * on both sides, the size of a minimum vertex cover of the bipartite graph
 * whose vertices are their distinct inside and outside parts (a term is
 * summed into the channel of its inside part when that is in the cover,
 * else into the channel of its outside part); out[0] = 0.  For a multi-set
 * operator (ttn_set_multiset_hamiltonian): per set, one pre-summed channel
 * for its terms acting only inside the subtree and one for those acting
 * only outside; for the terms crossing the bond (same-set terms acting on
 * both sides, every set-coupling term -- an empty part of a coupling is
 * the overlap of the two sets' functions there), per set pair, one channel
 * per distinct inside part and one summed mean-field channel per distinct
 * inside part where the pair has fewer distinct inside than outside parts
 * there, else one channel per distinct inside and per distinct outside
 * part.  Works on
 * host-resident contexts (no device work).  TTN_E_STATE without a
 * Hamiltonian. */
ttn_status ttn_operator_dims(const ttn_ctx* ctx, int* out);

/* Set the configuration ttn_tuning reports (to reuse one context's tuning
 * for others of the same shape): blocks as for ttn_set_cluster, variants
 * [65] (may be NULL: unchanged) with entries 0, 1 or 2.  TTN_E_INVALID for
 * other values. */
ttn_status ttn_set_tuning(ttn_ctx* ctx, int blocks, const unsigned char* variants);

/* One mode product of the mixed-precision bulk alone (kernel-level entry
 * point, like ttn_heff_apply; the contraction of Sec. II.C Eq. psi_eom_1
 * along one tensor index):
 *     y[l, p, r] = w sum_m M[p, m] x[l, m, r]   (+ y[l, p, r] if accumulate)
 * for an L x n x R complex64 tensor x (interleaved float pairs, row-major)
 * and an n x n complex64 matrix M, all device pointers; w = wr + i wi.
 * tensor_cores = 1: tcgen05 tensor cores with 3xTF32 split products and FP32
 * accumulation (x = hi + lo with hi its TF32 rounding; hi*hi + hi*lo + lo*hi),
 * one block per SM over tiles of 128 fibres; 0: the FFMA routine the sweep
 * uses (one block).  1 <= n <= 64.  Runs on `stream` and waits.
 * Errors through ttn_last_error(NULL); TTN_E_TIMEOUT if a tensor-core
 * operation did not complete within its bounded wait. */
ttn_status ttn_mode_product_c64(void* stream, int64_t L, int n, int64_t R, const void* M, const void* x, void* y,
                                double wr, double wi, int accumulate, int tensor_cores);

/* Measured arithmetic peaks of the current device (no counterpart in the
 * paper: the denominators of the roofline the sweep kernel is measured
 * against).  fp32_tflops / fp64_tflops receive the sustained rate of fused
 * multiply-adds (2 flops each) of a kernel that fills every SM with
 * independent FMA chains, timed with CUDA events on `stream` (NULL: the
 * legacy default stream) over about `seconds` per pipe (0 < seconds <= 60).
 * Errors through ttn_last_error(NULL). */
ttn_status ttn_pipe_peaks(void* stream, double seconds, double* fp32_tflops, double* fp64_tflops);

/* Thread blocks that one instance of ctx runs on (no counterpart in the
 * paper: how a node update is spread over the GPU).  The sweep is a chain
 * of dependent node updates (Sec. II.C), so a large instance is sped up by
 * sharing each node's contractions, Krylov recurrences and QR among the
 * blocks of a thread-block cluster (distributed shared memory for the
 * team's sums, cluster barriers between phases).
 *   blocks  0 = automatic (default): one block per 4096 elements of the
 *           largest node tensor, a power of two, at most 16 -- a tree with
 *           nodes of 98 304 elements (the 2 x 24 vibronic tree) gets 16,
 *           one with nodes of a few hundred elements 1;
 *           1 = one thread block of 256 threads;
 *           2, 4, 8, 16 = a cluster of that many blocks of 512 threads.
 * A context whose largest index dimension exceeds 45 always runs on at
 * least 2 blocks.  ttn_step_batch runs every instance of a batch on the
 * largest count any of its contexts set explicitly (automatic contexts
 * count as 1 there: batches are spread over instances instead).  The
 * result of a step depends on the block count only through rounding.
 * Errors: TTN_E_INVALID for any other count. */
ttn_status ttn_set_cluster(ttn_ctx* ctx, int blocks);

/* The block count ttn_step uses for ctx with its current plan. */
ttn_status ttn_get_cluster(const ttn_ctx* ctx, int* blocks);

/* Step statistics of a context: total steps done since creation, the
 * algorithmic floating-point operations executed by its device programs
 * (complex multiply-add = 8; effective-Hamiltonian mode products, Gram-
 * Schmidt, environment builds, QR and bond absorption), and the device
 * completion time stamps (globaltimer, ns) of the last min(max_stamps,
 * steps, 4096) steps, oldest first.  Any output pointer may be NULL. */
ttn_status ttn_step_stats(ttn_ctx* ctx, int64_t* steps_done, double* flops, uint64_t* stamps,
                          int max_stamps, int* n_stamps);

/* Algorithmic floating-point operations executed by the context's device
 * programs since creation (the counter of ttn_step_stats) and the part of
 * them executed in FP64 arithmetic: QR and bond absorption always, and, in
 * TTN_FP64 mode, everything.  On GB300 the FP64 pipe runs at 1/64 of the
 * FP32 rate, so the split tells which pipe bounds a mixed-precision step.
 * Either pointer may be NULL. */
ttn_status ttn_flop_counts(ttn_ctx* ctx, double* total, double* fp64);

/* SM clock cycles the context's device programs spent per operation type,
 * cycles[32] (index: 1 QR towards a child, 2 QR towards the parent,
 * 3/4 bond absorption into child/parent, 5 environment builds, 6 operator
 * combinations, 7 Krylov exponentials, 8-10 observables, 11 step end,
 * 12 subspace-expansion tests, 13 ground-state eigen-solves;
 * inside those: 16 effective-Hamiltonian products, 17 Gram-Schmidt,
 * 18 small projected exponentials, 19 Gram contractions, 20 conversions). */
ttn_status ttn_op_cycles(ttn_ctx* ctx, uint64_t* cycles);

/* Run all further work of the context on this cudaStream_t. */
ttn_status ttn_set_stream(ttn_ctx* ctx, void* cuda_stream);

/* Device memory held by the context, in bytes. */
ttn_status ttn_device_bytes(const ttn_ctx* ctx, size_t* bytes);

/* ---------------------------------------------------------------------
 * Request server: continuous batching of independent propagations.
 *
 * The paper runs one propagation at a time; this is a serving layer over
 * the same step (Sec. II.C) for many independent requests on one device --
 * parameter sweeps over couplings, temperatures or bath discretisations.
 * A request is a context (tree, state, Hamiltonian) and (dt, nsteps).
 * Submitted requests wait in a FIFO queue holding no device memory (the
 * context is moved to the host).  A request runs on the block count its
 * context asks for (ttn_get_cluster: one block, or a cluster of 2..16);
 * the server keeps one lane per block count, each with its own stream and
 * launch, so one-block and cluster requests run side by side.
 * ttn_server_pump admits queued requests in arrival order to their lanes
 * while the lane has a free slot (max_slots for the one-block lane; for a
 * cluster lane, as many clusters as the device holds at once) and the sum
 * of all admitted footprints (ttn_footprint) stays within hbm_budget; an
 * admitted context keeps its tensors and environments on the device until
 * it finishes.  Each pump waits until some lane's launch has finished,
 * retires that lane's finished requests (their device time stamps are
 * recorded, their tensors copied back to the host context, their memory
 * returned), admits more, and starts the next launch of every idle lane:
 * one block or cluster per admitted context, each running whole steps of
 * its own dt until its steps are done or the launch's slice of device time
 * is used up.  Admission of new requests (allocation, upload, environment
 * build) runs on a separate stream while launches are in flight.  A
 * context's results do not depend on the other contexts in the launch nor
 * on how its steps are split over launches: they equal ttn_step's with
 * the same block count.
 * The server is driven by one host thread; it is not thread-safe.
 * --------------------------------------------------------------------- */
typedef struct ttn_server ttn_server;

typedef struct {
    size_t hbm_budget;   /* bytes the admitted contexts may hold together;
                            0 = 90% of the device's free memory at creation */
    int max_slots;       /* most contexts admitted at once to the one-block
                            lane (and a cap for cluster lanes); 0 = 2 per SM */
    double slice_ms;     /* device time per launch (at least one step of the
                            slowest admitted context); 0 = 20 ms           */
    int use_graph;       /* 1: each launch is the replay of one CUDA graph
                            (table upload, kernel, result read-back)        */
} ttn_server_opts;

typedef struct {
    int64_t submitted, completed, failed, queued, running;
    int64_t steps;        /* steps run for all requests                     */
    int64_t launches;
    int64_t peak_running; /* most contexts admitted at once                 */
    size_t bytes_in_use, peak_bytes;   /* sums of admitted footprints       */
    double p50_step_ms, p99_step_ms;   /* per-step latency: interval between
                            consecutive step completions of one request
                            (device time stamps), over finished requests    */
    int64_t n_latencies;
} ttn_server_stats;

/* Create a server on the current device for contexts of one precision.
 * opts may be NULL (defaults; use_graph = 1). */
ttn_status ttn_server_create(int precision, const ttn_server_opts* opts, ttn_server** out);

/* Queue ctx for nsteps steps of dt (opts: Krylov / QR settings; expand
 * must be 0; NULL = defaults).  The context must have a Hamiltonian and the
 * server's precision; a resident context is moved to the host first.  The
 * caller keeps ownership but must not use ctx until its ticket is returned
 * by ttn_server_poll (afterwards ctx is host-resident and usable; on
 * failure it is marked failed, see ttn_last_error). */
ttn_status ttn_server_submit(ttn_server* srv, ttn_ctx* ctx, double dt, int nsteps,
                             const ttn_step_opts* opts, int64_t* ticket);

/* One scheduling round (see above).  Returns after starting the next launch
 * (it does not wait for it).  n_running / n_queued may be NULL. */
ttn_status ttn_server_pump(ttn_server* srv, int* n_running, int* n_queued);

/* Pump until every submitted request has finished. */
ttn_status ttn_server_drain(ttn_server* srv);

/* Tickets of requests finished since the last poll (up to max), with their
 * status: TTN_OK, TTN_E_OOM (footprint larger than the budget), or the
 * device status that stopped it. */
ttn_status ttn_server_poll(ttn_server* srv, int max, int64_t* tickets, ttn_status* status, int* n);

/* Counters and per-step latency percentiles of the server. */
ttn_status ttn_server_get_stats(ttn_server* srv, ttn_server_stats* out);

/* Every recorded per-step latency (ms), in recording order (up to max). */
ttn_status ttn_server_latencies(ttn_server* srv, double* out_ms, int64_t max, int64_t* n);

/* Message for the server's most recent failure. */
const char* ttn_server_last_error(const ttn_server* srv);

/* Wait for the launch in flight, move admitted contexts back to the host
 * (unfinished) and release the server.  NULL is ignored. */
void ttn_server_destroy(ttn_server* srv);

/* Message for the most recent failure of a call on ctx (or of ttn_create
 * when ctx is NULL).  Valid until the next call on the same context. */
const char* ttn_last_error(const ttn_ctx* ctx);

/* Release the context and its device memory.  NULL is ignored. */
void ttn_destroy(ttn_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TTN_H */
