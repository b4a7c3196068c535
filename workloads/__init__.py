"""Seeded synthetic inputs for TTN / ML-MCTDH time evolution.

This module is shared by the CPU oracle (``oracle/``) and by the GPU library's
tests and benchmark.  It only *describes* problems: tree topologies with local
and bond dimensions (paper Sec. II.A, Eqs. wavefunction_expansion_spf and
spf_recursion), sum-of-product Hamiltonians (Sec. II.B.1, Eq. sop_ham),
discretised baths (Sec. II.E.1), the HEOM generator written as a
sum-of-product operator (Sec. II.E.3, Eq. fpheom_op) and initial product states.
It contains none of the time-evolution arithmetic (no environments, no
effective Hamiltonian, no Krylov, no QR).

Conventions
-----------
* Trees: node 0 is the root, ``parent[i] < i``, children are ordered by index.
  ``phys_dim[i] > 0`` marks a leaf (one physical mode), ``bond_dim[i]`` is the
  bond to the parent (the root's is 1).
* A node tensor is stored row-major with shape ``[n_1, ..., n_d, N]``: the child
  bond dimensions in child order (for a leaf the single physical dimension),
  then the parent bond dimension N.
* A sum-of-product Hamiltonian is ``H = sum_r c_r prod_{(leaf, M)} M_leaf``
  where every factor is a dense d x d matrix acting on one leaf; leaves not
  named in a term carry the identity.  hbar = 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

__all__ = [
    "Tree", "SOP", "build_tree", "clamp_bonds", "product_state",
    "boson_ops", "pauli", "ohmic_J", "thermal_J", "discretise_orthopol",
    "discretise_uniform_density", "spin_boson_sop", "vibronic_sop",
    "drude_lorentz_exponentials", "heom_sop",
    "config_c1", "config_c2", "config_c3", "config_c4", "config_c5_requests",
    "Problem", "MultiSetSOP", "MultiSetProblem", "multiset_product_state",
    "multiset_vibronic_problem",
]


# ----------------------------------------------------------------------------
# Trees
# ----------------------------------------------------------------------------
@dataclass
class Tree:
    parent: np.ndarray      # int, parent[0] = -1
    phys_dim: np.ndarray    # int, >0 on leaves, 0 on interior nodes
    bond_dim: np.ndarray    # int, bond to parent (root: 1)
    labels: list = field(default_factory=list)   # free-form tag per node

    @property
    def n(self) -> int:
        return len(self.parent)

    def children(self, z: int) -> list:
        return [c for c in range(z + 1, self.n) if self.parent[c] == z]

    def is_leaf(self, z: int) -> bool:
        return self.phys_dim[z] > 0

    def mode_dims(self, z: int) -> list:
        """Index dimensions of node z's tensor: children (or the physical
        index) followed by the parent bond."""
        if self.is_leaf(z):
            first = [int(self.phys_dim[z])]
        else:
            first = [int(self.bond_dim[c]) for c in self.children(z)]
        return first + [int(self.bond_dim[z]) if z > 0 else 1]

    def leaves(self) -> list:
        return [z for z in range(self.n) if self.is_leaf(z)]

    def subtree_leaves(self, z: int) -> list:
        out = []
        stack = [z]
        while stack:
            u = stack.pop()
            if self.is_leaf(u):
                out.append(u)
            else:
                stack.extend(self.children(u))
        return sorted(out)

    def leaf_of_label(self, label) -> int:
        return self.labels.index(label)


def build_tree(spec) -> Tree:
    """Build a tree from a nested spec.

    A leaf is ``("leaf", d, bond, label)``; an interior node is
    ``("node", bond, [child specs...])``.  The root's bond is ignored (1).
    Nodes are numbered in pre-order so that ``parent[i] < i`` and children are
    in index order.
    """
    parent, phys, bond, labels = [], [], [], []

    def rec(s, p):
        z = len(parent)
        parent.append(p)
        if s[0] == "leaf":
            _, d, b, lab = s
            phys.append(int(d)); bond.append(int(b)); labels.append(lab)
        else:
            _, b, ch = s
            phys.append(0); bond.append(int(b)); labels.append(None)
            for c in ch:
                rec(c, z)
        return z

    rec(spec, -1)
    bond[0] = 1
    t = Tree(np.array(parent, dtype=np.int64), np.array(phys, dtype=np.int64),
             np.array(bond, dtype=np.int64), labels)
    clamp_bonds(t)
    return t


def clamp_bonds(t: Tree) -> None:
    """Lower bond dimensions (in place) until every node is consistent:
    a leaf's bond is at most its local dimension, an interior node's parent
    bond is at most the product of its child bonds, and each child bond is at
    most the product of the node's other index dimensions.  These are the
    conditions under which every matricisation used by the sweep has at least
    as many rows as columns."""
    changed = True
    while changed:
        changed = False
        for z in range(t.n):
            dims = t.mode_dims(z)
            if z > 0:
                cap = int(np.prod(dims[:-1]))
                if t.bond_dim[z] > cap:
                    t.bond_dim[z] = cap; changed = True
            if not t.is_leaf(z):
                ch = t.children(z)
                dims = t.mode_dims(z)
                tot = int(np.prod(dims))
                for k, c in enumerate(ch):
                    others = tot // dims[k]
                    if t.bond_dim[c] > others:
                        t.bond_dim[c] = others; changed = True


def balanced_spec(leaves, chi, node_bond=None):
    """Balanced binary grouping of a list of leaf specs; interior bonds chi."""
    if len(leaves) == 1:
        return leaves[0]
    h = (len(leaves) + 1) // 2
    return ("node", chi if node_bond is None else node_bond,
            [balanced_spec(leaves[:h], chi), balanced_spec(leaves[h:], chi)])


# ----------------------------------------------------------------------------
# Operators
# ----------------------------------------------------------------------------
def boson_ops(d: int):
    """Truncated Fock-basis matrices: a, a^dagger, n, x = a + a^dagger."""
    a = np.diag(np.sqrt(np.arange(1, d, dtype=np.float64)), k=1).astype(np.complex128)
    ad = a.conj().T.copy()
    n = np.diag(np.arange(d, dtype=np.float64)).astype(np.complex128)
    return {"a": a, "adag": ad, "n": n, "x": a + ad}


def pauli():
    """Basis |0> = up, |1> = down: sigma_z = |0><0| - |1><1|."""
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    sy = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    sz = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    p0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
    p1 = np.array([[0, 0], [0, 1]], dtype=np.complex128)
    return {"x": sx, "y": sy, "z": sz, "p0": p0, "p1": p1, "I": np.eye(2, dtype=np.complex128)}


@dataclass
class SOP:
    """H = sum_r coeffs[r] * prod_{(leaf, m) in factors[r]} mats[m] (on leaf)."""
    coeffs: list = field(default_factory=list)
    factors: list = field(default_factory=list)
    mats: list = field(default_factory=list)
    hermitian: bool = True

    def mat_id(self, M) -> int:
        M = np.ascontiguousarray(M, dtype=np.complex128)
        for i, X in enumerate(self.mats):
            if X.shape == M.shape and np.array_equal(X, M):
                return i
        self.mats.append(M)
        return len(self.mats) - 1

    def add(self, c, *pairs):
        """Add the term c * prod (leaf, matrix).  Zero coefficients are dropped."""
        if c == 0:
            return
        self.coeffs.append(complex(c))
        self.factors.append([(int(l), self.mat_id(M)) for (l, M) in pairs])

    @property
    def n_terms(self) -> int:
        return len(self.coeffs)

    def to_csr(self):
        """Flat arrays in the layout the C ABI takes."""
        coeff = np.array(self.coeffs, dtype=np.complex128)
        term_ptr = np.zeros(self.n_terms + 1, dtype=np.int32)
        leaf, off = [], []
        mat_off = np.zeros(len(self.mats) + 1, dtype=np.int64)
        for i, M in enumerate(self.mats):
            mat_off[i + 1] = mat_off[i] + M.size
        flat = np.concatenate([M.ravel() for M in self.mats]) if self.mats else np.zeros(0, np.complex128)
        for r, fs in enumerate(self.factors):
            term_ptr[r + 1] = term_ptr[r] + len(fs)
            for (l, m) in fs:
                leaf.append(l); off.append(mat_off[m])
        return (coeff, term_ptr, np.array(leaf, dtype=np.int32),
                np.ascontiguousarray(flat), np.array(off, dtype=np.int64))


@dataclass
class MultiSetSOP(SOP):
    """Multi-set Hamiltonian (paper Sec. II.A, multi-set ansatz)
    H = sum_r coeffs[r] |bra[r]><ket[r]| (x) prod_{(leaf, m) in factors[r]} mats[m]:
    the set index (the system state alpha) is not a leaf of the tree; every
    term names the pair of set states it connects and a product of leaf
    factors acting on the environment degrees of freedom (an empty product
    is the identity there)."""
    n_sets: int = 1
    bra: list = field(default_factory=list)
    ket: list = field(default_factory=list)

    def add(self, c, *pairs):
        raise TypeError("multi-set terms name their set pair: use add_set(alpha, beta, c, ...)")

    def add_set(self, alpha, beta, c, *pairs):
        """Add c |alpha><beta| (x) prod (leaf, matrix).  Zero coefficients are dropped."""
        assert 0 <= alpha < self.n_sets and 0 <= beta < self.n_sets
        if c == 0:
            return
        self.coeffs.append(complex(c))
        self.factors.append([(int(l), self.mat_id(M)) for (l, M) in pairs])
        self.bra.append(int(alpha))
        self.ket.append(int(beta))

    def to_csr(self):
        """The single-set flat arrays plus the per-term set pair."""
        return super().to_csr() + (np.array(self.bra, dtype=np.int32), np.array(self.ket, dtype=np.int32))


# ----------------------------------------------------------------------------
# Initial states
# ----------------------------------------------------------------------------
def _complete_columns(first: np.ndarray, ncols: int) -> np.ndarray:
    """Columns: ``first`` (normalised) followed by unit vectors e_0, e_1, ...
    made orthogonal to the previous columns (two classical Gram-Schmidt
    passes); a unit vector whose remainder has norm below 1/2 is skipped."""
    d = first.shape[0]
    cols = [first / np.linalg.norm(first)]
    j = 0
    while len(cols) < ncols:
        e = np.zeros(d, dtype=np.complex128); e[j] = 1.0
        j += 1
        for _ in range(2):
            for c in cols:
                e = e - c * np.vdot(c, e)
        nrm = np.linalg.norm(e)
        if nrm > 0.5:
            cols.append(e / nrm)
    return np.stack(cols, axis=1)


def product_state(t: Tree, leaf_vecs: dict) -> list:
    """Tensors of the product state prod_leaf |v_leaf> with unoccupied
    single-particle functions chosen deterministically:

    * leaf: column 0 is v (normalised), further columns complete it with the
      lowest-index unit vectors;
    * interior node: column i is the unit tensor at the i-th child multi-index
      in row-major (lexicographic) order, so column 0 selects SPF 0 of every
      child;
    * root: a single 1 at multi-index (0, ..., 0).
    The result is in canonical gauge with the orthogonality centre at the root.
    A missing entry in ``leaf_vecs`` means the basis vector e_0.
    """
    A = []
    for z in range(t.n):
        dims = t.mode_dims(z)
        N = dims[-1]
        if t.is_leaf(z):
            d = dims[0]
            v = leaf_vecs.get(z)
            if v is None:
                v = np.zeros(d, dtype=np.complex128); v[0] = 1.0
            A.append(_complete_columns(np.asarray(v, dtype=np.complex128), N))
        else:
            M = np.zeros((int(np.prod(dims[:-1])), N), dtype=np.complex128)
            for i in range(N):
                M[i, i] = 1.0
            A.append(M.reshape(dims))
    return [np.ascontiguousarray(a.reshape(t.mode_dims(z))) for z, a in enumerate(A)]


def multiset_product_state(t: Tree, amps, leaf_vecs=None) -> list:
    """Per-set tensor lists of sum_alpha amps[alpha] |alpha> prod_leaf |v_leaf^alpha>:
    every set is ``product_state`` of its own leaf vectors (``leaf_vecs[alpha]``,
    default the basis vector e_0 on every leaf) with its root tensor scaled by
    amps[alpha] (``leaf_vecs`` indexed by alpha; zero amplitudes allowed: an unoccupied set keeps orthonormal
    single-particle functions and a zero top tensor)."""
    out = []
    for a, amp in enumerate(amps):
        A = product_state(t, {} if leaf_vecs is None else leaf_vecs[a])
        A[0] = A[0] * complex(amp)
        out.append(A)
    return out


# ----------------------------------------------------------------------------
# Bath spectral densities and discretisation (paper Sec. II.E.1)
# ----------------------------------------------------------------------------
def ohmic_J(alpha: float, wc: float):
    """J(w) = (pi/2) alpha w exp(-w/wc) (paper Sec. III)."""
    return lambda w: 0.5 * np.pi * alpha * w * np.exp(-np.abs(w) / wc)


def thermal_J(J, beta: float):
    """J_beta(w) = J(w) (1 + coth(beta w / 2)) / 2 (Eq. effective_spec_dens);
    beta = inf gives J(w) on w > 0 and 0 on w < 0."""
    def Jb(w):
        w = np.asarray(w, dtype=np.float64)
        if np.isinf(beta):
            return np.where(w > 0, J(w), 0.0)
        x = beta * w / 2.0
        with np.errstate(divide="ignore", invalid="ignore"):
            c = np.where(np.abs(x) > 1e-12, 1.0 / np.tanh(x), 0.0)
        return 0.5 * J(w) * (1.0 + c)
    return Jb


def discretise_uniform_density(J, w_lo: float, w_hi: float, n: int):
    """Density-of-frequencies rule with a uniform density on [w_lo, w_hi]:
    w_k equally spaced including both ends, g_k^2 = J(w_k) / (pi rho) with
    rho = 1 / spacing (paper Sec. II.E.1)."""
    w = np.linspace(w_lo, w_hi, n)
    dw = (w_hi - w_lo) / (n - 1)
    g = np.sqrt(J(w) * dw / np.pi)
    return w, g


def discretise_orthopol(J, w_min: float, w_max: float, n: int, n_fine: int | None = None):
    """Orthogonal-polynomial discretisation (paper Sec. II.E.1): the n-point
    Gauss rule of the measure J(w) dw on [w_min, w_max]; nodes w_i, weights
    alpha_i, couplings g_i = sqrt(alpha_i / pi).

    The recurrence coefficients are computed with the discretised Stieltjes
    (Lanczos) procedure on a fine Gauss-Legendre discretisation of the
    measure, followed by the Golub-Welsch eigenvalue problem."""
    n_fine = n_fine or max(8 * n, 400)
    x, w = np.polynomial.legendre.leggauss(n_fine)
    x = 0.5 * (w_max - w_min) * x + 0.5 * (w_max + w_min)
    w = 0.5 * (w_max - w_min) * w * J(x)
    keep = w > 0
    x, w = x[keep], w[keep]
    mu0 = w.sum()
    q = np.sqrt(w / mu0)
    Q = np.zeros((len(x), n))
    a = np.zeros(n); b = np.zeros(n)
    Q[:, 0] = q
    for k in range(n):
        v = x * Q[:, k]
        a[k] = Q[:, k] @ v
        v = v - a[k] * Q[:, k] - (b[k - 1] * Q[:, k - 1] if k > 0 else 0.0)
        v -= Q[:, :k + 1] @ (Q[:, :k + 1].T @ v)
        v -= Q[:, :k + 1] @ (Q[:, :k + 1].T @ v)
        if k + 1 < n:
            b[k] = np.linalg.norm(v)
            Q[:, k + 1] = v / b[k]
    T = np.diag(a) + np.diag(b[:n - 1], 1) + np.diag(b[:n - 1], -1)
    lam, V = np.linalg.eigh(T)
    alpha = mu0 * V[0, :] ** 2
    return lam, np.sqrt(alpha / np.pi)


# ----------------------------------------------------------------------------
# Model Hamiltonians
# ----------------------------------------------------------------------------
def spin_boson_sop(spin_leaf: int, mode_leaves, d_modes, eps, delta, g, w) -> SOP:
    """H = eps/2 sz + delta/2 sx + sz sum_k g_k (a_k + a_k^+) + sum_k w_k n_k
    (paper Eq. sbm_hamiltonian)."""
    P = pauli()
    H = SOP(hermitian=True)
    H.add(eps / 2.0, (spin_leaf, P["z"]))
    H.add(delta / 2.0, (spin_leaf, P["x"]))
    for k, leaf in enumerate(mode_leaves):
        dk = d_modes[k] if np.ndim(d_modes) else d_modes
        B = boson_ops(int(dk))
        H.add(g[k], (spin_leaf, P["z"]), (leaf, B["x"]))
        H.add(w[k], (leaf, B["n"]))
    return H


def vibronic_sop(el_leaf, mode_leaves, d_modes, omega, kappa, gamma_quad,
                 quad_modes, lam, lam_modes, delta) -> SOP:
    """Two-state linear/quadratic vibronic model (the form of paper Sec. IV.A):
    H = sum_i w_i (n_i + 1/2) - delta sz + sum_{i,s} kappa_i^s |s><s| Q_i
        + sum_{i in quad, s} gamma_i^s |s><s| Q_i^2 + sum_{i in G3} lam_i sx Q_i
    with Q = (a + a^+)/sqrt(2), sz = |0><0| - |1><1|."""
    P = pauli()
    H = SOP(hermitian=True)
    H.add(-delta, (el_leaf, P["z"]))
    proj = [P["p0"], P["p1"]]
    for i, leaf in enumerate(mode_leaves):
        B = boson_ops(int(d_modes[i]))
        Q = B["x"] / np.sqrt(2.0)
        num = B["n"] + 0.5 * np.eye(int(d_modes[i]))
        H.add(omega[i], (leaf, num))
        for s in range(2):
            H.add(kappa[i, s], (el_leaf, proj[s]), (leaf, Q))
    for j, i in enumerate(quad_modes):
        B = boson_ops(int(d_modes[i]))
        Q = B["x"] / np.sqrt(2.0)
        for s in range(2):
            H.add(gamma_quad[j, s], (el_leaf, proj[s]), (mode_leaves[i], Q @ Q))
    for j, i in enumerate(lam_modes):
        B = boson_ops(int(d_modes[i]))
        H.add(lam[j], (el_leaf, P["x"]), (mode_leaves[i], B["x"] / np.sqrt(2.0)))
    return H


def drude_lorentz_exponentials(lam: float, gamma: float, beta: float, n_matsubara: int):
    """C(t) = sum_k alpha_k exp(-nu_k t) for J(w) = 2 lam gamma w / (w^2 + gamma^2)
    (Drude-Lorentz pole plus Matsubara terms)."""
    nu = [gamma]
    al = [lam * gamma * (1.0 / np.tan(beta * gamma / 2.0) - 1j)]
    for j in range(1, n_matsubara + 1):
        vj = 2.0 * np.pi * j / beta
        nu.append(vj)
        al.append(4.0 * lam * gamma * vj / (beta * (vj * vj - gamma * gamma)))
    return np.array(al, dtype=np.complex128), np.array(nu, dtype=np.complex128)


def heom_sop(sys_leaf: int, a_leaves, b_leaves, depth: int, Hs: np.ndarray,
             S: np.ndarray, alpha, nu) -> SOP:
    """Free-pole HEOM generator in operator form (paper Eq. fpheom_op, read with
    the sums running over the K exponentials and nu_k on the number operators):
        d|rho)/dt = -i G |rho),
        G = L_s - i sum_k (nu_k a_k^+ a_k + nu_k^* b_k^+ b_k)
            + sum_k (alpha_k/sqrt|alpha_k|) S^L a_k^+ - (alpha_k^*/sqrt|alpha_k|) S^R b_k^+
            + sum_k sqrt|alpha_k| S^- (a_k + b_k)
    on |rho) = vec(rho) (row-major, index 2i+j) times 2K bosonic modes of
    dimension depth+1.  L_s rho = [H_s, rho]; S^L rho = S rho; S^R rho = rho S;
    S^- = S^L - S^R.  The generator is not Hermitian."""
    I2 = np.eye(Hs.shape[0], dtype=np.complex128)
    Ls = np.kron(Hs, I2) - np.kron(I2, Hs.T)
    SL = np.kron(S, I2)
    SR = np.kron(I2, S.T)
    Sm = SL - SR
    B = boson_ops(depth + 1)
    G = SOP(hermitian=False)
    G.add(1.0, (sys_leaf, Ls))
    for k in range(len(alpha)):
        ak, nk = complex(alpha[k]), complex(nu[k])
        r = np.sqrt(abs(ak))
        G.add(-1j * nk, (a_leaves[k], B["n"]))
        G.add(-1j * np.conj(nk), (b_leaves[k], B["n"]))
        G.add(ak / r, (sys_leaf, SL), (a_leaves[k], B["adag"]))
        G.add(-np.conj(ak) / r, (sys_leaf, SR), (b_leaves[k], B["adag"]))
        G.add(r, (sys_leaf, Sm), (a_leaves[k], B["a"]))
        G.add(r, (sys_leaf, Sm), (b_leaves[k], B["a"]))
    return G


# ----------------------------------------------------------------------------
# Configurations
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    tree: Tree
    H: SOP
    tensors: list            # initial TTN tensors (centre at root)
    dt: float
    nsteps: int
    obs_leaves: list         # leaves whose populations are reported
    meta: dict = field(default_factory=dict)


def config_c1(full_bonds: bool = False, d: int = 8, chi: int = 4, alpha: float = 0.2,
              wc: float = 5.0, eps: float = 0.0, delta: float = 1.0, g_scale: float = 1.0,
              nsteps: int = 200, dt: float = 0.05) -> Problem:
    """Spin + 4 modes, tree root(L(spin, b1), R(b2, R'(b3, b4))).  Frequencies
    {0.1, 0.9, 1.7, 2.5}, g_k = sqrt(J(w_k) * 0.8 / pi) (uniform density of
    frequencies).  full_bonds=True uses the exact bond dimensions."""
    if full_bonds:
        bL = bR = 2 * d; bRp = d * d; bm = d
    else:
        bL = bR = bRp = chi; bm = min(chi, d)
    spec = ("node", 1, [
        ("node", bL, [("leaf", 2, 2, "spin"), ("leaf", d, bm, "b1")]),
        ("node", bR, [("leaf", d, bm, "b2"),
                      ("node", bRp, [("leaf", d, bm, "b3"), ("leaf", d, bm, "b4")])]),
    ])
    t = build_tree(spec)
    w, g = discretise_uniform_density(ohmic_J(alpha, wc), 0.1, 2.5, 4)
    g = g * g_scale
    spin = t.leaf_of_label("spin")
    modes = [t.leaf_of_label(f"b{k}") for k in range(1, 5)]
    H = spin_boson_sop(spin, modes, d, eps, delta, g, w)
    A = product_state(t, {})
    return Problem("c1_spin_boson_4modes" + ("_fullbond" if full_bonds else ""), t, H, A,
                   dt, nsteps, [spin] + modes, {"w": w, "g": g, "spin": spin, "modes": modes})


def _vibronic_tree(d_modes, bonds=(24, 16, 12, 8)):
    b_rootA, b_AC, b_CD, b_Dleaf = bonds
    k = 0
    def D():
        nonlocal k
        ls = []
        for _ in range(2):
            ls.append(("leaf", int(d_modes[k]), b_Dleaf, f"m{k}")); k += 1
        return ("node", b_CD, ls)
    def C():
        return ("node", b_AC, [D(), D()])
    def A():
        return ("node", b_rootA, [C(), C(), C()])
    spec = ("node", 1, [("leaf", 2, 2, "el"), A(), A()])
    return build_tree(spec)


def config_c2(seed: int = 2, n_modes: int = 24, bonds=(24, 16, 12, 8), d_range=(10, 30),
              nsteps: int = 1000, dt: float = 0.1, delta: float = 0.1) -> Problem:
    """2 electronic states x 24 modes (seeded): w ~ U[0.05, 0.5],
    kappa ~ N(0, 0.05^2), 20% of modes with quadratic gamma ~ N(0, 0.01^2),
    interstate coupling lam ~ N(0, 0.05^2) on 3 seeded modes, d ~ U{10..30}.
    Initial |1> x vacuum."""
    assert n_modes == 24, "the ML tree layout is fixed at 24 modes"
    rng = np.random.default_rng(seed)
    omega = rng.uniform(0.05, 0.5, n_modes)
    kappa = rng.normal(0.0, 0.05, (n_modes, 2))
    n_quad = int(round(0.2 * n_modes))
    quad = np.sort(rng.choice(n_modes, n_quad, replace=False))
    gq = rng.normal(0.0, 0.01, (n_quad, 2))
    lam_modes = np.sort(rng.choice(n_modes, 3, replace=False))
    lam = rng.normal(0.0, 0.05, 3)
    d_modes = rng.integers(d_range[0], d_range[1] + 1, n_modes)
    t = _vibronic_tree(d_modes, bonds)
    el = t.leaf_of_label("el")
    modes = [t.leaf_of_label(f"m{i}") for i in range(n_modes)]
    H = vibronic_sop(el, modes, d_modes, omega, kappa, gq, quad, lam, lam_modes, delta)
    v = np.zeros(2, dtype=np.complex128); v[1] = 1.0
    A = product_state(t, {el: v})
    return Problem(f"c2_vibronic_2x{n_modes}_seed{seed}", t, H, A, dt, nsteps, [el] + modes,
                   {"el": el, "modes": modes, "d_modes": d_modes})


def spin_boson_star_problem(n_modes: int, d: int, chi: int, alpha: float, wc: float = 5.0,
                            wmax_factor: float = 10.0, delta: float = 1.0, eps: float = 0.0,
                            beta: float = np.inf, dt: float = 0.01, nsteps: int = 500,
                            name: str = "spin_boson_star") -> Problem:
    """Spin-boson (star topology) on root(spin, balanced binary tree over the
    bath), bath from the orthogonal-polynomial rule on [0, wmax] (or the
    thermal density on [-wmax, wmax] when beta is finite)."""
    J = ohmic_J(alpha, wc)
    wmax = wmax_factor * wc
    if np.isinf(beta):
        w, g = discretise_orthopol(J, 0.0, wmax, n_modes)
    else:
        w, g = discretise_orthopol(thermal_J(J, beta), -wmax, wmax, n_modes)
    bath = [("leaf", d, min(chi, d), f"b{k}") for k in range(n_modes)]
    spec = ("node", 1, [("leaf", 2, 2, "spin"), balanced_spec(bath, chi)])
    t = build_tree(spec)
    spin = t.leaf_of_label("spin")
    modes = [t.leaf_of_label(f"b{k}") for k in range(n_modes)]
    H = spin_boson_sop(spin, modes, d, eps, delta, g, w)
    A = product_state(t, {})
    return Problem(name, t, H, A, dt, nsteps, [spin] + modes,
                   {"w": w, "g": g, "spin": spin, "modes": modes})


def config_c3(alpha: float = 0.1, n_modes: int = 300, d: int = 20, chi: int = 8) -> Problem:
    """Spin + 300 Ohmic modes (wc = 5, wmax = 10 wc), d = 20, initial chi = 8."""
    return spin_boson_star_problem(n_modes, d, chi, alpha, dt=0.01, nsteps=500,
                                   name=f"c3_spin_boson_{n_modes}modes_alpha{alpha}")


def config_c4(K_matsubara: int = 15, depth: int = 10, chi: int = 24, lam: float = 0.1,
              gamma: float = 5.0, beta: float = 1.0, delta: float = 1.0, eps: float = 0.0,
              dt: float = 0.015, nsteps: int = 2000) -> Problem:
    """HEOM spin-boson as a TTN: K = K_matsubara + 1 exponentials, 2K modes of
    dimension depth+1 under a balanced binary tree, system leaf holding vec(rho_S)
    (d = 4), S = sigma_z, initial rho_S = |up><up|, bath ADOs in the vacuum."""
    al, nu = drude_lorentz_exponentials(lam, gamma, beta, K_matsubara)
    K = len(al)
    bath = []
    for k in range(K):
        bath.append(("leaf", depth + 1, min(chi, depth + 1), f"a{k}"))
        bath.append(("leaf", depth + 1, min(chi, depth + 1), f"b{k}"))
    spec = ("node", 1, [("leaf", 4, 4, "sys"), balanced_spec(bath, chi)])
    t = build_tree(spec)
    sysl = t.leaf_of_label("sys")
    a_l = [t.leaf_of_label(f"a{k}") for k in range(K)]
    b_l = [t.leaf_of_label(f"b{k}") for k in range(K)]
    P = pauli()
    Hs = eps / 2.0 * P["z"] + delta / 2.0 * P["x"]
    G = heom_sop(sysl, a_l, b_l, depth, Hs, P["z"], al, nu)
    rho0 = np.zeros(4, dtype=np.complex128); rho0[0] = 1.0
    A = product_state(t, {sysl: rho0})
    return Problem(f"c4_heom_K{K}_L{depth}", t, G, A, dt, nsteps, [sysl],
                   {"sys": sysl, "a": a_l, "b": b_l, "alpha": al, "nu": nu, "Hs": Hs})


def vibronic_balanced_problem(n_modes: int, d: int, chi: int, seed: int, dt: float = 0.1,
                              delta: float = 0.1, nsteps: int = 100) -> Problem:
    """Two-state vibronic model with the parameter recipe of config_c2
    (seeded) on root(el, balanced binary tree over n_modes leaves of local
    dimension d), interior bonds chi.  Initial |1> x vacuum."""
    rng = np.random.default_rng(seed)
    omega = rng.uniform(0.05, 0.5, n_modes)
    kappa = rng.normal(0.0, 0.05, (n_modes, 2))
    n_quad = int(round(0.2 * n_modes))
    quad = np.sort(rng.choice(n_modes, n_quad, replace=False))
    gq = rng.normal(0.0, 0.01, (n_quad, 2))
    n_lam = min(3, n_modes)
    lam_modes = np.sort(rng.choice(n_modes, n_lam, replace=False))
    lam = rng.normal(0.0, 0.05, n_lam)
    d_modes = np.full(n_modes, d)
    bath = [("leaf", d, min(chi, d), f"m{k}") for k in range(n_modes)]
    t = build_tree(("node", 1, [("leaf", 2, 2, "el"), balanced_spec(bath, chi)]))
    el = t.leaf_of_label("el")
    modes = [t.leaf_of_label(f"m{i}") for i in range(n_modes)]
    H = vibronic_sop(el, modes, d_modes, omega, kappa, gq, quad, lam, lam_modes, delta)
    v = np.zeros(2, dtype=np.complex128); v[1] = 1.0
    A = product_state(t, {el: v})
    return Problem(f"vibronic_2x{n_modes}_d{d}_chi{chi}_seed{seed}", t, H, A, dt, nsteps, [el] + modes,
                   {"el": el, "modes": modes, "d_modes": d_modes})


@dataclass
class MultiSetProblem:
    name: str
    tree: Tree               # the environment tree (shared by every set)
    H: MultiSetSOP
    tensors: list            # tensors[alpha][z], centre at the root of every set
    dt: float
    nsteps: int
    meta: dict = field(default_factory=dict)


def multiset_vibronic_problem(n_states: int = 3, n_modes: int = 6, d: int = 6, chi: int = 4,
                              seed: int = 7, dt: float = 0.1, nsteps: int = 50,
                              n_coupling_modes: int = 2, amps=None) -> MultiSetProblem:
    """Linear vibronic coupling model in the multi-set form (the electronic
    states are the sets, the modes the environment tree; the form of the
    exciton models of paper Sec. IV.B), seeded:
      H^{ss}   = E_s + sum_i w_i (n_i + 1/2) + sum_i kappa_i^s Q_i
      H^{ss'}  = J_{ss'} + sum_{i in coupling modes} lam_i^{ss'} Q_i   (s != s', symmetric)
    with w ~ U[0.05, 0.5], E_s ~ N(0, 0.05^2), kappa ~ N(0, 0.05^2),
    J ~ N(0, 0.03^2), lam ~ N(0, 0.03^2), Q = (a + a^+)/sqrt(2), on a balanced
    binary tree over the modes (leaf bonds min(chi, d), interior bonds chi).
    Initial state: sum_s amps[s] |s> x vibrational vacuum; default set 0
    alone (the other sets empty)."""
    rng = np.random.default_rng(seed)
    omega = rng.uniform(0.05, 0.5, n_modes)
    E = rng.normal(0.0, 0.05, n_states)
    kappa = rng.normal(0.0, 0.05, (n_modes, n_states))
    cm = np.sort(rng.choice(n_modes, min(n_coupling_modes, n_modes), replace=False))
    J = rng.normal(0.0, 0.03, (n_states, n_states))
    lam = rng.normal(0.0, 0.03, (len(cm), n_states, n_states))
    leaves = [("leaf", d, min(chi, d), f"m{k}") for k in range(n_modes)]
    spec = balanced_spec(leaves, chi)
    if spec[0] == "leaf":
        spec = ("node", 1, [spec])
    t = build_tree(spec)
    modes = [t.leaf_of_label(f"m{i}") for i in range(n_modes)]
    B = boson_ops(d)
    Q = B["x"] / np.sqrt(2.0)
    num = B["n"] + 0.5 * np.eye(d)
    H = MultiSetSOP(hermitian=True, n_sets=n_states)
    for s_ in range(n_states):
        H.add_set(s_, s_, E[s_])
        for i, leaf in enumerate(modes):
            H.add_set(s_, s_, omega[i], (leaf, num))
            H.add_set(s_, s_, kappa[i, s_], (leaf, Q))
    for s_ in range(n_states):
        for s2 in range(n_states):
            if s2 == s_:
                continue
            a, b = min(s_, s2), max(s_, s2)
            H.add_set(s_, s2, J[a, b])
            for j, i in enumerate(cm):
                H.add_set(s_, s2, lam[j, a, b], (modes[i], Q))
    if amps is None:
        amps = [1.0] + [0.0] * (n_states - 1)
    amps = np.asarray(amps, dtype=np.complex128)
    A = multiset_product_state(t, list(amps / np.linalg.norm(amps)))
    return MultiSetProblem(f"multiset_vibronic_{n_states}x{n_modes}_d{d}_chi{chi}_seed{seed}", t, H, A,
                           dt, nsteps, {"modes": modes, "coupling_modes": cm, "omega": omega, "E": E,
                                        "kappa": kappa, "J": J, "lam": lam, "d": d})


def c5_problem(req: dict) -> Problem:
    """The propagation one serving request asks for: spin-boson (dt 0.05) or
    two-state vibronic (dt 0.1) on a balanced binary tree, with the request's
    modes, local and bond dimensions and step count."""
    if req["kind"] == "sb":
        return spin_boson_star_problem(req["n_modes"], req["d"], req["chi"], req["alpha"], beta=req["beta"],
                                       dt=0.05, nsteps=req["steps"], name=f"req{req['id']}_spin_boson")
    return vibronic_balanced_problem(req["n_modes"], req["d"], req["chi"], req["seed"], dt=0.1,
                                     nsteps=req["steps"])


def config_c5_requests(n_requests: int = 512, seed: int = 5, n_modes_range=(8, 128),
                       d_range=(8, 20), chi_range=(8, 48), steps_range=(100, 400)):
    """Seeded request parameters for the serving stream: half spin-boson
    (alpha ~ U[0.05, 1], beta in {inf, 5, 1}), half two-state vibronic; modes,
    local and bond dimensions and step counts drawn uniformly."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_requests):
        kind = "sb" if rng.random() < 0.5 else "vib"
        reqs.append(dict(
            id=i, kind=kind,
            n_modes=int(rng.integers(n_modes_range[0], n_modes_range[1] + 1)),
            d=int(rng.integers(d_range[0], d_range[1] + 1)),
            chi=int(rng.integers(chi_range[0], chi_range[1] + 1)),
            steps=int(rng.integers(steps_range[0], steps_range[1] + 1)),
            alpha=float(rng.uniform(0.05, 1.0)),
            beta=[np.inf, 5.0, 1.0][int(rng.integers(0, 3))],
            seed=int(rng.integers(0, 2**31 - 1)),
        ))
    return reqs
