// Host-side planning for libttn (see ttn_plan.hpp).
//
// Operator grouping.  For the bond between node c and its parent, every SOP
// term r (paper Eq. sop_ham) splits into the factors inside the subtree of c
// and the factors outside.  Following the node decomposition of Sec. II.B.1
// (Eqs. sop_node_naive, spf_hamiltonian_op, shf_hamiltonian_op) the bond
// carries
//   * up channels   (single-particle operators, Sec. II.C matrices h):
//       LOC  = sum of all terms acting only inside the subtree (one matrix),
//       PROD = the inside part of each term that acts on both sides;
//   * down channels (mean-field operators, matrices H):
//       LOC  = sum of all terms acting only outside the subtree,
//       PROD = the outside part of each term that acts on both sides.
// Each channel's matrix at a node is a sum of products of its children's
// channels, which is what the environment builds evaluate.  Identity
// factors are skipped (the copy optimisation the paper describes for the
// hierarchical SOP form); the result is exactly the plain SOP operator.
#include "ttn_plan.hpp"

#include <algorithm>
#include <cstring>
#include <cmath>
#include <functional>
#include <set>
#include <sstream>
#include <tuple>

namespace ttn {

namespace {

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Minimum vertex cover of a bipartite graph (Konig's theorem): a maximum
// matching by augmenting paths, then Z = the vertices reachable from the
// unmatched left vertices along alternating paths (left to right on
// non-matching edges, right to left on matching ones); the cover is
// (L minus Z) together with (R in Z), its size that of the matching.
// Returns the size and the cover's left part.
size_t min_vertex_cover(const std::set<Key>& L, const std::set<Key>& R, const std::set<std::pair<Key, Key>>& E,
                        std::set<Key>& cover_left) {
    std::vector<Key> lv(L.begin(), L.end()), rv(R.begin(), R.end());
    std::map<Key, int> li, ri;
    for (size_t i = 0; i < lv.size(); ++i) li[lv[i]] = (int)i;
    for (size_t i = 0; i < rv.size(); ++i) ri[rv[i]] = (int)i;
    std::vector<std::vector<int>> adj(lv.size());
    for (auto& e : E) adj[li[e.first]].push_back(ri[e.second]);
    std::vector<int> ml(lv.size(), -1), mr(rv.size(), -1);
    std::vector<char> seen;
    std::function<bool(int)> augment = [&](int u) -> bool {
        for (int v : adj[u]) {
            if (seen[v]) continue;
            seen[v] = 1;
            if (mr[v] < 0 || augment(mr[v])) { ml[u] = v; mr[v] = u; return true; }
        }
        return false;
    };
    for (size_t u = 0; u < lv.size(); ++u) {
        seen.assign(rv.size(), 0);
        augment((int)u);
    }
    std::vector<char> zl(lv.size(), 0), zr(rv.size(), 0);
    std::function<void(int)> walk = [&](int u) {
        zl[u] = 1;
        for (int v : adj[u]) {
            if (zr[v] || ml[u] == v) continue;
            zr[v] = 1;
            if (mr[v] >= 0 && !zl[mr[v]]) walk(mr[v]);
        }
    };
    for (size_t u = 0; u < lv.size(); ++u)
        if (ml[u] < 0 && !zl[u]) walk((int)u);
    size_t size = 0;
    cover_left.clear();
    for (size_t u = 0; u < lv.size(); ++u)
        if (!zl[u]) { cover_left.insert(lv[u]); ++size; }
    for (size_t v = 0; v < rv.size(); ++v) size += zr[v] ? 1 : 0;
    return size;
}

// Smallest eigenvalue of a Hermitian d x d matrix (row-major) by cyclic
// Jacobi rotations (Golub & Van Loan, Sec. 8.5, in the complex form that
// first makes the pivot real).
double min_eig_hermitian(std::vector<cplx> A, int d) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) (i == j ? dia : off) += std::norm(A[i * d + j]);
        if (off <= 1e-30 * (off + dia) || off == 0.0) break;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                const cplx apq = A[p * d + q];
                const double r = std::abs(apq);
                if (r <= 1e-300) continue;
                const double theta = (A[q * d + q].real() - A[p * d + p].real()) / (2.0 * r);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                const cplx e = std::conj(apq) / r;
                for (int row = 0; row < d; ++row) {
                    const cplx ap = A[row * d + p], aq = e * A[row * d + q];
                    A[row * d + p] = c * ap - sn * aq;
                    A[row * d + q] = sn * ap + c * aq;
                }
                const cplx ec = std::conj(e);
                for (int col = 0; col < d; ++col) {
                    const cplx ap = A[p * d + col], aq = ec * A[q * d + col];
                    A[p * d + col] = c * ap - sn * aq;
                    A[q * d + col] = sn * ap + c * aq;
                }
            }
    }
    double m = A[0].real();
    for (int i = 1; i < d; ++i) m = std::min(m, A[i * d + i].real());
    return m;
}

}  // namespace

std::vector<int> Tree::preorder() const {
    std::vector<int> out;
    std::vector<int> st{0};
    while (!st.empty()) {
        int z = st.back(); st.pop_back();
        out.push_back(z);
        for (int i = (int)ch[z].size() - 1; i >= 0; --i) st.push_back(ch[z][i]);
    }
    return out;
}

std::vector<int> Tree::postorder() const {
    std::vector<int> out;
    std::function<void(int)> rec = [&](int z) {
        for (int c : ch[z]) rec(c);
        out.push_back(z);
    };
    rec(0);
    return out;
}

std::string build_tree(int n, const int* parent, const int* phys, const int* bond, Tree& t) {
    std::ostringstream err;
    if (n < 1 || n > 65535) return "n_nodes must be in 1..65535";
    if (!parent || !phys || !bond) return "null tree array";
    t = Tree();
    t.n = n;
    t.parent.assign(parent, parent + n);
    t.phys.assign(phys, phys + n);
    t.bond.assign(bond, bond + n);
    t.ch.assign(n, {});
    if (t.parent[0] != -1) return "parent[0] must be -1";
    for (int i = 1; i < n; ++i) {
        if (t.parent[i] < 0 || t.parent[i] >= i) {
            err << "parent[" << i << "] = " << t.parent[i] << " must be in [0, " << i << ")";
            return err.str();
        }
        t.ch[t.parent[i]].push_back(i);
    }
    t.bond[0] = 1;
    for (int z = 0; z < n; ++z) {
        if (t.phys[z] < 0) return "negative phys_dim";
        if (t.phys[z] > 0 && !t.ch[z].empty()) { err << "node " << z << " has children and phys_dim > 0"; return err.str(); }
        if (t.phys[z] == 0 && t.ch[z].empty()) { err << "interior node " << z << " has no children"; return err.str(); }
        if (t.phys[z] > TTN_MAXCHI) { err << "phys_dim of node " << z << " exceeds " << TTN_MAXCHI; return err.str(); }
        if (z > 0 && (t.bond[z] < 1 || t.bond[z] > TTN_MAXCHI)) { err << "bond_dim of node " << z << " must be in 1.." << TTN_MAXCHI; return err.str(); }
        if ((int)t.ch[z].size() + 1 > TTN_MAXD) { err << "node " << z << " has more than " << TTN_MAXD - 1 << " children"; return err.str(); }
    }
    t.dims.assign(n, {});
    t.size.assign(n, 0);
    for (int z = 0; z < n; ++z) {
        if (t.leaf(z)) t.dims[z].push_back(t.phys[z]);
        else for (int c : t.ch[z]) t.dims[z].push_back(t.bond[c]);
        t.dims[z].push_back(z == 0 ? 1 : t.bond[z]);
        int64_t s = 1;
        for (int d : t.dims[z]) s *= d;
        t.size[z] = s;
        if (s > (int64_t(1) << 28)) { err << "tensor of node " << z << " is too large"; return err.str(); }
        // every matricisation used by the sweep needs rows >= columns
        for (size_t k = 0; k < t.dims[z].size(); ++k) {
            if (z == 0 && k + 1 == t.dims[z].size()) continue;   // root's dummy index
            if (t.leaf(z) && k == 0) continue;                   // a leaf is never split along its physical index
            if (s / t.dims[z][k] < t.dims[z][k]) {
                err << "node " << z << ": index " << k << " of dimension " << t.dims[z][k]
                    << " exceeds the product " << s / t.dims[z][k] << " of the other indices";
                return err.str();
            }
        }
    }
    // Euler tour
    t.tin.assign(n, 0); t.tout.assign(n, 0);
    int clock = 0;
    std::function<void(int)> rec = [&](int z) {
        t.tin[z] = clock++;
        for (int c : t.ch[z]) rec(c);
        t.tout[z] = clock;
    };
    rec(0);
    return "";
}

std::string build_hamiltonian(const Tree& t, int n_terms, const cplx* coeff, const int* term_ptr,
                              const int* factor_leaf, const cplx* mats, const int64_t* mat_off,
                              int hermitian, Hamiltonian& h, int n_sets, const int* bra, const int* ket) {
    std::ostringstream err;
    if (n_terms < 1) return "n_terms must be >= 1";
    if (!coeff || !term_ptr) return "null coefficient / term_ptr";
    if (term_ptr[0] != 0) return "term_ptr[0] must be 0";
    if (n_sets < 1 || n_sets > TTN_MAX_SETS) return "n_sets must be in 1.." + std::to_string(TTN_MAX_SETS);
    if (n_sets > 1 && (!bra || !ket)) return "a multi-set operator needs bra and ket set indices";
    h = Hamiltonian();
    h.hermitian = hermitian != 0;
    h.n_sets = n_sets;
    std::map<std::pair<int, std::vector<double>>, int> dedup;
    for (int r = 0; r < n_terms; ++r) {
        if (term_ptr[r + 1] < term_ptr[r]) return "term_ptr must be non-decreasing";
        if (!std::isfinite(coeff[r].real()) || !std::isfinite(coeff[r].imag())) return "non-finite coefficient";
        Key key;
        for (int f = term_ptr[r]; f < term_ptr[r + 1]; ++f) {
            int l = factor_leaf[f];
            if (l < 0 || l >= t.n || !t.leaf(l)) { err << "factor " << f << " acts on node " << l << ", which is not a leaf"; return err.str(); }
            int d = t.phys[l];
            std::vector<double> raw(2 * d * d);
            for (int i = 0; i < d * d; ++i) {
                cplx v = mats[mat_off[f] + i];
                if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return "non-finite factor matrix entry";
                raw[2 * i] = v.real(); raw[2 * i + 1] = v.imag();
            }
            auto it = dedup.find({d, raw});
            int id;
            if (it == dedup.end()) {
                id = (int)h.mats.size();
                h.mats.emplace_back(mats + mat_off[f], mats + mat_off[f] + d * d);
                h.mat_dim.push_back(d);
                dedup[{d, raw}] = id;
            } else id = it->second;
            key.push_back({l, id});
        }
        std::sort(key.begin(), key.end());
        for (size_t i = 1; i < key.size(); ++i)
            if (key[i].first == key[i - 1].first) { err << "term " << r << " has two factors on leaf " << key[i].first; return err.str(); }
        if (n_sets > 1 && (bra[r] < 0 || bra[r] >= n_sets || ket[r] < 0 || ket[r] >= n_sets)) {
            err << "term " << r << " names a set outside 0.." << n_sets - 1; return err.str();
        }
        if (coeff[r] == cplx(0.0)) continue;
        h.coeff.push_back(coeff[r]);
        h.terms.push_back(key);
        if (n_sets > 1) { h.bra.push_back(bra[r]); h.ket.push_back(ket[r]); }
    }
    if (h.coeff.empty()) {
        h.coeff.push_back(0.0); h.terms.push_back({});
        if (n_sets > 1) { h.bra.push_back(0); h.ket.push_back(0); }
    }
    return "";
}

// ---------------------------------------------------------------------------
// Operator planning
// ---------------------------------------------------------------------------
namespace {

struct Proto {
    cplx w;
    int out;
    std::vector<int> slot;
    int src = 0, dst = 0;   // multi-set: ket and bra set of the entry
};

struct Builder {
    const Tree& t;
    const Hamiltonian* h;
    Plan& p;
    // Grouping direction per bond (edge to the parent): terms acting on both
    // sides of the bond are summed either by their common outside factor
    // (UPGRP: the up channel is sum_r c_r (inside part of r), paper Sec.
    // II.B.2 term (C)) or by their common inside factor (DNGRP: the down
    // channel is the sum of outside parts, term (B)), whichever gives fewer
    // channels.
    // MIXED: the terms crossing the bond are assigned term by term from a
    // minimum vertex cover of the bipartite graph whose vertices are their
    // distinct inside parts and outside parts and whose edges are the terms
    // (the hierarchical-SOP construction of Sec. II.B.2): a term whose inside
    // part is in the cover is summed into that part's down channel, every
    // other term into its outside part's up channel (whose vertex the cover
    // then holds).  Used where this needs fewer channels than either uniform
    // direction.
    enum { NONE = 0, UPGRP = 1, DNGRP = 2, MIXED = 3 };
    std::vector<int> dir;
    std::vector<std::set<Key>> dn_cover;          // MIXED bonds: inside parts in the cover
    std::vector<char> has_in, has_out;           // some term entirely inside / outside the subtree
    std::vector<int> up_loc, down_loc, phys_loc;
    std::vector<std::map<Key, int>> up_prod, down_prod, up_grp, down_grp, phys_grp;
    std::vector<std::map<int, int>> phys_mat;
    struct Pending { int kind; int c; Key key; int slot; };
    enum { K_UP_LOC, K_UP_PROD, K_UP_GRP, K_DOWN_LOC, K_DOWN_PROD, K_DOWN_GRP };
    std::vector<Pending> todo;
    std::vector<std::vector<Proto>> up_entries, down_entries;   // per bond
    int one_slot = -1;     // 1x1 matrix holding 1 (root Gram matrix)

    Builder(const Tree& t_, const Hamiltonian* h_, Plan& p_) : t(t_), h(h_), p(p_) {}

    int new_slot(int rows, int cols) {
        SlotInfo s; s.rows = rows; s.cols = cols;
        p.slots.push_back(s);
        return (int)p.slots.size() - 1;
    }
    int const_slot(int rows, int cols, const std::vector<cplx>& data) {
        int id = new_slot(rows, cols);
        p.slots[id].constant = true;
        p.slots[id].data = data;
        return id;
    }
    Key restrict_to(const Key& k, int c, bool inside) const {
        Key out;
        for (auto& f : k) if (t.in_sub(f.first, c) == inside) out.push_back(f);
        return out;
    }
    // mode of node z that leaf l falls into: child index, 0 for the leaf itself, D-1 outside
    int mode_of(int z, int l) const {
        int D = (int)t.dims[z].size();
        if (!t.in_sub(l, z)) return D - 1;
        if (t.leaf(z)) return 0;
        for (size_t k = 0; k < t.ch[z].size(); ++k)
            if (t.in_sub(l, t.ch[z][k])) return (int)k;
        return -1;
    }
    Key restrict_mode(int z, const Key& key, int mode) const {
        Key out;
        for (auto& f : key) if (mode_of(z, f.first) == mode) out.push_back(f);
        return out;
    }
    std::set<int> modes_of(int z, const Key& key) const {
        std::set<int> m;
        for (auto& f : key) m.insert(mode_of(z, f.first));
        return m;
    }

    // Assignment of a term crossing bond c (its key restricted to both sides
    // of the bond is non-empty): summed by its outside part (up group) or by
    // its inside part (down group).
    bool up_at(int c, const Key& key) const {
        if (dir[c] == UPGRP) return true;
        if (dir[c] != MIXED) return false;
        return dn_cover[c].count(restrict_to(key, c, true)) == 0;
    }
    bool dn_at(int c, const Key& key) const {
        if (dir[c] == DNGRP) return true;
        if (dir[c] != MIXED) return false;
        return dn_cover[c].count(restrict_to(key, c, true)) != 0;
    }
    // The up group of child bond ck for outside part E may stand for its
    // members inside the up group being defined at bond c only if every one
    // of its members belongs there too (true unless bond c is MIXED).
    bool child_group_within(int ck, const Key& E, int c) const {
        if (dir[c] != MIXED) return true;
        for (const Key& key : h->terms) {
            if (key.empty() || restrict_to(key, ck, true).empty() || restrict_to(key, ck, false) != E) continue;
            if (!up_at(ck, key)) continue;
            if (!up_at(c, key)) return false;
        }
        return true;
    }

    // ---- channels (created on first use, defined by the closure loop) -----
    int chan(std::map<Key, int>& m, int kind, int c, const Key& key) {
        auto it = m.find(key);
        if (it != m.end()) return it->second;
        int s = new_slot(t.bond[c], t.bond[c]);
        m[key] = s;
        todo.push_back({kind, c, key, s});
        return s;
    }
    int get_up_prod(int c, const Key& key) { return chan(up_prod[c], K_UP_PROD, c, key); }
    int get_down_prod(int c, const Key& key) { return chan(down_prod[c], K_DOWN_PROD, c, key); }
    int get_up_grp(int c, const Key& key) { return chan(up_grp[c], K_UP_GRP, c, key); }
    int get_down_grp(int c, const Key& key) { return chan(down_grp[c], K_DOWN_GRP, c, key); }
    int get_up_loc(int c) {
        if (up_loc[c] < 0) { up_loc[c] = new_slot(t.bond[c], t.bond[c]); todo.push_back({K_UP_LOC, c, {}, up_loc[c]}); }
        return up_loc[c];
    }
    int get_down_loc(int c) {
        if (down_loc[c] < 0) { down_loc[c] = new_slot(t.bond[c], t.bond[c]); todo.push_back({K_DOWN_LOC, c, {}, down_loc[c]}); }
        return down_loc[c];
    }
    int get_phys_mat(int l, int m) {
        auto it = phys_mat[l].find(m);
        if (it != phys_mat[l].end()) return it->second;
        int d = t.phys[l];
        return phys_mat[l][m] = const_slot(d, d, h->mats[m]);
    }
    // sum_{r: straddling leaf l, outside part == D} c_r M_r  (constant)
    int get_phys_grp(int l, const Key& D) {
        auto it = phys_grp[l].find(D);
        if (it != phys_grp[l].end()) return it->second;
        int d = t.phys[l];
        std::vector<cplx> sum(d * d, 0.0);
        for (size_t r = 0; r < h->terms.size(); ++r) {
            const Key& key = h->terms[r];
            Key in = restrict_to(key, l, true), out = restrict_to(key, l, false);
            if (in.empty() || out != D || !up_at(l, key)) continue;
            for (int i = 0; i < d * d; ++i) sum[i] += h->coeff[r] * h->mats[in[0].second][i];
        }
        return phys_grp[l][D] = const_slot(d, d, sum);
    }
    // up channel on mode k of node z for an individual inside part
    int child_up_prod(int z, int k, const Key& part) {
        if (t.leaf(z)) return get_phys_mat(z, part.at(0).second);
        return get_up_prod(t.ch[z][k], part);
    }

    // Accumulator for one operator: group entries are added once (their
    // coefficients live in the group channel), individual entries are summed.
    struct Acc {
        std::set<std::vector<int>> grp;
        std::map<std::vector<int>, cplx> ind;
        void add(bool group, const std::vector<int>& s, cplx w) {
            if (group) grp.insert(s);
            else ind[s] += w;
        }
        std::vector<Proto> out(int out_slot) const {
            std::vector<Proto> es;
            for (auto& s : grp) { Proto e; e.w = 1.0; e.out = out_slot; e.slot = s; es.push_back(e); }
            for (auto& kv : ind) {
                if (kv.second == cplx(0.0)) continue;
                Proto e; e.w = kv.second; e.out = out_slot; e.slot = kv.first; es.push_back(e);
            }
            return es;
        }
    };

    // Entry of term `key` (coefficient w) on node z when it touches >= 2 of
    // z's modes.  The choice depends only on the set of touched modes, so
    // every member of a group channel is routed to the same entry.
    void term_entry(int z, const Key& key, cplx w, Acc& acc) {
        const int D = (int)t.dims[z].size(), P = D - 1;
        std::set<int> T = modes_of(z, key);
        std::vector<int> sl(D, -1);
        auto fill_rest = [&](int skip_mode) {
            for (int j : T) {
                if (j == skip_mode) continue;
                Key part = restrict_mode(z, key, j);
                sl[j] = (j == P) ? get_down_prod(z, part) : child_up_prod(z, j, part);
            }
        };
        if (t.leaf(z)) {
            // modes {0 (physical), P}
            if (up_at(z, key)) {
                Key Dk = restrict_to(key, z, false);
                sl[0] = get_phys_grp(z, Dk);
                sl[P] = get_down_prod(z, Dk);
                acc.add(true, sl, 1.0);
                return;
            }
            if (dn_at(z, key)) {
                Key U = restrict_to(key, z, true);
                sl[P] = get_down_grp(z, U);
                sl[0] = get_phys_mat(z, U.at(0).second);
                acc.add(true, sl, 1.0);
                return;
            }
            fill_rest(-1);
            acc.add(false, sl, w);
            return;
        }
        for (int k : T) {
            if (k == P || !up_at(t.ch[z][k], key)) continue;
            int c = t.ch[z][k];
            sl[k] = get_up_grp(c, restrict_to(key, c, false));
            fill_rest(k);
            acc.add(true, sl, 1.0);
            return;
        }
        if (T.count(P) && z > 0 && dn_at(z, key)) {
            sl[P] = get_down_grp(z, restrict_to(key, z, true));
            fill_rest(P);
            acc.add(true, sl, 1.0);
            return;
        }
        fill_rest(-1);
        acc.add(false, sl, w);
    }

    void define(const Pending& q) {
        const int c = q.c;
        const int R = (int)h->terms.size();
        Acc acc;
        if (q.kind == K_UP_LOC || q.kind == K_UP_PROD || q.kind == K_UP_GRP) {
            // built at node c from its children (or its physical index)
            const int D = (int)t.dims[c].size();
            std::vector<int> sl(D, -1);
            if (q.kind == K_UP_LOC) {
                if (t.leaf(c)) { sl[0] = phys_loc[c]; acc.add(true, sl, 1.0); }
                else {
                    for (size_t k = 0; k < t.ch[c].size(); ++k)
                        if (has_in[t.ch[c][k]]) { std::vector<int> s2(D, -1); s2[k] = get_up_loc(t.ch[c][k]); acc.add(true, s2, 1.0); }
                    for (int r = 0; r < R; ++r) {
                        const Key& key = h->terms[r];
                        if (key.empty() || !restrict_to(key, c, false).empty()) continue;
                        if (modes_of(c, key).size() < 2) continue;
                        term_entry(c, key, h->coeff[r], acc);
                    }
                }
            } else if (q.kind == K_UP_PROD) {
                if (t.leaf(c)) sl[0] = get_phys_mat(c, q.key.at(0).second);
                else for (int k : modes_of(c, q.key)) sl[k] = get_up_prod(t.ch[c][k], restrict_mode(c, q.key, k));
                acc.add(true, sl, 1.0);
            } else {  // K_UP_GRP: sum_{r: out^c_r == key} c_r (inside part)
                if (t.leaf(c)) { sl[0] = get_phys_grp(c, q.key); acc.add(true, sl, 1.0); }
                else {
                    for (int r = 0; r < R; ++r) {
                        const Key& key = h->terms[r];
                        Key in = restrict_to(key, c, true);
                        if (in.empty() || restrict_to(key, c, false) != q.key || !up_at(c, key)) continue;
                        std::set<int> T = modes_of(c, in);
                        std::vector<int> s2(D, -1);
                        if (T.size() == 1) {
                            int k = *T.begin();
                            int ck = t.ch[c][k];
                            if (up_at(ck, key) && child_group_within(ck, q.key, c)) { s2[k] = get_up_grp(ck, q.key); acc.add(true, s2, 1.0); }
                            else { s2[k] = get_up_prod(ck, in); acc.add(false, s2, h->coeff[r]); }
                            continue;
                        }
                        bool done = false;
                        for (int k : T) {
                            int ck = t.ch[c][k];
                            if (!up_at(ck, key)) continue;
                            // the first child where the term is grouped; its group only
                            // if all of the group's members belong to this channel
                            if (!child_group_within(ck, restrict_to(key, ck, false), c)) break;
                            s2[k] = get_up_grp(ck, restrict_to(key, ck, false));
                            for (int j : T) if (j != k) s2[j] = get_up_prod(t.ch[c][j], restrict_mode(c, in, j));
                            acc.add(true, s2, 1.0);
                            done = true;
                            break;
                        }
                        if (!done) {
                            for (int j : T) s2[j] = get_up_prod(t.ch[c][j], restrict_mode(c, in, j));
                            acc.add(false, s2, h->coeff[r]);
                        }
                    }
                }
            }
            auto es = acc.out(q.slot);
            up_entries[c].insert(up_entries[c].end(), es.begin(), es.end());
            return;
        }
        // down channels of bond c: built at its parent z (child index k)
        const int z = t.parent[c];
        const int k = (int)(std::find(t.ch[z].begin(), t.ch[z].end(), c) - t.ch[z].begin());
        const int D = (int)t.dims[z].size(), P = D - 1;
        if (q.kind == K_DOWN_LOC) {
            if (z > 0 && has_out[z]) { std::vector<int> s2(D, -1); s2[P] = get_down_loc(z); acc.add(true, s2, 1.0); }
            for (size_t j = 0; j < t.ch[z].size(); ++j)
                if ((int)j != k && has_in[t.ch[z][j]]) { std::vector<int> s2(D, -1); s2[j] = get_up_loc(t.ch[z][j]); acc.add(true, s2, 1.0); }
            for (int r = 0; r < R; ++r) {
                const Key& key = h->terms[r];
                if (key.empty() || !restrict_to(key, c, true).empty()) continue;
                if (modes_of(z, key).size() < 2) continue;
                term_entry(z, key, h->coeff[r], acc);
            }
        } else if (q.kind == K_DOWN_PROD) {
            std::vector<int> s2(D, -1);
            for (int j : modes_of(z, q.key)) {
                Key part = restrict_mode(z, q.key, j);
                s2[j] = (j == P) ? get_down_prod(z, part) : get_up_prod(t.ch[z][j], part);
            }
            acc.add(true, s2, 1.0);
        } else {  // K_DOWN_GRP: sum_{r: in^c_r == key} c_r (outside part)
            for (int r = 0; r < R; ++r) {
                const Key& key = h->terms[r];
                Key out = restrict_to(key, c, false);
                if (out.empty() || restrict_to(key, c, true) != q.key || !dn_at(c, key)) continue;
                std::set<int> T = modes_of(z, out);
                std::vector<int> s2(D, -1);
                if (T.size() == 1) {
                    int j = *T.begin();
                    if (j == P) {
                        if (z > 0 && dn_at(z, key)) { s2[P] = get_down_grp(z, q.key); acc.add(true, s2, 1.0); }
                        else { s2[P] = get_down_prod(z, out); acc.add(false, s2, h->coeff[r]); }
                    } else {
                        int cj = t.ch[z][j];
                        if (up_at(cj, key)) { s2[j] = get_up_grp(cj, q.key); acc.add(true, s2, 1.0); }
                        else { s2[j] = get_up_prod(cj, out); acc.add(false, s2, h->coeff[r]); }
                    }
                    continue;
                }
                bool done = false;
                for (int j : T) {
                    if (j == P || !up_at(t.ch[z][j], key)) continue;
                    int cj = t.ch[z][j];
                    s2[j] = get_up_grp(cj, restrict_to(key, cj, false));
                    for (int i : T) if (i != j) { Key part = restrict_mode(z, out, i); s2[i] = (i == P) ? get_down_prod(z, part) : get_up_prod(t.ch[z][i], part); }
                    acc.add(true, s2, 1.0);
                    done = true;
                    break;
                }
                if (!done && T.count(P) && z > 0 && dn_at(z, key)) {
                    s2[P] = get_down_grp(z, restrict_to(key, z, true));
                    for (int i : T) if (i != P) s2[i] = get_up_prod(t.ch[z][i], restrict_mode(z, out, i));
                    acc.add(true, s2, 1.0);
                    done = true;
                }
                if (!done) {
                    for (int i : T) { Key part = restrict_mode(z, out, i); s2[i] = (i == P) ? get_down_prod(z, part) : get_up_prod(t.ch[z][i], part); }
                    acc.add(false, s2, h->coeff[r]);
                }
            }
        }
        auto es = acc.out(q.slot);
        down_entries[c].insert(down_entries[c].end(), es.begin(), es.end());
    }

    void close() {
        while (!todo.empty()) {
            Pending q = todo.back();
            todo.pop_back();
            define(q);
        }
    }

    void make_channels() {
        int n = t.n;
        dir.assign(n, NONE);
        has_in.assign(n, 0); has_out.assign(n, 0);
        up_loc.assign(n, -1); down_loc.assign(n, -1); phys_loc.assign(n, -1);
        up_prod.assign(n, {}); down_prod.assign(n, {}); up_grp.assign(n, {}); down_grp.assign(n, {});
        phys_grp.assign(n, {}); phys_mat.assign(n, {});
        up_entries.assign(n, {}); down_entries.assign(n, {});
        if (!h) return;
        const int R = (int)h->terms.size();
        std::vector<std::vector<cplx>> loc_sum(n);
        for (int r = 0; r < R; ++r) {
            const Key& key = h->terms[r];
            if (key.size() == 1) {
                int l = key[0].first, d = t.phys[l];
                if (loc_sum[l].empty()) loc_sum[l].assign(d * d, 0.0);
                for (int i = 0; i < d * d; ++i) loc_sum[l][i] += h->coeff[r] * h->mats[key[0].second][i];
            }
        }
        for (int l = 0; l < n; ++l) {
            if (loc_sum[l].empty()) continue;
            if (p.esz == 8 && h->hermitian) {      // complex64 bulk: store excitation energies
                const int d = t.phys[l];
                const double lam = min_eig_hermitian(loc_sum[l], d);
                for (int i = 0; i < d; ++i) loc_sum[l][i * d + i] -= lam;
                p.e_shift += lam;
            }
            phys_loc[l] = const_slot(t.phys[l], t.phys[l], loc_sum[l]);
        }
        dn_cover.assign(n, {});
        for (int c = 1; c < n; ++c) {
            std::set<Key> ins, outs;
            std::set<std::pair<Key, Key>> edges;
            for (int r = 0; r < R; ++r) {
                const Key& key = h->terms[r];
                if (key.empty()) continue;
                Key in = restrict_to(key, c, true), out = restrict_to(key, c, false);
                if (!in.empty() && out.empty()) has_in[c] = 1;
                else if (in.empty() && !out.empty()) has_out[c] = 1;
                else { ins.insert(in); outs.insert(out); edges.insert({in, out}); }
            }
            if (ins.empty()) continue;
            std::set<Key> cov_in;
            const size_t mvc = min_vertex_cover(ins, outs, edges, cov_in);
            if (mvc < std::min(ins.size(), outs.size())) {
                dir[c] = MIXED;
                dn_cover[c] = cov_in;
            } else {
                dir[c] = outs.size() <= ins.size() ? UPGRP : DNGRP;
            }
        }
    }

    // ---- operator entry lists ------------------------------------------------
    std::vector<Proto> heff_terms(int z) {
        Acc acc;
        const int D = (int)t.dims[z].size(), P = D - 1;
        int nchild = t.leaf(z) ? 1 : (int)t.ch[z].size();
        for (int k = 0; k < nchild; ++k) {
            std::vector<int> sl(D, -1);
            if (t.leaf(z)) { if (phys_loc[z] < 0) continue; sl[0] = phys_loc[z]; }
            else { if (!has_in[t.ch[z][k]]) continue; sl[k] = get_up_loc(t.ch[z][k]); }
            acc.add(true, sl, 1.0);
        }
        if (z > 0 && has_out[z]) { std::vector<int> sl(D, -1); sl[P] = get_down_loc(z); acc.add(true, sl, 1.0); }
        for (size_t r = 0; r < h->terms.size(); ++r) {
            const Key& key = h->terms[r];
            if (key.empty()) { acc.add(false, std::vector<int>(D, -1), h->coeff[r]); continue; }
            if (modes_of(z, key).size() < 2) continue;
            term_entry(z, key, h->coeff[r], acc);
        }
        return acc.out(-1);
    }

    std::vector<Proto> bond_terms(int c) {
        Acc acc;
        if (has_in[c]) acc.add(true, {get_up_loc(c), -1}, 1.0);
        if (has_out[c]) acc.add(true, {-1, get_down_loc(c)}, 1.0);
        for (size_t r = 0; r < h->terms.size(); ++r) {
            const Key& key = h->terms[r];
            if (key.empty()) { acc.add(false, {-1, -1}, h->coeff[r]); continue; }
            Key in = restrict_to(key, c, true), out = restrict_to(key, c, false);
            if (in.empty() || out.empty()) continue;
            if (up_at(c, key)) acc.add(true, {get_up_grp(c, out), get_down_prod(c, out)}, 1.0);
            else if (dn_at(c, key)) acc.add(true, {get_up_prod(c, in), get_down_grp(c, in)}, 1.0);
            else acc.add(false, {get_up_prod(c, in), get_down_prod(c, out)}, h->coeff[r]);
        }
        return acc.out(-1);
    }

    // Repeatedly combine entries that differ in exactly one mode into one
    // entry whose factor on that mode is a linear combination (a "combo"
    // slot, evaluated by COMBO ops right before the operator is applied).
    std::vector<Proto> combine(std::vector<Proto> es, const std::vector<int>& dims,
                               std::vector<std::vector<Proto>>& combo_rounds) {
        int D = (int)dims.size();
        for (int round = 0; round < 4 * D; ++round) {
            int best = -1; size_t best_gain = 0;
            for (int j = 0; j < D; ++j) {
                std::map<std::pair<int, std::vector<int>>, size_t> cnt;
                for (auto& e : es) {
                    auto s = e.slot; s[j] = -2;
                    cnt[{e.out, s}]++;
                }
                size_t gain = 0;
                for (auto& kv : cnt) gain += kv.second - 1;
                if (gain > best_gain) { best_gain = gain; best = j; }
            }
            if (best < 0) break;
            std::map<std::pair<int, std::vector<int>>, std::vector<size_t>> groups;
            for (size_t i = 0; i < es.size(); ++i) {
                auto s = es[i].slot; s[best] = -2;
                groups[{es[i].out, s}].push_back(i);
            }
            std::vector<Proto> next, combos;
            for (auto& kv : groups) {
                if (kv.second.size() == 1) { next.push_back(es[kv.second[0]]); continue; }
                int cs = new_slot(dims[best], dims[best]);
                for (size_t i : kv.second) {
                    Proto ce; ce.w = es[i].w; ce.out = cs; ce.slot.assign(1, es[i].slot[best]);
                    combos.push_back(ce);
                }
                Proto ne = es[kv.second[0]];
                ne.w = 1.0; ne.slot[best] = cs;
                next.push_back(ne);
            }
            es.swap(next);
            combo_rounds.push_back(combos);
        }
        return es;
    }

    // ---- emission -----------------------------------------------------------
    // Entries are ordered by output slot, then by their last factor (mode,
    // slot) so that the device can share the last factor within a run.
    std::pair<int, int> push_entries(const std::vector<Proto>& es) {
        int e0 = (int)p.entries.size();
        std::vector<Proto> sorted = es;
        auto last = [](const Proto& e) {
            int lm = -1;
            for (size_t j = 0; j < e.slot.size(); ++j) if (e.slot[j] >= 0) lm = (int)j;
            return std::make_pair(lm, lm >= 0 ? e.slot[lm] : -1);
        };
        std::stable_sort(sorted.begin(), sorted.end(), [&](const Proto& a, const Proto& b) {
            if (a.out != b.out) return a.out < b.out;
            return last(a) < last(b);
        });
        for (auto& e : sorted) {
            TtnEntry te{};
            te.wr = e.w.real(); te.wi = e.w.imag(); te.out = e.out;
            for (int j = 0; j < TTN_MAXD; ++j) te.slot[j] = j < (int)e.slot.size() ? e.slot[j] : -1;
            p.entries.push_back(te);
        }
        return {e0, (int)sorted.size()};
    }

    OpSpec tensor_op(int type, int z, int k) {
        OpSpec s;
        std::memset(&s.op, 0, sizeof(TtnOp));
        s.op.type = type;
        s.op.D = (int)t.dims[z].size();
        for (int j = 0; j < s.op.D; ++j) s.op.dims[j] = t.dims[z][j];
        s.op.k = k;
        s.a_off = p.tensor_off[z];
        return s;
    }
    OpSpec bond_op(int type, int c) {
        OpSpec s;
        std::memset(&s.op, 0, sizeof(TtnOp));
        s.op.type = type;
        s.op.D = 2;
        s.op.dims[0] = s.op.dims[1] = t.bond[c];
        s.a_off = p.bond_off;
        return s;
    }

    // cached per-node / per-bond operator entry ranges
    std::vector<std::vector<std::pair<int, int>>> heff_combo, bond_combo;
    std::vector<std::pair<int, int>> heff_rng, bond_rng, up_rng, bond_raw_rng;
    std::vector<std::vector<std::pair<int, int>>> down_rng;

    void prepare_entries() {
        int n = t.n;
        heff_combo.assign(n, {}); bond_combo.assign(n, {});
        heff_rng.assign(n, {0, 0}); bond_rng.assign(n, {0, 0}); up_rng.assign(n, {0, 0});
        bond_raw_rng.assign(n, {0, 0});
        down_rng.assign(n, {});
        std::vector<std::vector<Proto>> heff(n), bond(n);
        p.op_bond_dim.assign(n, 0);
        for (int z = 0; z < n; ++z) {
            heff[z] = heff_terms(z);
            if (z > 0) bond[z] = bond_terms(z);
        }
        close();
        for (int z = 0; z < n; ++z) {
            std::vector<std::vector<Proto>> rounds;
            auto es = combine(heff[z], t.dims[z], rounds);
            for (auto& rd : rounds) heff_combo[z].push_back(push_entries(rd));
            heff_rng[z] = push_entries(es);
            if (z > 0) {
                std::vector<std::vector<Proto>> br;
                auto bs = combine(bond[z], {t.bond[z], t.bond[z]}, br);
                for (auto& rd : br) bond_combo[z].push_back(push_entries(rd));
                bond_rng[z] = push_entries(bs);
                bond_raw_rng[z] = push_entries(bond[z]);
                p.op_bond_dim[z] = (int)bond[z].size();
                up_rng[z] = push_entries(up_entries[z]);
            }
        }
        for (int z = 0; z < n; ++z) {
            if (t.leaf(z)) continue;
            for (size_t k = 0; k < t.ch[z].size(); ++k) down_rng[z].push_back(push_entries(down_entries[t.ch[z][k]]));
        }
    }

    void emit_combos(Program& pr, const std::vector<std::pair<int, int>>& rounds) {
        for (auto& rg : rounds) {
            if (rg.second == 0) continue;
            OpSpec s;
            std::memset(&s.op, 0, sizeof(TtnOp));
            s.op.type = TTN_OP_COMBO; s.op.e0 = rg.first; s.op.ne = rg.second;
            pr.ops.push_back(s);
        }
    }
    void emit_env_up(Program& pr, int c) {
        if (up_rng[c].second == 0) return;
        OpSpec s = tensor_op(TTN_OP_ENV, c, (int)t.dims[c].size() - 1);
        s.op.e0 = up_rng[c].first; s.op.ne = up_rng[c].second;
        pr.ops.push_back(s);
    }
    void emit_env_down(Program& pr, int z, int k) {
        auto rg = down_rng[z][k];
        if (rg.second == 0) return;
        OpSpec s = tensor_op(TTN_OP_ENV, z, k);
        s.op.e0 = rg.first; s.op.ne = rg.second;
        pr.ops.push_back(s);
    }
    void emit_evolve_node(Program& pr, int z) {
        emit_combos(pr, heff_combo[z]);
        OpSpec s = tensor_op(TTN_OP_EVOLVE, z, 0);
        s.op.e0 = heff_rng[z].first; s.op.ne = heff_rng[z].second;
        s.op.hermitian = h->hermitian ? 1 : 0;
        s.op.tau_coef = 0.5;
        pr.ops.push_back(s);
    }
    void emit_evolve_bond(Program& pr, int c) {
        emit_combos(pr, bond_combo[c]);
        OpSpec s = bond_op(TTN_OP_EVOLVE, c);
        s.op.e0 = bond_rng[c].first; s.op.ne = bond_rng[c].second;
        s.op.hermitian = h->hermitian ? 1 : 0;
        s.op.tau_coef = -0.5;                    // exp(+i dt/2 K): backward bond step
        pr.ops.push_back(s);
    }
    void emit_qr_down(Program& pr, int z, int k) {
        OpSpec s = tensor_op(TTN_OP_QR_DOWN, z, k);
        s.b_off = p.bond_off;
        pr.ops.push_back(s);
    }
    void emit_qr_up(Program& pr, int c) {
        OpSpec s = tensor_op(TTN_OP_QR_UP, c, (int)t.dims[c].size() - 1);
        s.b_off = p.bond_off;
        pr.ops.push_back(s);
    }
    void emit_absorb_child(Program& pr, int c) {
        OpSpec s = tensor_op(TTN_OP_ABSORB_CHILD, c, (int)t.dims[c].size() - 1);
        s.b_off = p.bond_off;
        pr.ops.push_back(s);
    }
    void emit_absorb_parent(Program& pr, int z, int k) {
        OpSpec s = tensor_op(TTN_OP_ABSORB_PARENT, z, k);
        s.b_off = p.bond_off;
        pr.ops.push_back(s);
    }

    // Recursive projector-splitting sweeps (paper Sec. II.C): S visits the
    // children in index order and updates the node last; S* is its adjoint.
    void emit_S(Program& pr, int z) {
        for (size_t k = 0; k < t.ch[z].size(); ++k) {
            int c = t.ch[z][k];
            emit_qr_down(pr, z, (int)k);
            emit_absorb_child(pr, c);
            emit_env_down(pr, z, (int)k);
            emit_S(pr, c);
            emit_qr_up(pr, c);
            emit_env_up(pr, c);
            emit_evolve_bond(pr, c);
            emit_absorb_parent(pr, z, (int)k);
        }
        emit_evolve_node(pr, z);
    }
    void emit_Sstar(Program& pr, int z) {
        emit_evolve_node(pr, z);
        for (int k = (int)t.ch[z].size() - 1; k >= 0; --k) {
            int c = t.ch[z][k];
            emit_qr_down(pr, z, k);
            emit_env_down(pr, z, k);
            emit_evolve_bond(pr, c);
            emit_absorb_child(pr, c);
            emit_Sstar(pr, c);
            emit_qr_up(pr, c);
            emit_env_up(pr, c);
            emit_absorb_parent(pr, z, k);
        }
    }

    // One-site ground-state sweep (tree DMRG; the paper lists it beside the
    // time evolution, Sec. I and Sec. II.C): the visiting order of S with
    // the centre moved by QR and every node replaced by the lowest
    // eigenvector of its effective Hamiltonian; no bond step.  The root's
    // eigenvalue (the energy of the normalised state) lands in the scalar
    // area at byte offset 64.
    void emit_eigen_node(Program& pr, int z) {
        emit_combos(pr, heff_combo[z]);
        OpSpec s = tensor_op(TTN_OP_EIGEN, z, 0);
        s.op.e0 = heff_rng[z].first; s.op.ne = heff_rng[z].second;
        s.op.hermitian = 1;
        s.out_off = p.scal_off + 64;
        pr.ops.push_back(s);
    }
    void emit_ground(Program& pr, int z) {
        for (size_t k = 0; k < t.ch[z].size(); ++k) {
            int c = t.ch[z][k];
            emit_qr_down(pr, z, (int)k);
            emit_absorb_child(pr, c);
            emit_env_down(pr, z, (int)k);
            emit_ground(pr, c);
            emit_qr_up(pr, c);
            emit_env_up(pr, c);
            emit_absorb_parent(pr, z, (int)k);
        }
        emit_eigen_node(pr, z);
    }

    // Subspace-expansion pass (paper Sec. II.D): the sweep order of S with
    // the centre moved by QR but no time evolution; the SPAWN op of a bond
    // stops the program when it accepts new functions.
    void emit_spawn_visit(Program& pr, int z) {
        for (size_t k = 0; k < t.ch[z].size(); ++k) {
            int c = t.ch[z][k];
            OpSpec s = tensor_op(TTN_OP_SPAWN, z, (int)k);
            s.op.c = nullptr;
            s.b_off = p.tensor_off[c];          // child tensor (linked as op.b, copied to op.c)
            s.op.Dc = (int)t.dims[c].size();
            for (int j = 0; j < s.op.Dc; ++j) s.op.dimsc[j] = t.dims[c][j];
            s.op.e0 = up_rng[c].first; s.op.ne = up_rng[c].second;
            s.op.e1 = down_rng[z][k].first; s.op.ne1 = down_rng[z][k].second;
            s.op.e2 = bond_raw_rng[c].first; s.op.ne2 = bond_raw_rng[c].second;
            s.op.node = z; s.op.child = c;
            s.out_off = p.spawn_out_off;
            pr.ops.push_back(s);
            emit_qr_down(pr, z, (int)k);
            emit_absorb_child(pr, c);
            emit_env_down(pr, z, (int)k);
            emit_spawn_visit(pr, c);
            emit_qr_up(pr, c);
            emit_env_up(pr, c);
            emit_absorb_parent(pr, z, (int)k);
        }
    }
    void make_to_root() {
        p.to_root_prog.assign(t.n, {});
        for (int z = 1; z < t.n; ++z) {
            Program& pr = p.to_root_prog[z];
            for (int u = z; u > 0; u = t.parent[u]) {
                int par = t.parent[u];
                int k = (int)(std::find(t.ch[par].begin(), t.ch[par].end(), u) - t.ch[par].begin());
                emit_qr_up(pr, u);
                emit_absorb_parent(pr, par, k);
            }
        }
    }

    // ---- observables ----------------------------------------------------------
    void make_observables() {
        int n = t.n;
        one_slot = const_slot(1, 1, {cplx(1.0)});
        // Gram matrices <Psi_i^z|Psi_j^z> along every root-to-leaf path.
        std::vector<int> gram(n, -1);
        gram[0] = one_slot;
        for (int z = 1; z < n; ++z) gram[z] = new_slot(t.bond[z], t.bond[z]);
        p.rdm_prog.assign(n, {}); p.rdm_slot.assign(n, -1);
        p.vac_prog.assign(n, {}); p.vac_slot.assign(n, -1);
        for (int l = 0; l < n; ++l) {
            if (!t.leaf(l)) continue;
            std::vector<int> path;
            for (int u = l; u > 0; u = t.parent[u]) path.push_back(u);
            std::reverse(path.begin(), path.end());
            Program& pr = p.rdm_prog[l];
            for (int c : path) {
                int z = t.parent[c];
                int k = (int)(std::find(t.ch[z].begin(), t.ch[z].end(), c) - t.ch[z].begin());
                Proto e; e.w = 1.0; e.out = gram[c]; e.slot.assign(t.dims[z].size(), -1);
                e.slot.back() = gram[z];
                auto rg = push_entries({e});
                OpSpec s = tensor_op(TTN_OP_ENV, z, k);
                s.op.e0 = rg.first; s.op.ne = rg.second;
                pr.ops.push_back(s);
            }
            int rs = new_slot(t.phys[l], t.phys[l]);
            p.rdm_slot[l] = rs;
            Proto e; e.w = 1.0; e.out = rs; e.slot.assign(2, -1); e.slot[1] = gram[l];
            auto rg = push_entries({e});
            OpSpec s = tensor_op(TTN_OP_ENV, l, 0);
            s.op.e0 = rg.first; s.op.ne = rg.second;
            pr.ops.push_back(s);
        }
        // vacuum projections: bottom-up contraction with basis vector 0 on all
        // leaves but the kept one.
        std::vector<int> e0_slot(TTN_MAXCHI + 1, -1);
        for (int keep = 0; keep < n; ++keep) {
            if (!t.leaf(keep)) continue;
            Program& pr = p.vac_prog[keep];
            std::vector<int> res(n, -1);
            std::vector<int> on_path(n, 0);
            for (int u = keep; u >= 0; u = t.parent[u]) { on_path[u] = 1; if (u == 0) break; }
            std::vector<int> order = t.postorder();
            for (int z : order) {
                int rows;  // leading dimension of the result: d_keep on the path, else 1
                OpSpec s = tensor_op(TTN_OP_CONTRACT_VEC, z, 0);
                Proto e; e.w = 1.0; e.out = -1; e.slot.assign(t.dims[z].size(), -1);
                if (t.leaf(z)) {
                    if (z == keep) {
                        // the kept leaf's tensor itself is the factor for its parent
                        rows = t.phys[z];
                        int sl = new_slot(rows, t.dims[z].back());
                        e.slot[0] = -1;
                        res[z] = sl;
                        auto rg = push_entries({e});
                        s.op.e0 = rg.first; s.op.ne = rg.second;
                        s.op.k = sl;                   // output slot
                        pr.ops.push_back(s);
                        continue;
                    }
                    int d = t.phys[z];
                    if (e0_slot[d] < 0) {
                        std::vector<cplx> v(d, 0.0); v[0] = 1.0;
                        e0_slot[d] = const_slot(1, d, v);
                    }
                    e.slot[0] = e0_slot[d];
                    rows = 1;
                } else {
                    rows = 1;
                    for (size_t k = 0; k < t.ch[z].size(); ++k) {
                        int c = t.ch[z][k];
                        e.slot[k] = res[c];
                        if (on_path[c]) rows = t.phys[keep];
                    }
                }
                int sl = new_slot(rows, t.dims[z].back());
                res[z] = sl;
                auto rg = push_entries({e});
                s.op.e0 = rg.first; s.op.ne = rg.second;
                s.op.k = sl;
                pr.ops.push_back(s);
            }
            p.vac_slot[keep] = res[0];
        }
        // norm and energy at the root
        {
            Program& pr = p.norm_energy_prog;
            OpSpec s = tensor_op(TTN_OP_DOT, 0, 0);
            s.op.ne = 0;
            s.out_off = p.scal_off;
            pr.ops.push_back(s);
            if (h) {
                emit_combos(pr, heff_combo[0]);
                OpSpec e = tensor_op(TTN_OP_DOT, 0, 0);
                e.op.e0 = heff_rng[0].first; e.op.ne = heff_rng[0].second;
                e.out_off = p.scal_off + 16;
                pr.ops.push_back(e);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Multi-set operators (paper Sec. II.A, multi-set ansatz).  Every set has its
// own tensors on the shared tree; term r = c_r |a_r><b_r| (x) (factors).
// A channel is keyed by (bra set, ket set, part of the term on one side of
// a bond) and stands for that part's matrix element between the bra set's
// and the ket set's functions there.  Only a same-set channel with an empty
// part is the identity; for a != b an empty part is the overlap of the two
// sets' functions, a real matrix.  Per set, the terms acting only inside a
// subtree are pre-summed into one local channel of its bond (LOC), those
// acting only outside into one local mean-field channel (DLOC), and a
// leaf's own terms into one constant matrix (the single-set planner's local
// channels); terms crossing a bond and terms coupling two sets keep a
// channel per (set pair, part).
// ---------------------------------------------------------------------------
struct MsBuilder {
    const Tree& t;
    const Hamiltonian& h;
    Plan& p;
    const int S;
    using CKey = std::tuple<int, int, Key>;
    enum { D_DN = 0, D_UP = 1, D_LOC = 2, D_DLOC = 3, D_DG = 4 };
    struct Def { int up; int c; CKey key; int slot; };   // up: one of D_*
    std::vector<std::map<CKey, int>> up_ch, dn_ch;       // per bond (child node)
    // grouped mean-field channels per bond: key (a, b, inside part); the
    // set pairs whose crossing terms a bond groups that way (those with fewer
    // distinct inside than outside parts there)
    std::vector<std::map<CKey, int>> dg_ch;
    std::vector<std::set<std::pair<int, int>>> dg_pair;
    std::vector<Def> todo;
    std::map<std::pair<int, int>, int> phys;             // (leaf, matrix id) -> constant slot
    // ENV entries per bond and set pair: built at the child (up) or at the
    // parent keeping the child's mode (down)
    std::vector<std::map<std::pair<int, int>, std::vector<Proto>>> up_env, dn_env;
    std::vector<std::pair<int, int>> heff_rng, bond_rng;
    std::vector<std::map<std::pair<int, int>, std::pair<int, int>>> up_rng, dn_rng;

    // local channels per (node, set): slot, or -1 before creation; existence
    std::vector<std::vector<int>> loc_slot, dloc_slot;
    std::vector<std::vector<char>> has_loc, has_dloc;
    std::map<std::pair<int, int>, int> pl;               // (leaf, set) -> constant slot of its own terms

    MsBuilder(const Tree& t_, const Hamiltonian& h_, Plan& p_) : t(t_), h(h_), p(p_), S(h_.n_sets) {
        up_ch.resize(t.n); dn_ch.resize(t.n); dg_ch.resize(t.n); up_env.resize(t.n); dn_env.resize(t.n);
        loc_slot.assign(t.n, std::vector<int>(S, -1));
        dloc_slot.assign(t.n, std::vector<int>(S, -1));
        has_loc.assign(t.n, std::vector<char>(S, 0));
        has_dloc.assign(t.n, std::vector<char>(S, 0));
        dg_pair.assign(t.n, {});
        for (int c = 1; c < t.n; ++c) {
            std::map<std::pair<int, int>, std::pair<std::set<Key>, std::set<Key>>> parts;
            for (size_t r = 0; r < h.terms.size(); ++r) {
                if (!crossing(r, c)) continue;
                auto& pr = parts[{h.bra[r], h.ket[r]}];
                pr.first.insert(restrict_to(h.terms[r], c, true));
                pr.second.insert(restrict_to(h.terms[r], c, false));
            }
            for (auto& kv : parts)
                if (kv.second.first.size() < kv.second.second.size()) dg_pair[c].insert(kv.first);
        }
        for (size_t r = 0; r < h.terms.size(); ++r) {
            if (!diag(r)) continue;
            for (int c = 1; c < t.n; ++c) {
                const bool in = !restrict_to(h.terms[r], c, true).empty(), out = !restrict_to(h.terms[r], c, false).empty();
                if (in && !out) has_loc[c][h.bra[r]] = 1;
                if (out && !in) has_dloc[c][h.bra[r]] = 1;
            }
        }
    }
    // a same-set term acting somewhere (pre-summed where it is local)
    bool diag(size_t r) const { return h.bra[r] == h.ket[r] && !h.terms[r].empty(); }
    // mode of node z holding leaf l: its child index, 0 for a leaf's own factor, D-1 outside
    int mode_of(int z, int l) const {
        const int D = (int)t.dims[z].size();
        if (!t.in_sub(l, z)) return D - 1;
        if (t.leaf(z)) return 0;
        for (size_t k = 0; k < t.ch[z].size(); ++k)
            if (t.in_sub(l, t.ch[z][k])) return (int)k;
        return -1;
    }
    std::set<int> touched(int z, const Key& key) const {
        std::set<int> m;
        for (auto& f : key) m.insert(mode_of(z, f.first));
        return m;
    }
    // term r crosses bond c: a set coupling always (overlaps on both sides),
    // a same-set term when it acts on both sides
    bool crossing(size_t r, int c) const {
        if (h.bra[r] != h.ket[r]) return true;
        return !restrict_to(h.terms[r], c, true).empty() && !restrict_to(h.terms[r], c, false).empty();
    }
    // DG(c, a, b, in) = sum over the terms of set pair (a, b) crossing bond c
    // with inside part `in` of c_r H_r(c) (their mean fields, weighted)
    int get_dg(int c, int a, int b, const Key& in) {
        CKey key{a, b, in};
        auto it = dg_ch[c].find(key);
        if (it != dg_ch[c].end()) return it->second;
        int s = new_slot(t.bond[c], t.bond[c]);
        dg_ch[c][key] = s;
        todo.push_back({D_DG, c, key, s});
        return s;
    }
    // Entry of term r at node z (mode `skip` kept, -1: none; `out`: ENV
    // output slot or -1).  A term that crosses z's own bond enters through
    // z's grouped channel for its inside part -- weight 1, once per (set
    // pair, inside part) in `seen` -- else term by term.
    void term_at(int z, size_t r, int skip, int out, std::set<CKey>& seen, std::vector<Proto>& es) {
        const int a = h.bra[r], b = h.ket[r];
        Proto e;
        e.out = out; e.dst = a; e.src = b;
        if (z > 0 && crossing(r, z) && dg_pair[z].count({a, b})) {
            const Key in = restrict_to(h.terms[r], z, true);
            if (!seen.insert(CKey{a, b, in}).second) return;
            const int D = (int)t.dims[z].size();
            e.w = 1.0;
            e.slot = mode_slots(z, a, b, in, skip, false);
            e.slot[D - 1] = get_dg(z, a, b, in);
            es.push_back(e);
            return;
        }
        e.w = h.coeff[r];
        e.slot = mode_slots(z, a, b, h.terms[r], skip);
        es.push_back(e);
    }
    // built at the parent z keeping c's mode: z's grouped channels (or, at
    // the root, the terms one by one) with the siblings' parts
    void define_dg(int c, int a, int b, const Key& in, int slot) {
        const int z = t.parent[c];
        const int k = (int)(std::find(t.ch[z].begin(), t.ch[z].end(), c) - t.ch[z].begin());
        std::vector<Proto> es;
        std::set<CKey> seen;
        for (size_t r = 0; r < h.terms.size(); ++r) {
            if (h.bra[r] != a || h.ket[r] != b || !crossing(r, c) || restrict_to(h.terms[r], c, true) != in) continue;
            term_at(z, r, k, slot, seen, es);
        }
        auto& dst = dn_env[c][{a, b}];
        dst.insert(dst.end(), es.begin(), es.end());
    }
    int get_loc(int c, int a) {
        if (!has_loc[c][a]) return -1;
        if (loc_slot[c][a] < 0) {
            loc_slot[c][a] = new_slot(t.bond[c], t.bond[c]);
            todo.push_back({D_LOC, c, CKey{a, a, {}}, loc_slot[c][a]});
        }
        return loc_slot[c][a];
    }
    int get_dloc(int c, int a) {
        if (c == 0 || !has_dloc[c][a]) return -1;
        if (dloc_slot[c][a] < 0) {
            dloc_slot[c][a] = new_slot(t.bond[c], t.bond[c]);
            todo.push_back({D_DLOC, c, CKey{a, a, {}}, dloc_slot[c][a]});
        }
        return dloc_slot[c][a];
    }
    // sum of c_r M_r over set a's terms whose only factor is on leaf l (constant)
    int get_pl(int l, int a) {
        auto it = pl.find({l, a});
        if (it != pl.end()) return it->second;
        const int d = t.phys[l];
        std::vector<cplx> sum((size_t)d * d, 0.0);
        for (size_t r = 0; r < h.terms.size(); ++r) {
            if (!diag(r) || h.bra[r] != a || h.terms[r].size() != 1 || h.terms[r][0].first != l) continue;
            const auto& M = h.mats[h.terms[r][0].second];
            for (int i = 0; i < d * d; ++i) sum[i] += h.coeff[r] * M[i];
        }
        int id = new_slot(d, d);
        p.slots[id].constant = true;
        p.slots[id].data = sum;
        return pl[{l, a}] = id;
    }
    int new_slot(int rows, int cols) {
        SlotInfo s; s.rows = rows; s.cols = cols;
        p.slots.push_back(s);
        return (int)p.slots.size() - 1;
    }
    Key restrict_to(const Key& k, int c, bool inside) const {
        Key out;
        for (auto& f : k) if (t.in_sub(f.first, c) == inside) out.push_back(f);
        return out;
    }
    int phys_slot(int l, int m) {
        auto it = phys.find({l, m});
        if (it != phys.end()) return it->second;
        int d = t.phys[l];
        int id = new_slot(d, d);
        p.slots[id].constant = true;
        p.slots[id].data = h.mats[m];
        return phys[{l, m}] = id;
    }
    // channel of bond c (created on first use; -1 = identity)
    int chan(bool up, int c, int a, int b, const Key& part) {
        if (a == b && part.empty()) return -1;
        auto& m = up ? up_ch[c] : dn_ch[c];
        CKey key{a, b, part};
        auto it = m.find(key);
        if (it != m.end()) return it->second;
        int s = new_slot(t.bond[c], t.bond[c]);
        m[key] = s;
        todo.push_back({up ? D_UP : D_DN, c, key, s});
        return s;
    }
    // slot list of a term part `key` (the whole term, or its part on one
    // side of a bond) on the modes of node z, skipping mode `skip`
    std::vector<int> mode_slots(int z, int a, int b, const Key& key, int skip, bool parent = true) {
        const int D = (int)t.dims[z].size();
        std::vector<int> sl(D, -1);
        if (t.leaf(z)) {
            if (skip != 0) {
                Key in = restrict_to(key, z, true);
                if (!in.empty()) sl[0] = phys_slot(z, in[0].second);
            }
        } else {
            for (size_t k = 0; k < t.ch[z].size(); ++k) {
                if ((int)k == skip) continue;
                int ck = t.ch[z][k];
                sl[k] = chan(true, ck, a, b, restrict_to(key, ck, true));
            }
        }
        if (parent && z > 0 && skip != D - 1) sl[D - 1] = chan(false, z, a, b, restrict_to(key, z, false));
        return sl;
    }
    void define(const Def& q) {
        const int a = std::get<0>(q.key), b = std::get<1>(q.key);
        const Key& part = std::get<2>(q.key);
        Proto e;
        e.w = 1.0;
        e.out = q.slot;
        if (q.up == D_LOC) { define_loc(q.c, a, q.slot); return; }
        if (q.up == D_DLOC) { define_dloc(q.c, a, q.slot); return; }
        if (q.up == D_DG) { define_dg(q.c, a, b, part, q.slot); return; }
        if (q.up == D_UP) {
            // at node c, every mode but the parent's
            e.slot = mode_slots(q.c, a, b, part, (int)t.dims[q.c].size() - 1);
            up_env[q.c][{a, b}].push_back(e);
        } else {
            // at the parent z keeping the mode of c; part is the part outside c
            const int z = t.parent[q.c];
            const int k = (int)(std::find(t.ch[z].begin(), t.ch[z].end(), q.c) - t.ch[z].begin());
            e.slot = mode_slots(z, a, b, part, k);
            dn_env[q.c][{a, b}].push_back(e);
        }
    }
    // LOC(c, a) = sum over set a's terms acting only inside c of c_r h_r(c),
    // built at node c: the children's LOC on their modes, the terms spanning
    // two or more children term by term (a leaf: its constant sum).
    void define_loc(int c, int a, int slot) {
        std::vector<Proto> es;
        const int D = (int)t.dims[c].size();
        Proto e;
        e.w = 1.0; e.out = slot; e.slot.assign(D, -1);
        if (t.leaf(c)) {
            e.slot[0] = get_pl(c, a);
            es.push_back(e);
        } else {
            for (size_t k = 0; k < t.ch[c].size(); ++k) {
                const int s = get_loc(t.ch[c][k], a);
                if (s < 0) continue;
                Proto f = e;
                f.slot[k] = s;
                es.push_back(f);
            }
            for (size_t r = 0; r < h.terms.size(); ++r) {
                if (!diag(r) || h.bra[r] != a || !restrict_to(h.terms[r], c, false).empty()) continue;
                if (touched(c, h.terms[r]).size() < 2) continue;
                Proto f;
                f.w = h.coeff[r]; f.out = slot;
                f.slot = mode_slots(c, a, a, h.terms[r], D - 1);
                es.push_back(f);
            }
        }
        auto& dst = up_env[c][{a, a}];
        dst.insert(dst.end(), es.begin(), es.end());
    }
    // DLOC(c, a) = sum over set a's terms acting only outside c of c_r H_r(c),
    // built at the parent z keeping c's mode: the siblings' LOC, z's DLOC and
    // the terms spanning two or more of those modes term by term.
    void define_dloc(int c, int a, int slot) {
        std::vector<Proto> es;
        const int z = t.parent[c];
        const int k = (int)(std::find(t.ch[z].begin(), t.ch[z].end(), c) - t.ch[z].begin());
        const int D = (int)t.dims[z].size();
        Proto e;
        e.w = 1.0; e.out = slot; e.slot.assign(D, -1);
        for (size_t j = 0; j < t.ch[z].size(); ++j) {
            if ((int)j == k) continue;
            const int s = get_loc(t.ch[z][j], a);
            if (s < 0) continue;
            Proto f = e;
            f.slot[j] = s;
            es.push_back(f);
        }
        const int sd = get_dloc(z, a);
        if (sd >= 0) {
            Proto f = e;
            f.slot[D - 1] = sd;
            es.push_back(f);
        }
        std::set<CKey> seen;
        for (size_t r = 0; r < h.terms.size(); ++r) {
            if (!diag(r) || h.bra[r] != a || !restrict_to(h.terms[r], c, true).empty()) continue;
            if (touched(z, h.terms[r]).size() < 2) continue;
            term_at(z, r, k, slot, seen, es);
        }
        auto& dst = dn_env[c][{a, a}];
        dst.insert(dst.end(), es.begin(), es.end());
    }
    void close() {
        for (size_t i = 0; i < todo.size(); ++i) {
            const Def q = todo[i];          // define() may grow todo
            define(q);
        }
    }

    // ---- entries -------------------------------------------------------------
    // Entries with the same (dst, src, slots) are merged; the order keeps
    // entries of one output slot, then of one destination set, then of one
    // last factor adjacent (the device sums such runs before their shared
    // last factor).
    std::pair<int, int> push(std::vector<Proto> es) {
        std::map<std::tuple<int, int, int, std::vector<int>>, cplx> merged;
        std::vector<std::tuple<int, int, int, std::vector<int>>> order;
        for (auto& e : es) {
            auto key = std::make_tuple(e.out, e.dst, e.src, e.slot);
            if (!merged.count(key)) order.push_back(key);
            merged[key] += e.w;
        }
        std::vector<Proto> out;
        for (auto& key : order) {
            if (merged[key] == cplx(0.0) && std::get<0>(key) < 0) continue;
            Proto e;
            e.w = merged[key]; e.out = std::get<0>(key); e.dst = std::get<1>(key); e.src = std::get<2>(key);
            e.slot = std::get<3>(key);
            out.push_back(e);
        }
        auto last = [](const Proto& e) {
            int lm = -1;
            for (size_t j = 0; j < e.slot.size(); ++j) if (e.slot[j] >= 0) lm = (int)j;
            return std::make_pair(lm, lm >= 0 ? e.slot[lm] : -1);
        };
        std::stable_sort(out.begin(), out.end(), [&](const Proto& a, const Proto& b) {
            if (a.out != b.out) return a.out < b.out;
            if (a.dst != b.dst) return a.dst < b.dst;
            return last(a) < last(b);
        });
        int e0 = (int)p.entries.size();
        for (auto& e : out) {
            TtnEntry te{};
            te.wr = e.w.real(); te.wi = e.w.imag(); te.out = e.out; te.src = e.src; te.dst = e.dst;
            for (int j = 0; j < TTN_MAXD; ++j) te.slot[j] = j < (int)e.slot.size() ? e.slot[j] : -1;
            p.entries.push_back(te);
        }
        return {e0, (int)out.size()};
    }

    void prepare() {
        const int n = t.n, R = (int)h.terms.size();
        std::vector<std::vector<Proto>> heff(n), bond(n);
        p.op_bond_dim.assign(n, 0);
        std::vector<cplx> konst(S, 0.0);                 // same-set constants
        for (int r = 0; r < R; ++r)
            if (h.bra[r] == h.ket[r] && h.terms[r].empty()) konst[h.bra[r]] += h.coeff[r];
        auto one = [&](int dst, int src, cplx w, std::vector<int> sl) {
            Proto e;
            e.w = w; e.out = -1; e.dst = dst; e.src = src; e.slot = std::move(sl);
            return e;
        };
        for (int z = 0; z < n; ++z) {
            const int D = (int)t.dims[z].size();
            for (int a = 0; a < S; ++a) {
                // local sums: the children's (a leaf's own terms), the outside's, constants
                if (t.leaf(z)) {
                    if (z > 0 && has_loc[z][a]) {
                        std::vector<int> sl(D, -1);
                        sl[0] = get_pl(z, a);
                        heff[z].push_back(one(a, a, 1.0, sl));
                    }
                } else {
                    for (size_t k = 0; k < t.ch[z].size(); ++k) {
                        const int s = get_loc(t.ch[z][k], a);
                        if (s < 0) continue;
                        std::vector<int> sl(D, -1);
                        sl[k] = s;
                        heff[z].push_back(one(a, a, 1.0, sl));
                    }
                }
                const int sd = get_dloc(z, a);
                if (sd >= 0) {
                    std::vector<int> sl(D, -1);
                    sl[D - 1] = sd;
                    heff[z].push_back(one(a, a, 1.0, sl));
                }
                if (konst[a] != cplx(0.0)) heff[z].push_back(one(a, a, konst[a], std::vector<int>(D, -1)));
                if (z == 0) continue;
                const int sl_ = get_loc(z, a), sdl = get_dloc(z, a);
                if (sl_ >= 0) bond[z].push_back(one(a, a, 1.0, {sl_, -1}));
                if (sdl >= 0) bond[z].push_back(one(a, a, 1.0, {-1, sdl}));
                if (konst[a] != cplx(0.0)) bond[z].push_back(one(a, a, konst[a], {-1, -1}));
            }
            std::set<CKey> seen_h, seen_b;
            for (int r = 0; r < R; ++r) {
                const int a = h.bra[r], b = h.ket[r];
                if (a == b && h.terms[r].empty()) continue;          // constants: above
                // same-set terms on one mode of z are in the local sums
                if (a != b || touched(z, h.terms[r]).size() >= 2) term_at(z, r, -1, -1, seen_h, heff[z]);
                if (z == 0 || !crossing(r, z)) continue;              // local: above
                const Key in = restrict_to(h.terms[r], z, true);
                if (!dg_pair[z].count({a, b})) {
                    bond[z].push_back(one(a, b, h.coeff[r], {chan(true, z, a, b, in),
                                                             chan(false, z, a, b, restrict_to(h.terms[r], z, false))}));
                    continue;
                }
                if (!seen_b.insert(CKey{a, b, in}).second) continue;
                bond[z].push_back(one(a, b, 1.0, {chan(true, z, a, b, in), get_dg(z, a, b, in)}));
            }
        }
        close();
        heff_rng.assign(n, {0, 0}); bond_rng.assign(n, {0, 0});
        up_rng.assign(n, {}); dn_rng.assign(n, {});
        for (int z = 0; z < n; ++z) {
            heff_rng[z] = push(heff[z]);
            if (z == 0) continue;
            bond_rng[z] = push(bond[z]);
            int nloc = 0;
            for (int a = 0; a < S; ++a) nloc += (loc_slot[z][a] >= 0) + (dloc_slot[z][a] >= 0);
            p.op_bond_dim[z] = (int)(up_ch[z].size() + dn_ch[z].size() + dg_ch[z].size()) + nloc;
            for (auto& kv : up_env[z]) up_rng[z][kv.first] = push(kv.second);
            for (auto& kv : dn_env[z]) dn_rng[z][kv.first] = push(kv.second);
        }
    }

    // ---- programs --------------------------------------------------------------
    int64_t set_off(int z, int a) const { return p.tensor_off[z] + (int64_t)a * t.size[z] * (int64_t)p.esz_state; }
    int64_t bond_buf(int a, int nb) const { return p.bond_off + (int64_t)a * nb * nb * (int64_t)p.esz_state; }
    OpSpec base(int type, int z, int k) const {
        OpSpec s;
        std::memset(&s.op, 0, sizeof(TtnOp));
        s.op.type = type;
        s.op.D = (int)t.dims[z].size();
        for (int j = 0; j < s.op.D; ++j) s.op.dims[j] = t.dims[z][j];
        s.op.k = k;
        return s;
    }
    void per_set(Program& pr, int type, int z, int k, int bond_child) {
        for (int a = 0; a < S; ++a) {
            OpSpec s = base(type, z, k);
            s.a_off = set_off(z, a);
            s.b_off = bond_buf(a, t.bond[bond_child]);
            pr.ops.push_back(s);
        }
    }
    void emit_env(Program& pr, int z, int k, const std::map<std::pair<int, int>, std::pair<int, int>>& rngs) {
        for (auto& kv : rngs) {
            if (kv.second.second == 0) continue;
            OpSpec s = base(TTN_OP_ENV, z, k);
            s.a_off = set_off(z, kv.first.first);
            if (kv.first.second != kv.first.first) s.c_off = set_off(z, kv.first.second);
            s.op.e0 = kv.second.first; s.op.ne = kv.second.second;
            pr.ops.push_back(s);
        }
    }
    void emit_env_up(Program& pr, int c) { emit_env(pr, c, (int)t.dims[c].size() - 1, up_rng[c]); }
    void emit_env_down(Program& pr, int z, int k) { emit_env(pr, z, k, dn_rng[t.ch[z][k]]); }
    void emit_evolve_node(Program& pr, int z) {
        OpSpec s = base(TTN_OP_EVOLVE, z, 0);
        s.a_off = p.tensor_off[z];
        s.op.nset = S;
        s.op.e0 = heff_rng[z].first; s.op.ne = heff_rng[z].second;
        s.op.hermitian = h.hermitian ? 1 : 0;
        s.op.tau_coef = 0.5;
        pr.ops.push_back(s);
    }
    void emit_evolve_bond(Program& pr, int c) {
        OpSpec s;
        std::memset(&s.op, 0, sizeof(TtnOp));
        s.op.type = TTN_OP_EVOLVE;
        s.op.D = 2;
        s.op.dims[0] = s.op.dims[1] = t.bond[c];
        s.a_off = p.bond_off;
        s.op.nset = S;
        s.op.e0 = bond_rng[c].first; s.op.ne = bond_rng[c].second;
        s.op.hermitian = h.hermitian ? 1 : 0;
        s.op.tau_coef = -0.5;                    // backward bond step
        pr.ops.push_back(s);
    }
    // The projector-splitting sweeps of the single-set plan, with the gauge
    // moves done set by set and the exponentials on all sets at once.
    void emit_S(Program& pr, int z) {
        for (size_t k = 0; k < t.ch[z].size(); ++k) {
            const int c = t.ch[z][k], Dc = (int)t.dims[c].size();
            per_set(pr, TTN_OP_QR_DOWN, z, (int)k, c);
            per_set(pr, TTN_OP_ABSORB_CHILD, c, Dc - 1, c);
            emit_env_down(pr, z, (int)k);
            emit_S(pr, c);
            per_set(pr, TTN_OP_QR_UP, c, Dc - 1, c);
            emit_env_up(pr, c);
            emit_evolve_bond(pr, c);
            per_set(pr, TTN_OP_ABSORB_PARENT, z, (int)k, c);
        }
        emit_evolve_node(pr, z);
    }
    void emit_Sstar(Program& pr, int z) {
        emit_evolve_node(pr, z);
        for (int k = (int)t.ch[z].size() - 1; k >= 0; --k) {
            const int c = t.ch[z][k], Dc = (int)t.dims[c].size();
            per_set(pr, TTN_OP_QR_DOWN, z, k, c);
            emit_env_down(pr, z, k);
            emit_evolve_bond(pr, c);
            per_set(pr, TTN_OP_ABSORB_CHILD, c, Dc - 1, c);
            emit_Sstar(pr, c);
            per_set(pr, TTN_OP_QR_UP, c, Dc - 1, c);
            emit_env_up(pr, c);
            per_set(pr, TTN_OP_ABSORB_PARENT, z, k, c);
        }
    }
    void make_programs() {
        for (int z : t.postorder())
            if (z > 0) emit_env_up(p.init_prog, z);
        emit_S(p.step_prog, 0);
        emit_Sstar(p.step_prog, 0);
        OpSpec end;
        std::memset(&end.op, 0, sizeof(TtnOp));
        end.op.type = TTN_OP_STEP_END;
        p.step_prog.ops.push_back(end);
        // norm and energy of the whole state, populations of the sets
        OpSpec nrm = base(TTN_OP_DOT, 0, 0);
        nrm.a_off = p.tensor_off[0]; nrm.op.nset = S; nrm.out_off = p.scal_off;
        p.norm_energy_prog.ops.push_back(nrm);
        OpSpec en = base(TTN_OP_DOT, 0, 0);
        en.a_off = p.tensor_off[0]; en.op.nset = S;
        en.op.e0 = heff_rng[0].first; en.op.ne = heff_rng[0].second;
        en.out_off = p.scal_off + 16;
        p.norm_energy_prog.ops.push_back(en);
        for (int a = 0; a < S; ++a) {
            OpSpec d = base(TTN_OP_DOT, 0, 0);
            d.a_off = set_off(0, a); d.out_off = p.setpop_off + 16 * a;
            p.setpop_prog.ops.push_back(d);
        }
        p.to_root_prog.assign(t.n, {});
        p.rdm_prog.assign(t.n, {}); p.rdm_slot.assign(t.n, -1);
        p.vac_prog.assign(t.n, {}); p.vac_slot.assign(t.n, -1);
    }
};

}  // namespace

std::string make_plan(const Tree& t, const Hamiltonian* h, int precision, Plan& p) {
    p = Plan();
    p.esz = precision == 1 ? 8 : 16;   // 1: mixed precision (complex64 bulk)
    const int nset = (h && h->n_sets > 1) ? h->n_sets : 1;
    p.nset = nset;
    // ---- state arena --------------------------------------------------------
    int64_t off = 0;
    p.tensor_off.assign(t.n, 0);
    int64_t smax = 1;
    int max_chi = 1;
    for (int z = 0; z < t.n; ++z) {
        p.tensor_off[z] = off;
        off = align_up(off + nset * t.size[z] * (int64_t)p.esz_state, 256);
        smax = std::max(smax, t.size[z]);
        for (int d : t.dims[z]) max_chi = std::max(max_chi, d);
    }
    smax = std::max<int64_t>(smax, (int64_t)max_chi * max_chi) * nset;   // Krylov vectors span all sets
    p.max_chi = max_chi;
    p.smax = align_up(smax, 32);
    p.bond_off = off;
    off = align_up(off + (int64_t)nset * max_chi * max_chi * 16, 256);
    p.work_off = off;
    // (KMAX+1) Krylov vectors + 3 scratch tensors in the bulk type, then 2
    // FP64 QR matrices
    off = align_up(off + (int64_t)(TTN_KMAX + 4) * p.smax * (int64_t)p.esz + 2 * p.smax * 16, 256);
    p.status_off = off; off += 64;
    p.steps_off = off; off += 64;
    p.flops_off = off; off += 64;
    p.cycles_off = off; off += 32 * 8;
    p.scal_off = off; off = align_up(off + 16 * 16, 256);
    {
        int64_t maxNJ = 1;
        for (int c = 1; c < t.n; ++c) maxNJ = std::max<int64_t>(maxNJ, t.size[c] / t.bond[c]);
        p.spawn_out_off = off;
        p.spawn_out_bytes = align_up(8 * (4 + TTN_SPAWN_MAX_NEW) + 16 * maxNJ * TTN_SPAWN_MAX_NEW, 256);
        off += p.spawn_out_bytes;
    }
    p.max_stamps = 4096;
    p.stamps_off = off; off = align_up(off + 8 * (int64_t)p.max_stamps, 256);
    p.setpop_off = off; off = align_up(off + 16 * (int64_t)nset, 256);
    p.total_bytes = off;

    if (nset > 1) {
        // multi-set state: per-pair channels, no expansion / ground state / RDM programs
        MsBuilder mb(t, *h, p);
        mb.prepare();
        mb.make_programs();
        p.spawn_kmax = 0;
        p.spawn_ws_off = p.total_bytes;
        int64_t soff = 0;
        for (auto& sl : p.slots) {
            sl.off = soff;
            soff = align_up(soff + (int64_t)sl.rows * sl.cols * (int64_t)p.esz, 256);
        }
        return "";
    }

    // ---- operators and programs ---------------------------------------------
    Builder b(t, h, p);
    b.make_channels();
    if (h) {
        b.prepare_entries();
        for (int z : t.postorder())
            if (z > 0) b.emit_env_up(p.init_prog, z);
        b.emit_S(p.step_prog, 0);
        b.emit_Sstar(p.step_prog, 0);
        b.emit_spawn_visit(p.spawn_prog, 0);
        if (h->hermitian) b.emit_ground(p.ground_prog, 0);
        b.make_to_root();
        // spawn workspace: K = (distinct up channels of a bond's terms) x bond dimension
        int kmax = 0;
        for (int c = 1; c < t.n; ++c) {
            std::set<int> ids;
            auto rg = b.bond_raw_rng[c];
            for (int i = 0; i < rg.second; ++i)
                if (p.entries[rg.first + i].slot[0] >= 0) ids.insert(p.entries[rg.first + i].slot[0]);
            kmax = std::max(kmax, (int)ids.size() * t.bond[c]);
        }
        p.spawn_kmax = std::min(kmax, TTN_SPAWN_MAX_K);
        p.spawn_ws_off = p.total_bytes;
        p.total_bytes = align_up(p.total_bytes + 16 * (p.smax + 6 * (int64_t)p.spawn_kmax * p.spawn_kmax), 256);
        if (p.e_shift != 0.0) {                    // global phase of the shift, on the root (the centre)
            OpSpec ph = b.tensor_op(TTN_OP_PHASE, 0, 0);
            ph.op.tau_coef = p.e_shift;
            p.step_prog.ops.push_back(ph);
        }
        OpSpec s;
        std::memset(&s.op, 0, sizeof(TtnOp));
        s.op.type = TTN_OP_STEP_END;
        p.step_prog.ops.push_back(s);
    }
    b.make_observables();
    // slot storage (complex elements of the bulk type)
    int64_t soff = 0;
    for (auto& s : p.slots) {
        s.off = soff;
        soff = align_up(soff + (int64_t)s.rows * s.cols * (int64_t)p.esz, 256);
    }
    (void)soff;
    return "";
}

void product_state(const Tree& t, const std::vector<std::vector<cplx>>& leaf_vecs,
                   std::vector<std::vector<cplx>>& A) {
    A.assign(t.n, {});
    for (int z = 0; z < t.n; ++z) {
        const auto& dims = t.dims[z];
        int N = dims.back();
        int64_t rows = t.size[z] / N;
        A[z].assign(t.size[z], 0.0);
        if (t.leaf(z)) {
            int d = t.phys[z];
            std::vector<std::vector<cplx>> cols;
            std::vector<cplx> v = leaf_vecs[z];
            double nrm = 0;
            for (auto& x : v) nrm += std::norm(x);
            nrm = std::sqrt(nrm);
            for (auto& x : v) x /= nrm;
            cols.push_back(v);
            int j = 0;
            while ((int)cols.size() < N && j < d) {
                std::vector<cplx> e(d, 0.0);
                e[j++] = 1.0;
                for (int pass = 0; pass < 2; ++pass)
                    for (auto& c : cols) {
                        cplx h = 0;
                        for (int i = 0; i < d; ++i) h += std::conj(c[i]) * e[i];
                        for (int i = 0; i < d; ++i) e[i] -= c[i] * h;
                    }
                double en = 0;
                for (auto& x : e) en += std::norm(x);
                en = std::sqrt(en);
                if (en > 0.5) {
                    for (auto& x : e) x /= en;
                    cols.push_back(e);
                }
            }
            for (int i = 0; i < d; ++i)
                for (int c = 0; c < N; ++c) A[z][i * N + c] = cols[c][i];
        } else {
            for (int c = 0; c < N && c < rows; ++c) A[z][c * N + c] = 1.0;
        }
    }
}

}  // namespace ttn
