"""Automatic hierarchical-SOP construction (paper Sec. II.B.2): for every
bond the library sums the terms that act on both sides into channels chosen
by a minimum vertex cover of the bipartite graph of their distinct inside
and outside parts.  Checked on the host (no GPU): the operator bond
dimensions it reports equal one channel for the purely inside terms, one for
the purely outside terms, plus the minimum vertex cover computed here by
brute force over subsets of inside parts -- including SOPs where neither
uniform grouping direction is minimal."""
import itertools

import numpy as np
import pytest

import workloads as W


def expected_dims(tree, H):
    """has_in + has_out + min vertex cover, per bond (index = child node)."""
    terms = [frozenset(f) for f in H.factors if f]
    out = np.zeros(tree.n, dtype=np.int32)
    for c in range(1, tree.n):
        inside = set(tree.subtree_leaves(c))
        has_in = has_out = False
        edges = set()
        for t in terms:
            a = tuple(sorted((l, m) for (l, m) in t if l in inside))
            b = tuple(sorted((l, m) for (l, m) in t if l not in inside))
            if a and not b:
                has_in = True
            elif b and not a:
                has_out = True
            else:
                edges.add((a, b))
        L = sorted({e[0] for e in edges})
        best = 0
        if edges:
            best = len(L) + len({e[1] for e in edges})
            for k in range(len(L) + 1):
                for S in itertools.combinations(L, k):
                    S = set(S)
                    right = {e[1] for e in edges if e[0] not in S}
                    best = min(best, len(S) + len(right))
        out[c] = int(has_in) + int(has_out) + best
    return out


def uniform_dims(tree, H):
    """The same count with one grouping direction per bond (the smaller of
    the distinct inside / outside parts)."""
    terms = [frozenset(f) for f in H.factors if f]
    out = np.zeros(tree.n, dtype=np.int32)
    for c in range(1, tree.n):
        inside = set(tree.subtree_leaves(c))
        ins, outs, hi, ho = set(), set(), False, False
        for t in terms:
            a = tuple(sorted((l, m) for (l, m) in t if l in inside))
            b = tuple(sorted((l, m) for (l, m) in t if l not in inside))
            if a and not b:
                hi = True
            elif b and not a:
                ho = True
            else:
                ins.add(a); outs.add(b)
        out[c] = int(hi) + int(ho) + (min(len(ins), len(outs)) if ins else 0)
    return out


def cross_problem():
    """root(L(l1, l2), R(r1, r2)) with terms A1 B1, A1 B2, A1 B3, A2 B1, A3 B1
    across the root bonds (A on l1, B on r1) plus local terms: on each of
    those bonds 3 distinct inside and 3 distinct outside parts, but a cover
    of 2 ({A1, B1})."""
    spec = ("node", 1, [("node", 4, [("leaf", 3, 3, "l1"), ("leaf", 3, 3, "l2")]),
                        ("node", 4, [("leaf", 3, 3, "r1"), ("leaf", 3, 3, "r2")])])
    t = W.build_tree(spec)
    rng = np.random.default_rng(11)

    def herm():
        X = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        return (X + X.conj().T) / 2

    z = {lab: t.leaf_of_label(lab) for lab in ("l1", "l2", "r1", "r2")}
    A = [herm() for _ in range(3)]
    B = [herm() for _ in range(3)]
    H = W.SOP()
    for lab in z:
        H.add(0.5, (z[lab], herm()))
    H.add(0.3, (z["l2"], herm()), (z["l1"], herm()))          # inside L only
    for i, j in [(0, 0), (0, 1), (0, 2), (1, 0), (2, 0)]:
        H.add(0.2 + 0.1 * i - 0.05 * j, (z["l1"], A[i]), (z["r1"], B[j]))
    vecs = {}
    for lab in z:
        v = rng.normal(size=3) + 1j * rng.normal(size=3)
        vecs[z[lab]] = v / np.linalg.norm(v)
    return W.Problem("cross", t, H, W.product_state(t, vecs), 0.05, 10, sorted(z.values()), {})


def random_sop_problem(seed, n_leaves=6, d=3, pool=3, n_terms=18):
    """A balanced tree over n_leaves leaves and a random Hermitian SOP whose
    two- and three-body terms draw their factors from a small pool per leaf,
    so inside and outside parts repeat across terms."""
    leaves = [("leaf", d, d, f"q{k}") for k in range(n_leaves)]
    t = W.build_tree(("node", 1, [W.balanced_spec(leaves[:n_leaves // 2], 4),
                                  W.balanced_spec(leaves[n_leaves // 2:], 4)]))
    rng = np.random.default_rng(seed)

    def herm():
        X = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        return (X + X.conj().T) / 2

    lv = [t.leaf_of_label(f"q{k}") for k in range(n_leaves)]
    mats = {l: [herm() for _ in range(pool)] for l in lv}
    H = W.SOP()
    for l in lv:
        H.add(0.5, (l, herm()))
    for _ in range(n_terms):
        k = int(rng.integers(2, 4))
        ls = rng.choice(lv, size=k, replace=False)
        H.add(float(rng.normal(0.0, 0.2)), *[(int(l), mats[int(l)][int(rng.integers(pool))]) for l in ls])
    vecs = {}
    for l in lv:
        v = rng.normal(size=d) + 1j * rng.normal(size=d)
        vecs[l] = v / np.linalg.norm(v)
    return W.Problem(f"random_sop{seed}", t, H, W.product_state(t, vecs), 0.05, 10, lv, {})


def host_dims(p):
    from paper_2503_15460_gb300 import ttn
    c = ttn.Context(p.tree, ttn.TTN_FP64, on_host=True)
    c.set_hamiltonian(p.H)
    d = c.operator_dims()
    c.close()
    return d


def test_cross_bond_uses_the_minimum_cover():
    p = cross_problem()
    got, want, uni = host_dims(p), expected_dims(p.tree, p.H), uniform_dims(p.tree, p.H)
    np.testing.assert_array_equal(got, want)
    assert np.any(want < uni)                 # neither uniform direction is minimal there


@pytest.mark.parametrize("seed", range(12))
def test_random_sops_match_brute_force_cover(seed):
    p = random_sop_problem(seed)
    np.testing.assert_array_equal(host_dims(p), expected_dims(p.tree, p.H))


def test_some_random_sop_needs_a_mixed_cover():
    assert any(np.any(expected_dims(p.tree, p.H) < uniform_dims(p.tree, p.H))
               for p in (random_sop_problem(s) for s in range(12)))
