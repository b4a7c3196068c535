"""Host-side checks of the multi-set planner (paper Sec. II.A, multi-set
ansatz), on host-resident contexts (no GPU): the channels crossing every
bond -- counted here by brute force -- are, per set, one pre-summed local
channel for its terms acting only inside the subtree and one for those
acting only outside, plus, for the terms crossing the bond (same-set terms
acting on both sides, and every term coupling two sets, whose empty parts
are overlaps rather than identities), per set pair: one single-particle
channel and one grouped mean-field channel per distinct inside part where
the pair has fewer distinct inside than outside parts there, else one
channel per distinct inside part and one per distinct outside part; set
counts that do not match are refused."""
import numpy as np
import pytest

import workloads as W
from tests.test_multiset_oracle import coupled_sop, small_tree


def expected_dims(tree, H):
    out = np.zeros(tree.n, dtype=np.int32)
    for c in range(1, tree.n):
        inside = set(tree.subtree_leaves(c))
        ins, outs, loc, dloc = {}, {}, set(), set()
        for fs, a, b, coef in zip(H.factors, H.bra, H.ket, H.coeffs):
            if coef == 0:
                continue
            fin = tuple(sorted((l, m) for (l, m) in fs if l in inside))
            fout = tuple(sorted((l, m) for (l, m) in fs if l not in inside))
            if a == b:
                if fin and not fout:
                    loc.add(a)
                elif fout and not fin:
                    dloc.add(a)
                elif fin and fout:
                    ins.setdefault((a, b), set()).add(fin); outs.setdefault((a, b), set()).add(fout)
            else:
                ins.setdefault((a, b), set()).add(fin); outs.setdefault((a, b), set()).add(fout)
        crossing = sum(2 * len(ins[k]) if len(ins[k]) < len(outs[k]) else len(ins[k]) + len(outs[k]) for k in ins)
        out[c] = len(loc) + len(dloc) + crossing
    return out


def host_ctx(p_tree, H):
    from paper_2503_15460_gb300 import ttn
    c = ttn.Context(p_tree, ttn.TTN_FP64, on_host=True)
    c.set_multiset_hamiltonian(H)
    return c


@pytest.mark.parametrize("which", ["random", "vibronic"])
def test_multiset_channels_match_brute_force(which):
    if which == "random":
        t = small_tree(False)
        H = coupled_sop(t, np.random.default_rng(3))
    else:
        p = W.multiset_vibronic_problem(n_states=3, n_modes=6, d=6, chi=4)
        t, H = p.tree, p.H
    c = host_ctx(t, H)
    assert c.n_sets() == H.n_sets
    np.testing.assert_array_equal(c.operator_dims(), expected_dims(t, H))
    c.close()


def test_set_count_mismatch_is_refused():
    from paper_2503_15460_gb300 import ttn
    t = small_tree(False)
    H3 = coupled_sop(t, np.random.default_rng(3), S=3)
    H2 = coupled_sop(t, np.random.default_rng(4), S=2)
    c = host_ctx(t, H3)
    with pytest.raises(ttn.TTNError):
        c.set_multiset_hamiltonian(H2)             # a 3-set state cannot take a 2-set operator
    with pytest.raises(ttn.TTNError):
        c.set_multiset_state(W.multiset_product_state(t, [1.0, 0.0]))
    with pytest.raises(ttn.TTNError):
        c.set_state(W.product_state(t, {}))
    c.set_multiset_state(W.multiset_product_state(t, [1.0, 0.0, 0.0]))
    c.set_multiset_hamiltonian(H3)                 # same set count: accepted
    c.close()


def test_bad_set_index_is_refused():
    from paper_2503_15460_gb300 import ttn
    t = small_tree(False)
    H = W.MultiSetSOP(n_sets=2)
    H.add_set(0, 1, 0.5)
    H.ket[0] = 2                                   # outside 0..1
    c = ttn.Context(t, ttn.TTN_FP64, on_host=True)
    with pytest.raises(ttn.TTNError):
        c.set_multiset_hamiltonian(H)
    c.close()


def test_multiset_checkpoint_round_trip_on_the_host():
    """A multi-set checkpoint restores the set count, the operator (channel
    counts), every set's tensors bit for bit and the coefficients' replay;
    a truncated one is refused and leaves the target context unchanged."""
    from paper_2503_15460_gb300 import ttn
    rng = np.random.default_rng(9)
    t = small_tree(False)
    H = coupled_sop(t, rng)
    A = W.multiset_product_state(t, [0.6, 0.48j, 0.64])
    c = host_ctx(t, H)
    c.set_multiset_state(A)
    blob = c.save()
    d = ttn.Context(W.build_tree(("node", 1, [("leaf", 2, 2, "a"), ("leaf", 3, 3, "b")])), ttn.TTN_FP64, on_host=True)
    with pytest.raises(ttn.TTNError):
        d.load(blob[: len(blob) // 2])
    assert d.n_sets() == 1
    d.load(blob)
    assert d.n_sets() == 3
    np.testing.assert_array_equal(d.operator_dims(), c.operator_dims())
    for a in range(3):
        for x, y in zip(c.get_multiset_state(a), d.get_multiset_state(a)):
            np.testing.assert_array_equal(x, y)
    d.set_coefficients(np.asarray(H.coeffs) * 0.5)      # the stored set pairs are replayed
    assert d.n_sets() == 3
    np.testing.assert_array_equal(d.operator_dims(), c.operator_dims())
    c.close()
    d.close()
