"""Host-resident contexts (ttn_create_host): the host logic behind admission
by device-memory footprint, exercised without a GPU."""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_2503_15460_gb300 import ttn
    return ttn


def host_ctx(lib, p, precision=None):
    c = lib.Context(p.tree, lib.TTN_MIXED if precision is None else precision, on_host=True)
    c.set_state(p.tensors)
    c.set_hamiltonian(p.H)
    return c


def test_host_context_holds_no_device_memory(lib):
    p = W.config_c1()
    c = host_ctx(lib, p)
    assert c.device_bytes() == 0
    assert c.footprint() > 0
    for a, b in zip(c.get_state(), p.tensors):
        assert np.array_equal(a, b)
    assert np.array_equal(c.bond_dims()[1:], p.tree.bond_dim[1:])
    steps, flops, stamps = lib.ttn_step_stats(c.h)
    assert steps == 0 and flops == 0.0 and stamps.size == 0
    c.evict()                       # already on the host: no-op
    c.close()


def test_footprint_grows_with_bond_dimension(lib):
    small = host_ctx(lib, W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6)))
    large = host_ctx(lib, W.config_c2(bonds=(12, 8, 6, 4), d_range=(4, 6)))
    assert large.footprint() > small.footprint()
    # complex128 bulk storage needs more than the mixed form of the same problem
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    assert host_ctx(lib, p, lib.TTN_FP64).footprint() > host_ctx(lib, p, lib.TTN_MIXED).footprint()


def test_footprint_covers_krylov_workspace(lib):
    """The state arena holds (Krylov dimension + 4) workspace vectors of the
    largest node tensor, so the footprint is at least that."""
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    smax = max(int(np.prod(a.shape)) for a in p.tensors)
    c = host_ctx(lib, p, lib.TTN_FP64)
    assert c.footprint() >= (32 + 4) * smax * 16


def test_host_context_validates_hamiltonian(lib):
    p = W.config_c1()
    c = lib.Context(p.tree, lib.TTN_MIXED, on_host=True)
    H = W.SOP()
    H.add(1.0, (0, np.eye(2)))      # node 0 is not a leaf
    with pytest.raises(lib.TTNError) as e:
        c.set_hamiltonian(H)
    assert e.value.status == lib.TTN_E_INVALID
    c.close()


def test_request_generator_shapes():
    """Serving requests: the stated ranges and both model families."""
    rs = W.config_c5_requests(64, seed=5)
    assert {r["kind"] for r in rs} == {"sb", "vib"}
    for r in rs:
        assert 8 <= r["n_modes"] <= 128 and 8 <= r["d"] <= 20 and 8 <= r["chi"] <= 48
        assert 100 <= r["steps"] <= 400
    small = W.config_c5_requests(6, seed=5, n_modes_range=(3, 6), d_range=(4, 6), chi_range=(2, 4),
                                 steps_range=(4, 8))
    for r in small:
        p = W.c5_problem(r)
        assert p.nsteps == r["steps"]
        assert p.dt == (0.05 if r["kind"] == "sb" else 0.1)
        assert len(p.obs_leaves) == r["n_modes"] + 1


def test_set_coefficients_on_host_context(lib):
    p = W.config_c1(eps=1.0)
    c = host_ctx(lib, p)
    fp = c.footprint()
    coeff = np.array(p.H.coeffs, dtype=np.complex128)
    coeff[0] *= 0.5
    c.set_coefficients(coeff)                       # same factors: accepted, no device work
    assert c.device_bytes() == 0 and c.footprint() == fp
    with pytest.raises(lib.TTNError) as e:
        c.set_coefficients(coeff[:-1])
    assert e.value.status == lib.TTN_E_INVALID
    bad = coeff.copy()
    bad[1] = np.nan
    with pytest.raises(lib.TTNError) as e:
        c.set_coefficients(bad)
    assert e.value.status == lib.TTN_E_INVALID
    c.close()


def test_checkpoint_round_trip_on_host(lib):
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    a = host_ctx(lib, p)
    blob = a.save()
    # load into a context built on another tree: tree, state and H are replaced
    q = W.config_c1()
    b = lib.Context(q.tree, lib.TTN_MIXED, on_host=True)
    b.load(blob)
    assert b.device_bytes() == 0
    assert b.footprint() == a.footprint()
    assert np.array_equal(b.bond_dims(), a.bond_dims())
    assert np.array_equal(b.tree.parent, p.tree.parent)     # tree view follows the load
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert b.save() == blob
    a.close(); b.close()


def test_checkpoint_rejects_bad_streams(lib):
    p = W.config_c1()
    a = host_ctx(lib, p)
    blob = a.save()
    for bad in (b"not a checkpoint", blob[: len(blob) // 2], b"\x00" * 64):
        with pytest.raises(lib.TTNError) as e:
            a.load(bad)
        assert e.value.status == lib.TTN_E_INVALID
    # the context is unchanged after the failed loads
    assert a.save() == blob
    a.close()


def test_tree_query_follows_the_context(lib):
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    c = host_ctx(lib, p)
    parent, phys, bond = lib.ttn_tree(c.h)
    assert np.array_equal(parent, p.tree.parent)
    assert np.array_equal(phys, p.tree.phys_dim)
    assert np.array_equal(bond[1:], p.tree.bond_dim[1:]) and bond[0] == 1
    c.close()
