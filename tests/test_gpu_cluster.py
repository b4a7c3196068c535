"""One instance spread over a thread-block cluster: the node updates' mode
products, Gram contractions, Krylov recurrences, Householder QR, subspace
expansion and eigensolver shared by 2..16 blocks give the oracle's results
(paper Sec. II.C-II.D), in both precisions, on trees small enough to be
spread thinly (many blocks idle) and on the full-size vibronic tree."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import TTN, ExpandingTTN

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-6


def gpu_ctx(lib, p, precision, blocks):
    c = lib.Context(p.tree, precision)
    c.set_cluster(blocks)
    c.set_state(p.tensors)
    c.set_hamiltonian(p.H)
    return c


def trajectory_error(lib, p, nsteps, every, precision, blocks):
    ref = TTN(p.tree, p.H, p.tensors)
    c = gpu_ctx(lib, p, precision, blocks)
    assert c.cluster() == blocks
    worst = 0.0
    for _ in range(nsteps // every):
        ref.step(p.dt, every)
        c.step(p.dt, every)
        a = np.concatenate(c.populations(p.obs_leaves))
        b = np.concatenate(ref.populations(p.obs_leaves))
        worst = max(worst, float(np.abs(a - b).max()))
    c.close()
    return worst


@pytest.mark.parametrize("blocks", [2, 4, 16])
def test_spin_boson_fp64_on_cluster(gpu_lib, blocks):
    assert trajectory_error(gpu_lib, W.config_c1(), 40, 10, gpu_lib.TTN_FP64, blocks) <= FP64_TOL


def test_spin_boson_mixed_on_cluster(gpu_lib):
    assert trajectory_error(gpu_lib, W.config_c1(), 40, 10, gpu_lib.TTN_MIXED, 4) <= MIXED_TOL


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_vibronic_reduced_on_cluster(gpu_lib, precision, tol):
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    assert trajectory_error(gpu_lib, p, 6, 3, precision, 8) <= tol


def test_local_dimension_above_one_block(gpu_lib):
    """Leaves of dimension 48: their reduced densities need the Gram tile
    layout of a cluster block (more than 45 values per index), so the
    context runs on a cluster even when one block is requested."""
    p = W.config_c1(d=48)
    c = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64, 1)
    assert c.cluster() >= 2
    c.close()
    assert trajectory_error(gpu_lib, p, 10, 5, gpu_lib.TTN_FP64, 2) <= FP64_TOL


def test_expansion_on_cluster(gpu_lib):
    p = W.config_c1(chi=2, d=4)
    ctx = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64, 4)
    ref = ExpandingTTN(p.tree, p.H, p.tensors)
    opts = gpu_lib.ttn_step_opts(expand=1, eps_spawn=1e-6, chi_max=6)
    worst = 0.0
    for _ in range(8):
        ref.step_adaptive(p.dt, 1e-6, 6, 1)
        ctx.step(p.dt, 1, opts)
        assert np.array_equal(ctx.bond_dims()[1:], ref.t.bond_dim[1:])
        a = np.concatenate(ctx.populations(p.obs_leaves))
        b = np.concatenate(ref.populations(p.obs_leaves))
        worst = max(worst, float(np.abs(a - b).max()))
    assert np.any(ctx.bond_dims()[1:] > p.tree.bond_dim[1:])
    ctx.close()
    assert worst <= FP64_TOL


def test_ground_state_on_cluster(gpu_lib):
    from tests.test_oracle_pins import random_canonical
    p = W.config_c1()
    A0 = random_canonical(p.tree, np.random.default_rng(3))
    ref = TTN(p.tree, p.H, A0)
    want = np.array(ref.ground_state(3))
    c = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    c.set_cluster(4)
    c.set_state(A0)
    c.set_hamiltonian(p.H)
    got = np.asarray(c.ground_state(3))
    pg = np.concatenate(c.populations(p.obs_leaves))
    c.close()
    pr = np.concatenate(ref.populations(p.obs_leaves))
    assert np.abs(got - want).max() <= 1e-10
    assert np.abs(pg - pr).max() <= 1e-9


def test_vibronic_full_size_on_cluster_matches_one_block(gpu_lib):
    """The 46-node vibronic tree on 16 blocks against one block (both
    complex128): the same trajectory up to rounding."""
    p = W.config_c2()
    a = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64, 16)
    b = gpu_ctx(gpu_lib, p, gpu_lib.TTN_FP64, 1)
    a.step(p.dt, 2)
    b.step(p.dt, 2)
    x = np.concatenate(a.populations(p.obs_leaves))
    y = np.concatenate(b.populations(p.obs_leaves))
    a.close()
    b.close()
    assert np.abs(x - y).max() <= FP64_TOL
