"""Entry points not exercised elsewhere, through the C ABI: product states
from leaf vectors, single-leaf expectation values, the flop and cycle
counters, running on a caller's CUDA stream, and error messages."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import TTN

pytestmark = pytest.mark.gpu


def test_product_state_and_expectations(gpu_lib):
    p = W.config_c1()
    spin = p.meta["spin"]
    rng = np.random.default_rng(21)
    vecs = {l: rng.normal(size=int(p.tree.phys_dim[l])) + 1j * rng.normal(size=int(p.tree.phys_dim[l]))
            for l in p.tree.leaves()}
    ctx = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    gpu_lib.ttn_set_product_state(ctx.h, vecs, p.tree.n)
    ctx.set_hamiltonian(p.H)
    ref = TTN(p.tree, p.H, W.product_state(p.tree, vecs))
    ctx.step(p.dt, 3)
    ref.step(p.dt, 3)
    a = np.concatenate(ctx.populations(p.obs_leaves))
    b = np.concatenate(ref.populations(p.obs_leaves))
    assert np.abs(a - b).max() <= 1e-10
    sz = np.diag([1.0, -1.0]).astype(np.complex128)
    sx = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    got = gpu_lib.ttn_expect(ctx.h, [spin, spin], [sz, sx])
    rho = ref.reduced_density(spin)
    want = [np.trace(rho @ sz), np.trace(rho @ sx)]
    assert np.abs(got - np.array(want)).max() <= 1e-10
    ctx.close()


def test_flop_and_cycle_counters(gpu_lib):
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    for prec in (gpu_lib.TTN_FP64, gpu_lib.TTN_MIXED):
        ctx = gpu_lib.Context(p.tree, prec)
        ctx.set_state(p.tensors)
        ctx.set_hamiltonian(p.H)
        t0, f0 = gpu_lib.ttn_flop_counts(ctx.h)
        ctx.step(p.dt, 2)
        t1, f1 = gpu_lib.ttn_flop_counts(ctx.h)
        assert t1 > t0 and f1 > f0
        if prec == gpu_lib.TTN_FP64:
            assert f1 - f0 == pytest.approx(t1 - t0, rel=1e-12)     # everything in complex128
        else:
            assert 0.0 < f1 - f0 < 0.5 * (t1 - t0)                 # QR / absorption only
        cyc = gpu_lib.ttn_op_cycles(ctx.h)
        for k in ("qr_down", "qr_up", "env", "evolve", "in:heff"):
            assert cyc.get(k, 0) > 0
        ctx.close()


def test_caller_stream(gpu_lib):
    import torch
    p = W.config_c1()
    s = torch.cuda.Stream()
    a = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    gpu_lib.ttn_set_stream(a.h, s.cuda_stream)
    a.set_state(p.tensors)
    a.set_hamiltonian(p.H)
    a.step(p.dt, 4)
    b = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    b.set_state(p.tensors)
    b.set_hamiltonian(p.H)
    b.step(p.dt, 4)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    a.close(); b.close()


def test_error_messages(gpu_lib):
    p = W.config_c1()
    ctx = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    with pytest.raises(gpu_lib.TTNError) as e:
        ctx.step(p.dt, 1)
    assert e.value.status == gpu_lib.TTN_E_STATE
    assert "Hamiltonian" in gpu_lib.ttn_last_error(ctx.h)
    with pytest.raises(gpu_lib.TTNError):
        gpu_lib.ttn_create([0, 0], [0, 2], [1, 2])        # parent of the root must be -1
    assert gpu_lib.ttn_last_error(None) != ""
    ctx.close()
