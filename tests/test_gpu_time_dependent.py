"""Time-dependent coefficients (ttn_set_coefficients) against the oracle on
the same schedule: the spin-boson model of the 5-node tree with its bias
driven as c(t) = c_0 cos(1.3 t), coefficients held at the step midpoints."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import TTN
from tests.test_oracle_pins import driven_bias

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("TTN_FP64", 1e-10), ("TTN_MIXED", 1e-6)])
def test_driven_spin_boson(gpu_lib, precision, tol):
    p = W.config_c1(eps=1.0)
    coeffs, _ = driven_bias(p, 1.3)
    ctx = gpu_lib.Context(p.tree, getattr(gpu_lib, precision))
    ctx.set_state(p.tensors)
    ctx.set_hamiltonian(p.H)
    ref = TTN(p.tree, p.H, p.tensors)
    worst = 0.0
    for i in range(40):
        c = coeffs((i + 0.5) * p.dt)
        ctx.set_coefficients(c)
        ref.set_coefficients(c)
        ctx.step(p.dt)
        ref.step(p.dt)
        if i % 10 == 9:
            a = np.concatenate(ctx.populations(p.obs_leaves))
            b = np.concatenate(ref.populations(p.obs_leaves))
            worst = max(worst, float(np.abs(a - b).max()))
    ctx.close()
    assert worst <= tol
