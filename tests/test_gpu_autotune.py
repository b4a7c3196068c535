"""The autotuner (ttn_autotune): candidate launch shapes and mode-product
routines are timed on the context's own problem from one snapshot; the
context ends bit-identical to how it began, the chosen configuration keeps
the oracle's results, and a configuration copied to another context gives
the same bits as the tuned one."""
import numpy as np
import pytest

import workloads as W
from oracle.ttn import TTN

pytestmark = pytest.mark.gpu


def ctx_of(lib, p, precision):
    c = lib.Context(p.tree, precision)
    c.set_state(p.tensors)
    c.set_hamiltonian(p.H)
    return c


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_autotune_keeps_state_and_oracle_parity(gpu_lib, precision, tol):
    p = W.config_c2(bonds=(6, 4, 3, 2), d_range=(4, 6))
    c = ctx_of(gpu_lib, p, precision)
    c.step(p.dt, 1)
    before = c.get_state()
    flags = 7 if precision == gpu_lib.TTN_MIXED else 3
    c.autotune(p.dt, 2, flags)
    after = c.get_state()
    for x, y in zip(before, after):
        assert np.array_equal(x, y)                      # tuning left the state as it was
    t = c.tuning()
    assert t["trials"] >= 3 and t["tuned_ms"] > 0 and t["tuned_ms"] <= t["default_ms"]
    ref = TTN(p.tree, p.H, p.tensors)
    ref.step(p.dt, 4)
    c.step(p.dt, 3)
    got = np.concatenate(c.populations(p.obs_leaves))
    want = np.concatenate(ref.populations(p.obs_leaves))
    assert np.abs(got - want).max() <= tol
    # the same configuration on a fresh context gives the same bits
    d = ctx_of(gpu_lib, p, precision)
    d.set_tuning(t["blocks"], t["variants"])
    d.step(p.dt, 4)
    for x, y in zip(c.get_state(), d.get_state()):
        assert np.array_equal(x, y)
    c.close()
    d.close()
