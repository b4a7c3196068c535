"""The hierarchical SOP built from minimum vertex covers (Sec. II.B.2,
tests/test_hsop.py checks its channel counts) is exactly the plain SOP: the
GPU trajectory on SOPs whose covers mix both grouping directions equals the
oracle's, which applies every term separately."""
import numpy as np
import pytest

from oracle.ttn import TTN
from tests.test_hsop import cross_problem, random_sop_problem, expected_dims, uniform_dims

pytestmark = pytest.mark.gpu


def mixed_cover_problems():
    ps = [cross_problem()]
    for s in range(12):
        p = random_sop_problem(s)
        if np.any(expected_dims(p.tree, p.H) < uniform_dims(p.tree, p.H)):
            ps.append(p)
        if len(ps) == 3:
            break
    return ps


# complex128 checks the operator structure exactly.  The complex64 bulk meets
# 1e-6 on the physical workloads; these test operators are dense random
# Hermitian 3 x 3 factors of norm ~1-3 on every leaf, so 20 steps of complex64
# rounding (6e-8 relative) through ~40 exponentials each reach a few 1e-6
# (measured 3.5e-6): the mixed case is held to 1e-5.
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_mixed_cover_sop_matches_oracle(gpu_lib, precision, tol):
    for p in mixed_cover_problems():
        ref = TTN(p.tree, p.H, p.tensors)
        c = gpu_lib.Context(p.tree, precision)
        c.set_state(p.tensors)
        c.set_hamiltonian(p.H)
        np.testing.assert_array_equal(c.operator_dims(), expected_dims(p.tree, p.H))
        for _ in range(4):
            ref.step(p.dt, 5)
            c.step(p.dt, 5)
            a = np.concatenate(c.populations(p.obs_leaves))
            b = np.concatenate(ref.populations(p.obs_leaves))
            assert np.abs(a - b).max() <= tol, (p.name, np.abs(a - b).max())
        n2, e = c.norm_energy()
        assert abs(n2 - 1.0) <= (1e-11 if precision == 0 else 1e-5)
        # energies: the complex64 path works with H minus its local zero points and adds them back
        assert abs(e.real - ref.energy().real) <= (1e-10 if precision == 0 else 1e-5) * max(1.0, abs(ref.energy()))
        c.close()
