"""Failure detection without a GPU fault: a Krylov exponential that cannot
converge (dimension 1, unreachable tolerance) makes the device halve the
interval up to 4096 substeps and then report non-convergence through its
status word -- bounded work, no trap, no hang.  The host turns the status
into TTN_E_NOCONV and marks the context failed; the request server retires
such a request with that status while the others complete."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def bad_opts(lib):
    return lib.ttn_step_opts(krylov_tol=1e-300, krylov_maxdim=1)


def test_device_failure_marks_context(gpu_lib):
    p = W.config_c1()
    ctx = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    ctx.set_state(p.tensors)
    ctx.set_hamiltonian(p.H)
    with pytest.raises(gpu_lib.TTNError) as e:
        ctx.step(p.dt, 1, bad_opts(gpu_lib))
    assert e.value.status == gpu_lib.TTN_E_NOCONV
    assert "converge" in gpu_lib.ttn_last_error(ctx.h)
    with pytest.raises(gpu_lib.TTNError) as e:
        ctx.step(p.dt, 1)                       # a failed context refuses further work
    assert e.value.status == gpu_lib.TTN_E_STATE
    ctx.close()
    # the device stays usable for everyone else
    ok = gpu_lib.Context(p.tree, gpu_lib.TTN_FP64)
    ok.set_state(p.tensors)
    ok.set_hamiltonian(p.H)
    ok.step(p.dt, 2)
    ok.close()


def test_server_isolates_a_failing_request(gpu_lib):
    rs = W.config_c5_requests(4, seed=5, n_modes_range=(3, 6), d_range=(4, 6), chi_range=(2, 4), steps_range=(4, 6))
    probs = [W.c5_problem(r) for r in rs]
    srv = gpu_lib.Server(gpu_lib.TTN_MIXED, slice_ms=0.5)
    tickets = {}
    ctxs = []
    for i, p in enumerate(probs):
        c = gpu_lib.Context(p.tree, gpu_lib.TTN_MIXED, on_host=True)
        c.set_state(p.tensors)
        c.set_hamiltonian(p.H)
        tickets[srv.submit(c, p.dt, p.nsteps, bad_opts(gpu_lib) if i == 1 else None)] = i
        ctxs.append(c)
    srv.drain()
    status = {tickets[t]: s for t, s in srv.poll()}
    assert status[1] == gpu_lib.TTN_E_NOCONV
    assert all(status[i] == gpu_lib.TTN_OK for i in (0, 2, 3))
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 3 and st["bytes_in_use"] == 0
    srv.close()
    for c in ctxs:
        c.close()
