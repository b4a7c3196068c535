"""The allocation-free effective-Hamiltonian entry point.

Callers that cannot allocate device memory during a call (a serving loop
whose memory belongs to its own pool allocator, or code that must avoid the
synchronisation cudaMalloc may cause) use ttn_heff_apply_noalloc, whose
scratch is a static device array.  It must give the same result as the
allocating ttn_heff_apply, also on a second call that reuses the array
left over from the first.  This file is named so that pytest collects it
last."""
import numpy as np
import pytest

from tests.test_gpu_heff import random_operator

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_on_two_calls(gpu_lib):
    import torch
    dev = torch.device("cuda")
    for call, (dims, n_terms, n_mats) in enumerate([((16, 16, 24), 9, 7), ((8, 6, 5, 7), 12, 9)]):
        rng = np.random.default_rng(100 + call)
        coeff, factor, mats = random_operator(rng, dims, n_terms, n_mats)
        x = rng.standard_normal(dims) + 1j * rng.standard_normal(dims)
        xd = torch.from_numpy(x).to(dev)
        md = [torch.from_numpy(np.ascontiguousarray(m)).to(dev) for m in mats]
        ptrs = [m.data_ptr() for m in md]
        y_alloc = torch.zeros_like(xd)
        y_noalloc = torch.full_like(xd, complex(np.nan, np.nan))   # output must be fully written
        torch.cuda.synchronize()
        gpu_lib.ttn_heff_apply(0, dims, coeff, factor, ptrs, xd.data_ptr(), y_alloc.data_ptr())
        gpu_lib.ttn_heff_apply_noalloc(0, dims, coeff, factor, ptrs, xd.data_ptr(), y_noalloc.data_ptr())
        a, b = y_alloc.cpu().numpy(), y_noalloc.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_noalloc_rejects_oversized_tensor(gpu_lib):
    import torch
    dims = (64, 64, 9)                       # 36864 elements > 32768
    x = torch.zeros(dims, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(gpu_lib.TTNError) as e:
        gpu_lib.ttn_heff_apply_noalloc(0, dims, [1.0], [[-1, -1, -1]], [], x.data_ptr(), y.data_ptr())
    assert e.value.status == gpu_lib.TTN_E_INVALID
    assert "32768" in str(e.value)
