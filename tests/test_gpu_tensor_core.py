"""The complex64 mode product (Sec. II.C Eq. psi_eom_1, one tensor index)
on the tcgen05 tensor cores with 3xTF32 split products, against an FP64
reference of the same product and against the FFMA routine of the sweep.
3xTF32 keeps the FP32 rounding level: each product carries a relative error
of about 2^-22 (the dropped lo*lo term and TF32 rounding of lo), so with
n terms the error is bounded by a few n * 2^-23 of sum |M| |x|."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def run(gpu_lib, L, n, R, w, accumulate, tensor_cores, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    x = (rng.normal(size=(L, n, R)) + 1j * rng.normal(size=(L, n, R))).astype(np.complex64)
    M = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))).astype(np.complex64)
    y0 = (rng.normal(size=(L, n, R)) + 1j * rng.normal(size=(L, n, R))).astype(np.complex64)
    dx = torch.from_numpy(x.view(np.float32).copy()).cuda()
    dM = torch.from_numpy(M.view(np.float32).copy()).cuda()
    dy = torch.from_numpy(y0.view(np.float32).copy()).cuda()
    torch.cuda.synchronize()
    gpu_lib.ttn_mode_product_c64(0, L, n, R, dM.data_ptr(), dx.data_ptr(), dy.data_ptr(), w, accumulate,
                                 tensor_cores)
    got = dy.cpu().numpy().view(np.complex64).reshape(L, n, R).astype(np.complex128)
    want = w * np.einsum("pm,lmr->lpr", M.astype(np.complex128), x.astype(np.complex128))
    if accumulate:
        want = want + y0.astype(np.complex128)
    scale = np.einsum("pm,lmr->lpr", np.abs(M).astype(np.float64), np.abs(x).astype(np.float64)) * abs(w)
    if accumulate:
        scale = scale + np.abs(y0)
    return got, want, scale


@pytest.mark.parametrize("L,n,R", [(2304, 48, 1), (48, 48, 48), (1, 48, 2304), (300, 24, 7), (513, 8, 1),
                                   (20, 20, 20), (130, 64, 3)])
def test_tensor_core_mode_product_matches_fp64(gpu_lib, L, n, R):
    got, want, scale = run(gpu_lib, L, n, R, 0.7 - 0.3j, True, True)
    err = np.abs(got - want)
    assert np.all(err <= 8 * n * 2.0**-23 * scale + 1e-30), float((err / scale).max())


def test_tensor_core_agrees_with_ffma_routine(gpu_lib):
    a, want, scale = run(gpu_lib, 96, 48, 48, 1.0, False, True, seed=3)
    b, _, _ = run(gpu_lib, 96, 48, 48, 1.0, False, False, seed=3)
    assert np.all(np.abs(a - b) <= 8 * 48 * 2.0**-23 * scale)
    assert np.all(np.abs(b - want) <= 8 * 48 * 2.0**-23 * scale)
