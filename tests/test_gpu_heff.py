"""GPU parity of the effective-Hamiltonian kernel (paper Eq. psi_eom_1) on
caller-owned device buffers against the oracle's mode products."""
import numpy as np
import pytest

from oracle.ttn import mode_product

pytestmark = pytest.mark.gpu


def random_operator(rng, dims, n_terms, n_mats, share_last=True):
    D = len(dims)
    mats, mat_dim = [], []
    for i in range(n_mats):
        j = i % D
        d = dims[j]
        mats.append(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)))
        mat_dim.append(j)
    factor = -np.ones((n_terms, D), dtype=np.int32)
    for t in range(n_terms):
        for j in range(D):
            cands = [i for i in range(n_mats) if mat_dim[i] == j]
            if cands and rng.random() < 0.5:
                factor[t, j] = rng.choice(cands)
    if share_last:                       # several terms ending in the same matrix
        last = [i for i in range(n_mats) if mat_dim[i] == D - 1][0]
        factor[: n_terms // 2, D - 1] = last
    factor[-1, :] = -1                   # a constant term
    coeff = rng.standard_normal(n_terms) + 1j * rng.standard_normal(n_terms)
    return coeff, factor, mats


def oracle_apply(x, coeff, factor, mats):
    y = np.zeros_like(x)
    for t, c in enumerate(coeff):
        T = x
        for j, f in enumerate(factor[t]):
            if f >= 0:
                T = mode_product(mats[f], T, j)
        y += c * T
    return y


@pytest.mark.parametrize("dims,n_terms,n_mats", [
    ((16, 16, 24), 9, 7),
    ((8, 6, 5, 7), 12, 9),
    ((30, 8), 5, 4),
    ((4, 4, 4, 4, 4, 3), 10, 12),
    ((48, 2), 4, 3),
])
def test_heff_apply_matches_oracle(gpu_lib, dims, n_terms, n_mats):
    import torch
    rng = np.random.default_rng(sum(dims) + n_terms)
    coeff, factor, mats = random_operator(rng, dims, n_terms, n_mats)
    x = rng.standard_normal(dims) + 1j * rng.standard_normal(dims)
    dev = torch.device("cuda")
    xd = torch.from_numpy(x).to(dev)
    md = [torch.from_numpy(np.ascontiguousarray(m)).to(dev) for m in mats]
    yd = torch.zeros_like(xd)
    torch.cuda.synchronize()
    gpu_lib.ttn_heff_apply(0, dims, coeff, factor, [m.data_ptr() for m in md], xd.data_ptr(), yd.data_ptr())
    got = yd.cpu().numpy()
    want = oracle_apply(x, coeff, factor, mats)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_heff_apply_rejects_bad_input(gpu_lib):
    with pytest.raises(gpu_lib.TTNError) as e:
        gpu_lib.ttn_heff_apply(0, [4, 65], [1.0], [[-1, -1]], [], 1, 2)
    assert e.value.status == gpu_lib.TTN_E_INVALID
