"""GPU parity of the FP64-accurate symmetric product on the BF16 tensor cores
(abft_symm_emu, the product of the refinement residuals) against the
extended-precision definition: exact on integer data, within the stated
bound n 2^-55 (row scale)(column scale) elsewhere -- including rows scaled by
powers of two far apart, ragged sizes and several 16-column blocks."""
import numpy as np
import pytest
import torch

from oracle import products
from paper_2301_03166_b300 import abft

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def run(A, X):
    Y = abft.symm_emu(torch.from_numpy(np.ascontiguousarray(A)).to(DEV),
                      torch.from_numpy(np.ascontiguousarray(X)).to(DEV))
    torch.cuda.synchronize()
    return Y.cpu().numpy()


def scale(v):
    """2^(e - 1022) with e the largest biased exponent of v: the splitting's scale."""
    m = np.abs(v).max()
    return 0.0 if m == 0 else 2.0 ** (np.frexp(m)[1])


def check_bound(A, X, Y):
    n = A.shape[0]
    S = products.symm_lower(A)
    ref = products.symm_product(A, X)
    err = np.abs(Y.astype(np.longdouble) - ref)
    rs = np.array([scale(S[i]) for i in range(n)])
    cs = np.array([scale(X[:, r]) for r in range(X.shape[1])])
    bound = n * 2.0 ** -55 * np.outer(rs, cs) * 4 + 1e-300
    assert np.all(err <= bound), float((err / bound).max())
    return err, ref


def test_integer_data_is_exact():
    rng = np.random.default_rng(1)
    n = 256
    A = rng.integers(-3, 4, (n, n)).astype(np.float64)
    X = rng.integers(-5, 6, (n, 16)).astype(np.float64)
    Y = run(A, X)
    S = products.symm_lower(A).astype(np.int64)
    assert np.array_equal(Y, (S @ X.astype(np.int64)).astype(np.float64))


@pytest.mark.parametrize("n,nrhs", [(1120, 16), (1024, 5), (544, 37)])
def test_random_within_bound(n, nrhs):
    rng = np.random.default_rng(n + nrhs)
    M = rng.standard_normal((n, n))
    A = M @ M.T / n + np.eye(n)
    X = rng.standard_normal((n, nrhs))
    Y = run(A, X)
    err, ref = check_bound(A, X, Y)
    # at least as accurate as the same product in FP64 arithmetic
    y64 = products.symm_lower(A) @ X
    err64 = np.abs(y64.astype(np.longdouble) - ref)
    assert err.max() <= 2 * err64.max()


def test_rows_scaled_by_far_apart_powers_of_two():
    rng = np.random.default_rng(7)
    n = 512
    M = rng.standard_normal((n, n))
    A = M @ M.T / n + np.eye(n)
    d = 2.0 ** rng.integers(-300, 300, n).astype(np.float64)
    A = A * d[:, None] * d[None, :]
    X = rng.standard_normal((n, 16)) * 2.0 ** rng.integers(-100, 100, 16)[None, :]
    Y = run(A, X)
    check_bound(A, X, Y)


def test_zero_and_upper_triangle_ignored():
    n = 128
    A = np.triu(np.full((n, n), np.nan), 1)   # the strict upper triangle is never read
    A[np.tril_indices(n)] = 0.0
    X = np.ones((n, 3))
    assert np.array_equal(run(A, X), np.zeros((n, 3)))


def test_unsupported_order():
    A = torch.eye(100, dtype=torch.float64, device=DEV)
    with pytest.raises(abft.AbftError):
        abft.symm_emu(A, torch.ones(100, 2, dtype=torch.float64, device=DEV))
