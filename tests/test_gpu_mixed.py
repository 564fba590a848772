"""Mixed-precision ABFT Cholesky (abft_potrf with a BF16 / FP16 trailing
update on the tensor cores): exactness on integer data, backward error of
the factor, fault location and correction, no false positives."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U_BF16, U_F16 = 2.0 ** -8, 2.0 ** -11


def run(A, nb, mode, dtype, faults=()):
    T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    rc, rep = abft.potrf(T, nb, mode, dtype=dtype, faults=faults)
    torch.cuda.synchronize()
    return rc, np.tril(T.cpu().numpy()), rep


def events(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16])
@pytest.mark.parametrize("mode", [abft.NONE, abft.SINGLE, abft.FULL])
@pytest.mark.parametrize("n", [256, 300, 640])
def test_integer_exact(dtype, mode, n):
    """Integer L0 with small entries: the per-tile power-of-two scaling, the
    16-bit quantization and the FP32 tensor-core sums are all exact, so the
    mixed factorization returns L0 bit for bit."""
    L0 = W.integer_l0(n, 3)
    A = L0 @ L0.T
    rc, L, rep = run(A, 128, mode, dtype)
    assert rc == 0 and np.array_equal(L, L0)
    assert rep["detected"] == 0


@pytest.mark.parametrize("dtype,u", [(abft.MIXED_BF16, U_BF16), (abft.MIXED_F16, U_F16)])
@pytest.mark.parametrize("n,nb", [(512, 128), (1000, 256), (2048, 256), (2048, 512)])
def test_backward_error_and_no_false_positive(dtype, u, n, nb):
    A = W.spd_mmt(n, seed=500 + n)
    rc, L, rep = run(A, nb, abft.FULL, dtype)
    assert rc == 0
    err = np.linalg.norm(L @ L.T - A) / np.linalg.norm(A)
    assert err <= 4 * u
    Lf = np.linalg.cholesky(A)
    assert np.abs(L - Lf).max() <= 8 * u * np.abs(Lf).max()
    assert rep["detected"] == 0 and rep["max_ratio"] < 1.0


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16])
@pytest.mark.parametrize("mode", [abft.SINGLE, abft.FULL])
def test_fault_located_and_corrected(dtype, mode):
    n, nb = 1024, 128
    A = W.spd_mmt(n, seed=1000)
    rc, Lc, _ = run(A, nb, mode, dtype)
    faults = [(3, abft.F_MEMORY, 900, 700, 1e3), (4, abft.F_COMPUTE, 1000, 650, -1e3),
              (5, abft.F_PANEL, 800, 700, 1e3)]
    rc, L, rep = run(A, nb, mode, dtype, faults)
    assert rc == 0
    assert events(rep) == [(3, 0, 900, 700), (4, 0, 1000, 650), (5, 0, 800, 700)]
    assert rep["corrected"] == 3 and rep["uncorrectable"] == 0
    # a correction is exact to ~ulp(1e3) in FP64; later FP32 panel solves may round
    # one ulp differently, so the factor equals the clean one to FP32 precision
    assert np.abs(L - Lc).max() <= 16 * 2.0 ** -24 * np.abs(Lc).max()


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16])
def test_full_size_n16384(dtype):
    n, nb = 16384, 256
    Ad = W.spd_mmt_torch(n, seed=1000 + n, device=DEV)
    faults = W.fault_schedule(n, nb, "cholesky", seed=2000 + n)
    r = W.rng(7)
    ii = r.integers(0, n, 200); jj = r.integers(0, n, 200)
    ii, jj = np.maximum(ii, jj), np.minimum(ii, jj)
    Aij = Ad[torch.as_tensor(ii, device=DEV), torch.as_tensor(jj, device=DEV)].cpu().numpy()
    rc, rep = abft.potrf(Ad, nb, abft.FULL, dtype=dtype, faults=faults)
    torch.cuda.synchronize()
    assert rc == 0
    assert events(rep) == sorted((f[0], 0, f[2], f[3]) for f in faults)
    assert rep["max_ratio"] < 1.0
    L = torch.tril(Ad)
    Li = L[torch.as_tensor(ii, device=DEV)].cpu().numpy()
    Lj = L[torch.as_tensor(jj, device=DEV)].cpu().numpy()
    u = U_BF16 if dtype == abft.MIXED_BF16 else U_F16
    assert np.abs(np.einsum("ij,ij->i", Li, Lj) - Aij).max() <= 8 * u


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16])
def test_full_size_small_faults(dtype):
    """n = 16384: errors of 1e-2 -- four hundred times below the scalar FP32
    bound 8 u32 n g max a_ii (about 4.1) that the abs-checksum thresholds
    replace -- at 1 per 10 steps are each located at the injected position
    and corrected; the clean tiles stay far below their thresholds."""
    n, nb = 16384, 256
    Ad = W.spd_mmt_torch(n, seed=1000 + n, device=DEV)
    faults = [(f[0], f[1], f[2], f[3], 1e-2) for f in W.fault_schedule(n, nb, "cholesky", seed=2000 + n)]
    rc, rep = abft.potrf(Ad, nb, abft.FULL, dtype=dtype, faults=faults)
    torch.cuda.synchronize()
    assert rc == 0
    assert events(rep) == sorted((f[0], 0, f[2], f[3]) for f in faults)
    assert rep["corrected"] == len(faults) and rep["uncorrectable"] == 0
    assert all(abs(e[4] - 1e-2) < 1e-4 for e in rep["loc"])
    assert rep["tau"] < 5e-3 and rep["max_ratio"] < 1e-2
