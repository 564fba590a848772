"""Solves with the ABFT Cholesky factor (abft_potrs) and the mixed-precision
solve with iterative refinement (abft_posv_ir): against the CPU oracle's
substitution, and the normwise backward error re-checked on the CPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def eta_cpu(A, X, B):
    """max_r ||B_r - A X_r||_inf / (||A||_inf ||X_r||_inf + ||B_r||_inf), FP64 on the CPU."""
    R = B - A @ X
    an = np.abs(A).sum(axis=1).max()
    return float(np.max(np.abs(R).max(axis=0) / (an * np.abs(X).max(axis=0) + np.abs(B).max(axis=0))))


@pytest.mark.parametrize("n,nrhs,nb", [(1, 1, 32), (100, 3, 32), (257, 16, 64), (700, 20, 128),
                                       (1024, 16, 256)])
def test_potrs_f64_vs_oracle(n, nrhs, nb):
    A = W.spd_mmt(n, seed=n)
    Lo, _ = oracle.potf2(A)
    Lo = np.tril(Lo)
    B = W.rhs(n, nrhs, seed=n + 1)
    Xo = oracle.potrs(Lo, B)
    Lt = torch.from_numpy(Lo).to(DEV)
    Bt = torch.from_numpy(B).to(DEV)
    abft.potrs(Lt, Bt, nb, abft.F64)
    X = Bt.cpu().numpy()
    assert np.abs(X - Xo).max() <= 1e-12 * max(1.0, np.abs(Xo).max())


def test_potrs_f32():
    n, nrhs = 777, 5
    A = W.spd_mmt(n, seed=3)
    Lo = np.linalg.cholesky(A)
    B = W.rhs(n, nrhs, seed=4)
    Bt = torch.from_numpy(B).to(DEV)
    abft.potrs(torch.from_numpy(Lo).to(DEV), Bt, 128, abft.F32)
    Xo = oracle.potrs(Lo, B)
    assert np.abs(Bt.cpu().numpy() - Xo).max() <= 1e-4 * np.abs(Xo).max()


@pytest.mark.parametrize("dtype", [abft.F64, abft.MIXED_BF16, abft.MIXED_F16])
@pytest.mark.parametrize("n,nb", [(512, 128), (2048, 256)])
def test_posv_ir_kappa_1e2(dtype, n, nb):
    A = W.spd_kappa(n, 1e2, seed=1002)
    B = W.rhs(n, 16, seed=1003)
    rc, X, L, rep = abft.posv_ir(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), nb,
                                 dtype, abft.FULL, tol=1e-12, maxit=60)
    torch.cuda.synchronize()
    assert rc == 0 and rep["detected"] == 0
    assert rep["backward_err"] <= 1e-12
    Xh = X.cpu().numpy()
    assert eta_cpu(A, Xh, B) <= 2e-12
    Xo = oracle.potrs(np.linalg.cholesky(A), B)
    assert np.abs(Xh - Xo).max() <= 1e-9 * np.abs(Xo).max()
    if dtype == abft.F64:
        assert rep["ir_iters"] <= 2


def test_posv_ir_with_fault():
    n, nb = 1024, 128
    A = W.spd_kappa(n, 1e2, seed=7)
    B = W.rhs(n, 16, seed=8)
    faults = [(2, abft.F_MEMORY, 900, 500, 1e3)]
    rc, X, L, rep = abft.posv_ir(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), nb,
                                 abft.MIXED_F16, abft.FULL, tol=1e-12, maxit=60, faults=faults)
    assert rc == 0 and [e[:4] for e in rep["loc"]] == [(2, 0, 900, 500)]
    assert eta_cpu(A, X.cpu().numpy(), B) <= 2e-12


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16])
def test_posv_ir_kappa_1e6_reports_outcome(dtype):
    """At kappa = 1e6 plain refinement from a 16-bit factor may not reach 1e-12;
    the call must then say so (backward_err > tol after maxit steps), never
    claim convergence it did not reach."""
    n = 1024
    A = W.spd_kappa(n, 1e6, seed=11)
    B = W.rhs(n, 16, seed=12)
    rc, X, L, rep = abft.posv_ir(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), 128,
                                 dtype, abft.FULL, tol=1e-12, maxit=30)
    if rc != 0:
        assert rc > 0 or rc == abft.ERR_UNCORRECTABLE
        return
    e = eta_cpu(A, X.cpu().numpy(), B)
    if rep["backward_err"] <= 1e-12:
        assert e <= 2e-12
    else:
        assert rep["ir_iters"] == 30
