"""GMRES-based iterative refinement (abft_posv_gmres_ir): the solution checked
against the CPU oracle's FP64 Cholesky solve and the normwise backward error
recomputed on the CPU; the scaling, shift and retry behaviour checked against
what the entry point documents."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def eta_cpu(A, X, B):
    R = B - A @ X
    an = np.abs(A).sum(axis=1).max()
    return float(np.max(np.abs(R).max(axis=0) / (an * np.abs(X).max(axis=0) + np.abs(B).max(axis=0))))


def solve(A, B, nb=256, dtype=abft.MIXED_BF16, **kw):
    return abft.posv_gmres_ir(torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV), nb, dtype,
                              abft.FULL, **kw)


def oracle_solution(A, B):
    Lo, info = oracle.potf2(A)
    assert info == 0
    return oracle.potrs(np.tril(Lo), B)


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16, abft.F64])
def test_kappa_1e2_matches_oracle(dtype):
    n = 1024
    A = W.spd_kappa(n, 1e2, seed=1002)
    B = W.rhs(n, 16, seed=1003)
    rc, X, L, rep = solve(A, B, 128, dtype, tol=1e-12, maxit=10, m=30)
    assert rc == 0 and rep["detected"] == 0 and rep["attempts"] == 1 and rep["shift"] == 0.0
    Xh = X.cpu().numpy()
    assert rep["backward_err"] <= 1e-12 and eta_cpu(A, Xh, B) <= 2e-12
    Xo = oracle_solution(A, B)
    assert np.abs(Xh - Xo).max() <= 1e-10 * np.abs(Xo).max()


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16])
def test_kappa_1e6_converges_with_shift(dtype):
    """Plain refinement cannot use a 16-bit factor here (the factorization of
    the unshifted matrix breaks down or refinement diverges); GMRES-IR with the
    automatic shift reaches the FP64-level backward error."""
    n = 2048
    A = W.spd_kappa(n, 1e6, seed=1002)
    B = W.rhs(n, 16, seed=1003)
    rc, X, L, rep = solve(A, B, 256, dtype, tol=1e-12, maxit=20, m=60)
    assert rc == 0
    Xh = X.cpu().numpy()
    assert rep["backward_err"] <= 1e-12
    assert eta_cpu(A, Xh, B) <= 2e-12
    assert rep["gmres_iters"] >= rep["ir_iters"] >= 1
    # the shift actually used is u_f * 4^(attempts - 2) after a failed first try
    uf = 2.0 ** -8 if dtype == abft.MIXED_BF16 else 2.0 ** -11
    if rep["attempts"] > 1:
        assert rep["shift"] == uf * 4.0 ** (rep["attempts"] - 2)
    Xo = oracle_solution(A, B)
    # forward error bound: kappa * eta (with slack)
    assert np.abs(Xh - Xo).max() <= 1e6 * 1e-11 * np.abs(Xo).max()


def test_kappa_1e10_reports_outcome():
    """At kappa = 1e10 a 16-bit factor is beyond what GMRES-IR with an FP64
    working precision can fix; the call must report the backward error it
    reached, never claim convergence it did not reach."""
    n = 1024
    A = W.spd_kappa(n, 1e10, seed=1002)
    B = W.rhs(n, 16, seed=1003)
    rc, X, L, rep = solve(A, B, 128, abft.MIXED_F16, tol=1e-12, maxit=4, m=40)
    assert rc == 0 and rep["attempts"] >= 2
    e = eta_cpu(A, X.cpu().numpy(), B)
    assert abs(e - rep["backward_err"]) <= 1e-3 * e + 1e-15
    if rep["backward_err"] > 1e-12:
        assert rep["ir_iters"] == 4


def test_ragged_many_rhs_and_fixed_shift():
    n, nrhs = 1000, 20          # n not a multiple of nb; two blocks of right-hand sides
    A = W.spd_kappa(n, 1e4, seed=5)
    B = W.rhs(n, nrhs, seed=6)
    rc, X, L, rep = solve(A, B, 128, abft.MIXED_F16, tol=1e-12, maxit=10, m=40, shift=1e-3)
    assert rc == 0 and rep["attempts"] == 1 and rep["shift"] == 1e-3
    assert eta_cpu(A, X.cpu().numpy(), B) <= 2e-12


def test_scaling_is_exact_and_factor_is_of_scaled_matrix():
    """A badly scaled SPD matrix D A0 D: the factor is of S (D A0 D) S + delta I
    with S a power-of-two diagonal, whose diagonal lies in [1/4, 2)."""
    n = 512
    A0 = W.spd_mmt(n, seed=9)
    d = 2.0 ** np.random.default_rng(10).integers(-20, 20, n)
    A = (A0 * d[:, None]) * d[None, :]
    B = W.rhs(n, 4, seed=11)
    rc, X, L, rep = solve(A, B, 128, abft.F64, tol=1e-12, maxit=5, m=20, shift=0.0)
    assert rc == 0 and rep["backward_err"] <= 1e-12
    e = np.frexp(np.diag(A))[1]
    s = 2.0 ** (-np.trunc(e / 2))
    As = (A * s[:, None]) * s[None, :]
    assert np.all(np.diag(As) >= 0.25) and np.all(np.diag(As) < 2.0)
    Lh = np.tril(L.cpu().numpy())
    assert np.abs(Lh @ Lh.T - As).max() <= 1e-13 * np.abs(As).max()
    assert eta_cpu(A, X.cpu().numpy(), B) <= 2e-12


def test_fault_in_factorization_is_corrected():
    n, nb = 1024, 128
    A = W.spd_kappa(n, 1e4, seed=7)
    B = W.rhs(n, 16, seed=8)
    faults = [(2, abft.F_MEMORY, 900, 500, 1e3)]
    rc, X, L, rep = solve(A, B, nb, abft.MIXED_BF16, tol=1e-12, maxit=10, m=40, shift=2.0 ** -8,
                          faults=faults)
    assert rc == 0 and [e[:4] for e in rep["loc"]] == [(2, 0, 900, 500)]
    assert eta_cpu(A, X.cpu().numpy(), B) <= 2e-12


def test_argument_errors():
    A = torch.eye(64, dtype=torch.float64, device=DEV)
    B = torch.ones(64, 2, dtype=torch.float64, device=DEV)
    with pytest.raises(abft.AbftError):
        abft.posv_gmres_ir(A, B, 32, abft.MIXED_BF16, m=0)
    with pytest.raises(abft.AbftError):
        abft.posv_gmres_ir(A, B, 32, abft.MIXED_BF16, m=65)
    with pytest.raises(abft.AbftError):
        abft.posv_gmres_ir(A, B, 32, abft.MIXED_BF16, inner_tol=-1.0)
