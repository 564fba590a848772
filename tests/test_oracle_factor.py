"""Pins of the oracle's plain factorizations against what the mathematics fixes.

Sec. 2.1 (PD / PU / TMU skeleton) for Cholesky, LU and QR.  Each check is
independent of the oracle's own code: hand-worked golden fixtures, exact
integer constructions, closed forms, determinant identities, LAPACK as a
library special case, and residual bounds.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_2301_03166_b300 import workloads as W
from tests.golden.read import load

U = 2.0 ** -53


# ------------------------------------------------------------- Cholesky
def test_potf2_golden_3x3():
    g = load("chol_3x3.txt")
    L, info = oracle.potf2(g["A"])
    assert info == 0
    np.testing.assert_allclose(np.tril(L), g["L"], rtol=0, atol=4e-16)
    # strict upper triangle untouched
    assert np.array_equal(np.triu(L, 1), np.triu(g["A"], 1))


def test_potf2_closed_forms():
    L, info = oracle.potf2(np.array([[9.0]]))
    assert info == 0 and L[0, 0] == 3.0
    a, b, c = 5.0, 2.0, 7.0
    L, info = oracle.potf2(np.array([[a, b], [b, c]]))
    l11 = np.sqrt(a); l21 = b / l11; l22 = np.sqrt(c - l21 * l21)
    assert np.allclose(np.tril(L), [[l11, 0], [l21, l22]], rtol=1e-15)


def test_potf2_determinant_identity_4x4():
    """Brute force on 4x4: l_jj^2 = D_j / D_{j-1} (leading principal minors)
    and l_ij = det(A[[0..j-1, i], [0..j]]) / sqrt(D_{j-1} D_j)."""
    r = W.rng(5)
    for _ in range(20):
        M = r.standard_normal((4, 4))
        A = M @ M.T + 0.5 * np.eye(4)
        L, info = oracle.potf2(A)
        L = np.tril(L)
        D = [1.0] + [np.linalg.det(A[:j, :j]) for j in range(1, 5)]
        for j in range(4):
            assert np.isclose(L[j, j] ** 2, D[j + 1] / D[j], rtol=1e-12)
            for i in range(j + 1, 4):
                rows = list(range(j)) + [i]
                num = np.linalg.det(A[np.ix_(rows, list(range(j + 1)))])
                assert np.isclose(L[i, j], num / np.sqrt(D[j] * D[j + 1]), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n,nb", [(1, 1), (7, 3), (33, 8), (64, 16), (64, 64), (256, 128)])
def test_potrf_integer_exact(n, nb):
    """A = L0 L0^T with integer L0: every intermediate is an integer, so the
    blocked and the unblocked factorizations return L0 bit-exactly."""
    L0 = W.integer_l0(n, seed=n)
    A = L0 @ L0.T
    L, info = oracle.potf2(A)
    assert info == 0 and np.array_equal(np.tril(L), L0)
    for mode in (oracle.NONE, oracle.SINGLE, oracle.FULL):
        L, info, rep = oracle.potrf(A, nb, mode)
        assert info == 0 and np.array_equal(np.tril(L), L0)
        assert rep["detected"] == 0


@pytest.mark.parametrize("n,nb", [(100, 32), (129, 64), (256, 64)])
def test_potrf_residual_and_lapack(n, nb):
    A = W.spd_mmt(n, seed=n)
    L, info, rep = oracle.potrf(A, nb, oracle.FULL)
    L = np.tril(L)
    assert info == 0
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) <= 10 * n * U
    Lref = sl.cholesky(A, lower=True)
    assert np.abs(L - Lref).max() <= 1e-13
    Lu, _ = oracle.potf2(A)
    assert np.abs(np.tril(Lu) - L).max() <= 1e-13


def test_potrf_not_spd_info():
    A = W.spd_mmt(40, 3)
    A[17, 17] = -5.0
    _, info_u = oracle.potf2(A)
    _, info_b, _ = oracle.potrf(A, 8, oracle.FULL)
    assert info_u == 18 and info_b == 18


def test_potrf_empty_and_args():
    L, info, rep = oracle.potrf(np.zeros((0, 0)), 8)
    assert info == 0


# ------------------------------------------------------------------- LU
def test_getf2_golden_3x3():
    g = load("lu_3x3.txt")
    LU, ipiv, info = oracle.getf2(g["A"])
    assert info == 0
    assert list(ipiv) == [int(x) for x in g["IPIV"][0]]
    np.testing.assert_allclose(LU, g["LU"], rtol=0, atol=8 * U)


@pytest.mark.parametrize("n,nb", [(5, 2), (40, 8), (64, 16), (96, 32)])
def test_getrf_exact_plu(n, nb):
    """A = P0 L0 U0 with |l| < 1 and dyadic entries: partial pivoting must pick
    P0 and return L0, U0 bit-exactly (every intermediate is exact)."""
    A, P0, L0, U0 = W.lu_exact(n, seed=n)
    for fn in ("unblocked", "blocked"):
        if fn == "unblocked":
            LU, ipiv, info = oracle.getf2(A)
        else:
            LU, ipiv, info, rep = oracle.getrf(A, nb, oracle.FULL)
            assert rep["detected"] == 0
        P, L, Um = oracle.unpack_lu(LU, ipiv)
        assert info == 0
        assert np.array_equal(P, P0.T)
        assert np.array_equal(L, L0) and np.array_equal(Um, U0)


@pytest.mark.parametrize("n,nb", [(100, 32), (130, 64)])
def test_getrf_residual_and_lapack(n, nb):
    A = W.uniform(n, seed=n)
    LU, ipiv, info, rep = oracle.getrf(A, nb, oracle.FULL)
    P, L, Um = oracle.unpack_lu(LU, ipiv)
    growth = np.abs(Um).max() / np.abs(A).max()
    assert np.linalg.norm(P @ A - L @ Um) / np.linalg.norm(A) <= 10 * n * U * growth
    lu_ref, piv_ref = sl.lu_factor(A)
    assert np.array_equal(ipiv, piv_ref)
    assert np.abs(LU - lu_ref).max() <= 1e-12
    LU2, ipiv2, _ = oracle.getf2(A)
    assert np.array_equal(ipiv2, ipiv) and np.abs(LU2 - LU).max() <= 1e-12


def test_getf2_pivot_first_max_tie():
    A = np.array([[1.0, 0.0], [-1.0, 1.0]])  # |1| == |-1|: the first index wins
    LU, ipiv, info = oracle.getf2(A)
    assert list(ipiv) == [0, 1]


def test_getf2_singular_info():
    A = np.array([[0.0, 1.0], [0.0, 2.0]])
    _, _, info = oracle.getf2(A)
    assert info == 1


# ------------------------------------------------------------------- QR
def test_geqr2_golden_2x2():
    g = load("qr_2x2.txt")
    QR, tau = oracle.geqr2(g["A"])
    np.testing.assert_allclose(QR, g["QR"], rtol=0, atol=4e-16)
    np.testing.assert_allclose(tau, g["TAU"][0], rtol=0, atol=4e-16)


def test_geqr2_sign_of_zero_alpha():
    # alpha = 0: sign(0) = + so beta = -||x||
    QR, tau = oracle.geqr2(np.array([[0.0, 1.0], [2.0, 3.0]]))
    assert QR[0, 0] == -2.0 and tau[0] == 1.0


def test_geqrf_orthogonal_columns():
    """Orthogonal columns give |R| = diag(||a_j||)."""
    Q0, _ = np.linalg.qr(W.rng(3).standard_normal((48, 48)))
    d = np.arange(1, 49, dtype=float)
    A = Q0 * d
    QR, tau, info, rep = oracle.geqrf(A, 16, oracle.FULL)
    R = np.triu(QR)
    np.testing.assert_allclose(np.abs(np.diag(R)), d, rtol=1e-13)
    assert np.abs(R - np.diag(np.diag(R))).max() <= 1e-12 * d.max()


@pytest.mark.parametrize("n,nb", [(100, 32), (97, 16)])
def test_geqrf_residual_orthogonality_lapack(n, nb):
    A = W.uniform(n, seed=n)
    QR, tau, info, rep = oracle.geqrf(A, nb, oracle.FULL)
    assert rep["detected"] == 0
    Q = oracle.form_q(QR, tau)
    R = np.triu(QR)
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 10 * n * U
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 10 * n * U
    np.testing.assert_allclose(R.T @ R, A.T @ A, atol=1e-12 * np.linalg.norm(A) ** 2)
    (h, tau_ref), _ = sl.qr(A, mode="raw")
    np.testing.assert_allclose(tau, tau_ref, atol=1e-12)
    np.testing.assert_allclose(QR, h, atol=1e-12)  # h comes back C-ordered as A
    QR2, tau2 = oracle.geqr2(A)
    np.testing.assert_allclose(QR2, QR, atol=1e-12)


# ---------------------------------------------------------------- solves
def test_potrs_solves():
    A = W.spd_mmt(70, 4)
    B = W.rhs(70, 5)
    L, _ = oracle.potf2(A)
    X = oracle.potrs(np.tril(L), B)
    np.testing.assert_allclose(X, sl.cho_solve((np.tril(L), True), B), rtol=1e-12, atol=1e-13)
    assert np.abs(A @ X - B).max() <= 1e-12
