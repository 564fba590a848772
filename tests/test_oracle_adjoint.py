"""Pins of the oracle's Cholesky adjoint (Murray 2016, symbolic form) and of
the GP gradient closed form used for the differentiable Cholesky.

Independent facts: the 1x1 case a = l^2 (abar = lbar / (2 l)); logdet A =
2 sum log l_ii so Lbar = diag(2 / l_ii) must give Abar = A^{-1}; central finite
differences of a scalar function of chol(A) along symmetric directions; and
the GP closed form dK = (K^{-1} - alpha alpha^T)/2 against finite differences.
"""
import numpy as np
import scipy.linalg as sl

import oracle
from paper_2301_03166_b300 import workloads as W


def test_adjoint_1x1():
    l, lbar = 3.0, 0.7
    Abar = oracle.potrf_backward(np.array([[l]]), np.array([[lbar]]))
    assert np.isclose(Abar[0, 0], lbar / (2 * l), rtol=1e-15)


def test_adjoint_logdet_identity():
    A = W.spd_mmt(50, 2)
    L = sl.cholesky(A, lower=True)
    Abar = oracle.potrf_backward(L, np.diag(2.0 / np.diag(L)))
    np.testing.assert_allclose(Abar, np.linalg.inv(A), rtol=1e-11, atol=1e-13)


def test_adjoint_finite_differences():
    n = 12
    A = W.spd_mmt(n, 3)
    Wt = np.tril(W.rng(4).standard_normal((n, n)))
    f = lambda M: float(np.sum(Wt * sl.cholesky(M, lower=True)))
    Abar = oracle.potrf_backward(sl.cholesky(A, lower=True), Wt)
    r = W.rng(5)
    for _ in range(6):
        E = r.standard_normal((n, n)); E = E + E.T
        h = 1e-6
        fd = (f(A + h * E) - f(A - h * E)) / (2 * h)
        assert abs(np.sum(Abar * E) - fd) <= 1e-6 * max(1.0, abs(fd))


def test_gp_closed_form_fd():
    X, y = W.gp_inputs(40, 8, 6)
    K = W.gp_kernel(X)
    loss, G = oracle.gp_loss_grad(K, y)
    r = W.rng(7)
    for _ in range(4):
        E = r.standard_normal(K.shape); E = E + E.T
        h = 1e-6
        fd = (oracle.gp_loss_grad(K + h * E, y)[0] - oracle.gp_loss_grad(K - h * E, y)[0]) / (2 * h)
        assert abs(np.sum(G * E) - fd) <= 1e-6 * max(1.0, abs(fd))


def test_gp_chain_through_cholesky():
    """loss = y^T K^{-1} y / 2 + sum log l_ii via L: Lbar from the solve and the
    logdet, then the adjoint, reproduces the closed form."""
    X, y = W.gp_inputs(30, 8, 8)
    K = W.gp_kernel(X)
    L = sl.cholesky(K, lower=True)
    alpha = sl.cho_solve((L, True), y)
    # d(y^T K^{-1} y / 2)/dK = -alpha alpha^T / 2 ; via L: Lbar = tril((Kbar + Kbar^T) L)
    Kbar_solve = -0.5 * np.outer(alpha, alpha)
    Lbar = np.tril((Kbar_solve + Kbar_solve.T) @ L) + np.diag(1.0 / np.diag(L))
    G = oracle.potrf_backward(L, Lbar)
    _, Gc = oracle.gp_loss_grad(K, y)
    np.testing.assert_allclose(G, Gc, rtol=1e-9, atol=1e-11)
