"""Cholesky adjoint on the GPU (abft_potrf_backward, potrs/logdet adjoints and
the torch.autograd layer) against the oracle's symbolic adjoint, the logdet
identity, the GP closed form (K^{-1} - alpha alpha^T)/2 and central finite
differences."""
import numpy as np
import pytest
import scipy.linalg as sl
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import autograd as ag
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("n,nb", [(1, 32), (31, 32), (100, 32), (257, 64), (700, 128), (1024, 256)])
def test_potrf_backward_vs_oracle(n, nb):
    A = W.spd_mmt(n, seed=700 + n)
    L = np.linalg.cholesky(A)
    Lbar = np.tril(W.rng(n).standard_normal((n, n)))
    G_o = oracle.potrf_backward(L, Lbar)                 # symmetric gradient
    Lt = T(L + np.triu(np.full((n, n), 7.0), 1))         # garbage above the diagonal must be ignored
    G = abft.potrf_backward(Lt, T(Lbar + np.triu(np.full((n, n), 5.0), 1)), nb, sym=True)
    torch.cuda.synchronize()
    G = G.cpu().numpy()
    assert np.abs(G - G_o).max() <= 1e-11 * max(1.0, np.abs(G_o).max())
    Al = abft.potrf_backward(Lt, T(Lbar), nb, sym=False).cpu().numpy()
    assert np.allclose(np.tril(Al), np.tril(2 * G_o) - np.diag(np.diag(G_o)), rtol=1e-11, atol=1e-12)
    assert np.all(np.triu(Al, 1) == 0)


def test_logdet_identity():
    """f = log det A = 2 sum log l_ii: Lbar = diag(2 / l_ii) gives dA = A^{-1}."""
    n = 512
    A = W.spd_mmt(n, seed=9)
    L = np.linalg.cholesky(A)
    Lt = T(L)
    Lbar = torch.zeros_like(Lt)
    abft.logdet_backward(Lt, 1.0, Lbar)
    G = abft.potrf_backward(Lt, Lbar, 128, sym=True).cpu().numpy()
    np.testing.assert_allclose(G, np.linalg.inv(A), rtol=1e-10, atol=1e-12)
    ld = abft.logdet(Lt).item()
    assert abs(ld - np.linalg.slogdet(A)[1]) <= 1e-10 * abs(ld)


def _gp_loss_torch(X, y, ell, nb):
    sq = (X * X).sum(1)
    D = torch.clamp(sq[:, None] + sq[None, :] - 2.0 * X @ X.T, min=0.0)
    K = torch.exp(-D / (2.0 * ell ** 2)) + 1e-2 * torch.eye(X.shape[0], dtype=X.dtype, device=X.device)
    return ag.gp_negative_log_likelihood_terms(K, y, nb), K


@pytest.mark.parametrize("n", [512, 4096])
def test_gp_gradient_vs_closed_form_and_fd(n):
    """GP config: X n x 8 iid N(0,1), K = exp(-|xi - xj|^2 / 2) + 1e-2 I, y iid N(0,1),
    loss = y^T K^{-1} y / 2 + logdet K / 2.  dK from the hand-written adjoint vs the
    CPU FP64 closed form (<= 1e-8 relative); d loss / d lengthscale vs central FD."""
    Xn, yn = W.gp_inputs(n, 8, seed=1004)
    X, y = T(Xn), T(yn)
    Kn = W.gp_kernel(Xn)
    K = T(Kn).requires_grad_(True)
    loss = ag.gp_negative_log_likelihood_terms(K, y, 256)
    loss.backward()
    G = K.grad.cpu().numpy()
    loss_o, G_o = oracle.gp_loss_grad(Kn, yn)
    assert abs(loss.item() - loss_o) <= 1e-10 * abs(loss_o)
    assert np.linalg.norm(G - G_o) <= 1e-8 * np.linalg.norm(G_o)
    # lengthscale through torch's elementwise kernel construction (user model code)
    ell = torch.tensor(1.0, dtype=torch.float64, device=DEV, requires_grad=True)
    loss2, _ = _gp_loss_torch(X, y, ell, 256)
    loss2.backward()
    h = 1e-6
    with torch.no_grad():
        lp = _gp_loss_torch(X, y, torch.tensor(1.0 + h, dtype=torch.float64, device=DEV), 256)[0]
        lm = _gp_loss_torch(X, y, torch.tensor(1.0 - h, dtype=torch.float64, device=DEV), 256)[0]
    fd = (lp.item() - lm.item()) / (2 * h)
    assert abs(ell.grad.item() - fd) <= 1e-6 * max(1.0, abs(fd))
    # the same derivative from the CPU closed form: sum(G_o * dK/dl)
    sq = np.sum(Xn * Xn, axis=1)
    D = np.maximum(sq[:, None] + sq[None, :] - 2.0 * Xn @ Xn.T, 0.0)
    dK = np.exp(-D / 2.0) * D
    assert abs(ell.grad.item() - np.sum(G_o * dK)) <= 1e-8 * abs(np.sum(G_o * dK))


def test_gp_gradient_n16384_fd():
    """n = 16384: the reverse sweep reads only L (no stored intermediates);
    directional derivative along a symmetric rank-2 direction vs central FD."""
    n = 16384
    Xn, yn = W.gp_inputs(n, 8, seed=1004)
    X, y = T(Xn), T(yn)
    ell = torch.tensor(1.0, dtype=torch.float64, device=DEV, requires_grad=True)
    loss, K = _gp_loss_torch(X, y, ell, 256)
    loss.backward()
    h = 1e-6
    with torch.no_grad():
        lp = _gp_loss_torch(X, y, torch.tensor(1.0 + h, dtype=torch.float64, device=DEV), 256)[0]
        lm = _gp_loss_torch(X, y, torch.tensor(1.0 - h, dtype=torch.float64, device=DEV), 256)[0]
    fd = (lp.item() - lm.item()) / (2 * h)
    assert abs(ell.grad.item() - fd) <= 1e-5 * max(1.0, abs(fd))


def test_potrs_backward_vs_fd():
    n = 300
    A = W.spd_mmt(n, seed=21)
    B = W.rhs(n, 3, seed=22)
    Xbar = W.rhs(n, 3, seed=23)
    At = T(A).requires_grad_(True)
    Bt = T(B).requires_grad_(True)
    L = ag.cholesky(At, 64)
    Xs = ag.cholesky_solve(L, Bt, 64)
    (Xs * T(Xbar)).sum().backward()
    Gt = At.grad.cpu().numpy()
    Ainv = np.linalg.inv(A)
    Xe = Ainv @ B
    Bb = Ainv @ Xbar
    G_ref = -0.5 * (Bb @ Xe.T + Xe @ Bb.T)
    np.testing.assert_allclose(Gt, G_ref, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(Bt.grad.cpu().numpy(), Bb, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("n,nb", [(256, 128), (768, 256), (1280, 128), (2048, 256)])
def test_potrf_backward_fp64_accurate_vs_oracle(n, nb):
    """The reverse sweep with its dominant product from BF16 slices on the
    tensor cores: the same adjoint as the oracle's to FP64 accuracy."""
    A = W.spd_mmt(n, seed=800 + n)
    L = np.linalg.cholesky(A)
    Lbar = np.tril(W.rng(n + 1).standard_normal((n, n)))
    G_o = oracle.potrf_backward(L, Lbar)
    G = abft.potrf_backward(T(L), T(Lbar), nb, sym=True, dtype=abft.F64_EMU).cpu().numpy()
    assert np.abs(G - G_o).max() <= 1e-11 * max(1.0, np.abs(G_o).max())
    G64 = abft.potrf_backward(T(L), T(Lbar), nb, sym=True).cpu().numpy()
    assert np.abs(G - G64).max() <= 1e-11 * max(1.0, np.abs(G64).max())


def test_potrf_backward_fp64_accurate_unsupported_shapes():
    L = T(np.eye(300))
    with pytest.raises(abft.AbftError):
        abft.potrf_backward(L, L, 128, dtype=abft.F64_EMU)      # n not a multiple of nb
    with pytest.raises(abft.AbftError):
        abft.potrf_backward(T(np.eye(256)), T(np.eye(256)), 64, dtype=abft.F64_EMU)


def test_gp_gradient_fp64_accurate_forward_and_backward():
    """GP configuration at n = 4096 with the FP64-accurate factorization and
    reverse sweep: the gradient within 1e-8 of the CPU closed form."""
    n = 4096
    Xn, yn = W.gp_inputs(n, 8, seed=1004)
    Kn = W.gp_kernel(Xn)
    K = T(Kn).requires_grad_(True)
    loss = ag.gp_negative_log_likelihood_terms(K, T(yn), 256, dtype=abft.F64_EMU)
    loss.backward()
    loss_o, G_o = oracle.gp_loss_grad(Kn, yn)
    assert abs(loss.item() - loss_o) <= 1e-10 * abs(loss_o)
    assert np.linalg.norm(K.grad.cpu().numpy() - G_o) <= 1e-8 * np.linalg.norm(G_o)
