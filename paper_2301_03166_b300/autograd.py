"""torch.autograd Functions over the library's Cholesky, solve and logdet.

Forward and backward both run in libabft kernels (potrf / potrs / logdet and
their adjoints); torch only allocates the tensors.  The Cholesky adjoint is
the blocked reverse sweep, which needs L alone (no stored intermediates), so
memory stays at the size of the factor for any n.
"""
import torch

from . import abft


class Cholesky(torch.autograd.Function):
    """L = chol(A) (lower, zero above the diagonal) with ABFT checksums."""

    @staticmethod
    def forward(ctx, A, nb=256, mode=abft.FULL, dtype=abft.F64):
        L = A.detach().contiguous().clone()
        rc, rep = abft.potrf(L, nb, mode, dtype=dtype)
        if rc != 0:
            raise abft.AbftError(rc, abft.strerror(rc))
        abft.tril_(L)
        ctx.save_for_backward(L)
        ctx.nb = nb
        # the FP64-accurate forward keeps its arithmetic in the reverse sweep
        # where the sweep supports it (nb 128 or 256, n a multiple of nb)
        n = L.shape[0]
        ctx.bdtype = abft.F64_EMU if (dtype == abft.F64_EMU and nb in (128, 256) and n % nb == 0) \
            else abft.F64
        return L

    @staticmethod
    def backward(ctx, Lbar):
        (L,) = ctx.saved_tensors
        G = abft.potrf_backward(L, Lbar.contiguous(), ctx.nb, sym=True, dtype=ctx.bdtype)
        return G, None, None, None


class CholeskySolve(torch.autograd.Function):
    """X = A^{-1} B from the factor L of A."""

    @staticmethod
    def forward(ctx, L, B, nb=256):
        X = B.detach().contiguous().clone()
        abft.potrs(L.detach(), X, nb, abft.F64)
        ctx.save_for_backward(L, X)
        ctx.nb = nb
        return X

    @staticmethod
    def backward(ctx, Xbar):
        L, X = ctx.saved_tensors
        Lbar = torch.zeros_like(L)
        Bbar = abft.potrs_backward(L, X, Xbar.contiguous(), Lbar, ctx.nb)
        return Lbar, Bbar, None


class LogdetFromCholesky(torch.autograd.Function):
    """log det A = 2 sum log L_ii from the factor L of A."""

    @staticmethod
    def forward(ctx, L):
        out = abft.logdet(L.detach())
        ctx.save_for_backward(L)
        return out

    @staticmethod
    def backward(ctx, gbar):
        (L,) = ctx.saved_tensors
        Lbar = torch.zeros_like(L)
        abft.logdet_backward(L, float(gbar), Lbar)
        return Lbar


def cholesky(A, nb=256, mode=abft.FULL, dtype=abft.F64):
    """dtype ABFT_F64 (FP64 update) or ABFT_F64_EMU (FP64-accurate update on
    the BF16 tensor cores, nb 128 or 256)."""
    return Cholesky.apply(A, nb, mode, dtype)


def cholesky_solve(L, B, nb=256):
    return CholeskySolve.apply(L, B, nb)


def logdet_from_cholesky(L):
    return LogdetFromCholesky.apply(L)


def gp_negative_log_likelihood_terms(K, y, nb=256, dtype=abft.F64):
    """loss = y^T K^{-1} y / 2 + logdet(K) / 2 through the ABFT Cholesky."""
    L = cholesky(K, nb, dtype=dtype)
    alpha = cholesky_solve(L, y.reshape(-1, 1), nb)
    return 0.5 * (y.reshape(-1, 1) * alpha).sum() + 0.5 * logdet_from_cholesky(L)
