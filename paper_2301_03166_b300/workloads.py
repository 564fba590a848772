"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds input construction only -- none of the factorization or
checksum arithmetic -- so that both the CUDA path and the CPU oracle can be fed
the same matrices.  The paper measures on synthetic square dense matrices
(n = 30720, and 5120 and up for the size sweep) with no named distribution;
the recipes below are the ones the workload definitions fix:

* Cholesky:   A = M M^T / n + I,  M iid N(0, 1)
* LU and QR:  A iid U[-1, 1]
* mixed:      A = Q diag(sigma) Q^T, Q from the QR of an N(0,1) matrix with
              the sign fix Q diag(sign(diag R)), sigma geometric with
              condition number kappa; 16 right-hand sides iid N(0, 1)
* GP:         X n x 8 iid N(0,1), K = exp(-|xi - xj|^2 / (2 l^2)) + 1e-2 I, y iid N(0,1)
* batched:    n_i uniform in [32, 512], A_i = M_i M_i^T / n_i + I, per-matrix seeds
* exact:      integer L0 (entries in {-3..3}, diagonal in {1, 2, 4}) and
              A = P0 L0 U0 with dyadic L0 in {0, +-1/2, +-1/4} and integer U0
              with a power-of-two diagonal, whose factorizations are exact.
Generators use numpy PCG64 with the seed given; torch variants build the
large matrices on the GPU (input construction only).
"""
import numpy as np

F_MEMORY, F_COMPUTE, F_ROW1D, F_COL1D, F_PANEL = 0, 1, 2, 3, 4


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def spd_mmt(n, seed=1000):
    """A = M M^T / n + I with M iid N(0,1), float64."""
    M = rng(seed).standard_normal((n, n))
    A = M @ M.T / n
    A = 0.5 * (A + A.T)
    A[np.diag_indices(n)] += 1.0
    return A


def spd_mmt_torch(n, seed=1000, device="cuda"):
    """Large-n variant of spd_mmt built with torch on `device` (float64 result;
    the product is formed in float32 and its lower triangle mirrored, so the
    matrix is exactly symmetric and SPD with eigenvalues >= 1 - O(1e-5))."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    M = torch.randn(n, n, generator=g, device=device, dtype=torch.float32)
    A = (M @ M.T).div_(n).double()
    del M
    A = torch.tril(A) + torch.tril(A, -1).T
    A.diagonal().add_(1.0)
    return A


def uniform(n, seed=1001):
    """A iid U[-1, 1], float64 (LU and QR inputs)."""
    return rng(seed).uniform(-1.0, 1.0, (n, n))


def uniform_torch(n, seed=1001, device="cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.rand(n, n, generator=g, device=device, dtype=torch.float64).mul_(2.0).sub_(1.0)


def integer_l0(n, seed=7):
    """Lower-triangular integer L0: off-diagonal in {-3..3}, diagonal in {1,2,4}.
    A = L0 L0^T is exact in float64 for the n used in tests (n <= 64)."""
    r = rng(seed)
    L = np.tril(r.integers(-3, 4, (n, n)).astype(np.float64), -1)
    L[np.diag_indices(n)] = r.choice([1.0, 2.0, 4.0], n)
    return L


def lu_exact(n, seed=11):
    """(A, P0, L0, U0) with A = P0 L0 U0; L0 unit lower with off-diagonal
    entries in {0, +-1/2, +-1/4} (so |l| < 1 and partial pivoting picks P0),
    U0 upper with integer entries in {-3..3} and diagonal in {+-1, +-2, +-4}."""
    r = rng(seed)
    L = np.tril(r.choice([0.0, 0.5, -0.5, 0.25, -0.25], (n, n)), -1) + np.eye(n)
    U = np.triu(r.integers(-3, 4, (n, n)).astype(np.float64), 1)
    U[np.diag_indices(n)] = r.choice([1.0, -1.0, 2.0, -2.0, 4.0, -4.0], n)
    perm = r.permutation(n)
    P = np.eye(n)[perm]
    return P @ (L @ U), P, L, U


def spd_kappa(n, kappa, seed=1002):
    """A = Q diag(sigma) Q^T, sigma_i = kappa^(-i/(n-1)), Q orthogonal from the
    QR of an N(0,1) matrix with the sign fix (float64, numpy)."""
    G = rng(seed).standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))
    sig = kappa ** (-np.arange(n) / max(n - 1, 1))
    A = (Q * sig) @ Q.T
    return 0.5 * (A + A.T)


def spd_kappa_torch(n, kappa, seed=1002, device="cuda"):
    """Large-n variant of spd_kappa built with torch on `device` (input construction)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    G = torch.randn(n, n, generator=g, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    Q = Q * torch.sign(torch.diagonal(R))
    sig = kappa ** (-torch.arange(n, device=device, dtype=torch.float64) / max(n - 1, 1))
    A = (Q * sig) @ Q.T
    return 0.5 * (A + A.T)


def spd_kappa_butterfly_torch(n, kappa, seed=1002, device="cuda", passes=2):
    """A = Q diag(sigma) Q^T with sigma_i = kappa^(-i/(n-1)) for the largest
    orders (n a power of two), where the QR of an n x n Gaussian matrix would
    cost minutes on the FP64 pipe.  Q is a product of `passes` random butterfly
    networks -- log2(n) levels of Givens rotations pairing index i with
    i + 2^l, angles uniform in [0, 2 pi) -- with a random symmetric
    permutation after each; the eigenvalues start in a random order on the
    diagonal.  Dense, with exactly the spectrum sigma up to FP64 rounding, in
    O(passes n^2 log n) operations (input construction, float64, on `device`)."""
    import math
    import torch
    lv = n.bit_length() - 1
    if n < 2 or (1 << lv) != n:
        raise ValueError("n must be a power of two")
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    sig = kappa ** (-torch.arange(n, device=device, dtype=torch.float64) / (n - 1))
    A = torch.diag(sig[torch.randperm(n, generator=g, device=device)])
    for _ in range(passes):
        for l in range(lv):
            h = 1 << l
            th = torch.rand(n // 2, generator=g, device=device, dtype=torch.float64) * (2 * math.pi)
            c, s = torch.cos(th).view(n // (2 * h), h), torch.sin(th).view(n // (2 * h), h)
            # rows i and i + h of each pair: A <- G A
            V = A.view(n // (2 * h), 2, h, n)
            a0 = V[:, 0].clone()
            a1 = V[:, 1].clone()
            V[:, 0] = c[:, :, None] * a0 - s[:, :, None] * a1
            V[:, 1] = s[:, :, None] * a0 + c[:, :, None] * a1
            # the same rotation on the columns: A <- A G^T
            Wc = A.view(n, n // (2 * h), 2, h)
            b0 = Wc[:, :, 0].clone()
            b1 = Wc[:, :, 1].clone()
            Wc[:, :, 0] = c[None] * b0 - s[None] * b1
            Wc[:, :, 1] = s[None] * b0 + c[None] * b1
            del a0, a1, b0, b1
        p = torch.randperm(n, generator=g, device=device)
        A = A.index_select(0, p).index_select(1, p)
    A = 0.5 * (A + A.T)
    return A


def rhs(n, nrhs=16, seed=1003):
    return rng(seed).standard_normal((n, nrhs))


def gp_inputs(n, d=8, seed=1004):
    """X (n x d) iid N(0,1) and y (n) iid N(0,1)."""
    r = rng(seed)
    return r.standard_normal((n, d)), r.standard_normal(n)


def gp_kernel(X, lengthscale=1.0, jitter=1e-2):
    """K = exp(-|xi - xj|^2 / (2 l^2)) + jitter I (input construction)."""
    sq = np.sum(X * X, axis=1)
    D = np.maximum(sq[:, None] + sq[None, :] - 2.0 * X @ X.T, 0.0)
    return np.exp(-D / (2.0 * lengthscale ** 2)) + jitter * np.eye(X.shape[0])


def batched_sizes(count=4096, lo=32, hi=512, seed=1005):
    return rng(seed).integers(lo, hi + 1, count)


def batched_spd(sizes, seed0=100000):
    return [spd_mmt(int(n), seed0 + i) for i, n in enumerate(sizes)]


def fault_schedule(n, nb, kind="cholesky", rate_every=10, delta=1e3, seed=2000,
                   fault_kind=F_MEMORY):
    """Faults at steps k = o (mod rate_every), o a seeded offset in [0, rate_every),
    each at a uniform position in that step's updated region, value +delta.
    Region: Cholesky row >= col-block-row >= (k+1)b (lower block triangle),
    LU rows and cols >= (k+1)b, QR rows >= kb and cols >= (k+1)b.
    Returns a list of (step, kind, row, col, delta)."""
    r = rng(seed)
    N = (n + nb - 1) // nb
    o = int(r.integers(0, rate_every))
    out = []
    for k in range(o, N - 1, rate_every):
        T0 = (k + 1) * nb
        if kind == "qr":
            row = int(r.integers(k * nb, n))
            col = int(r.integers(T0, n))
        else:
            row = int(r.integers(T0, n))
            col = int(r.integers(T0, n))
            if kind == "cholesky" and col // nb > row // nb:
                row, col = col, row
        out.append((k, fault_kind, row, col, float(delta)))
    return out
