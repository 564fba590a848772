"""Plain FP64 CPU oracle for the ABFT one-sided decompositions.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2301_03166_b300``) and never imports it.

The decompositions and checksum logic are in ``abft_oracle.c`` (plain loops,
called through ctypes); the Cholesky adjoint and the GP gradient are written
here with numpy/scipy primitives (matmul, triangular solve, inverse).

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, exact integer cases, LAPACK (as a library
special case) and invariants.  Parity unpinned: none.
"""
import ctypes
import numpy as np

from . import build as _build

NONE, SINGLE, FULL = 0, 1, 2
F_MEMORY, F_COMPUTE, F_ROW1D, F_COL1D, F_PANEL = 0, 1, 2, 3, 4
E_0D, E_ROW, E_COL, E_UNCORR, E_CKSUM, E_PD = 0, 1, 2, 3, 4, 5


class _Event(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("row", ctypes.c_int64), ("col", ctypes.c_int64),
                ("delta", ctypes.c_double)]


class _Report(ctypes.Structure):
    _fields_ = [("detected", ctypes.c_int64), ("corrected", ctypes.c_int64),
                ("uncorrectable", ctypes.c_int64), ("checksum_repaired", ctypes.c_int64),
                ("nloc", ctypes.c_int32), ("info", ctypes.c_int32),
                ("loc", _Event * 64), ("max_ratio", ctypes.c_double),
                ("tau", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        L.orc_potf2.argtypes = [i64, dp, i64]
        L.orc_getf2.argtypes = [i64, i64, dp, i64, ctypes.POINTER(i64)]
        L.orc_geqr2.argtypes = [i64, i64, dp, i64, dp]
        L.orc_potrf.argtypes = [i64, i64, ctypes.c_int, dp, i64, ctypes.POINTER(_Event),
                                ctypes.c_int32, ctypes.c_double, ctypes.POINTER(_Report)]
        L.orc_getrf.argtypes = [i64, i64, ctypes.c_int, dp, i64, ctypes.POINTER(i64),
                                ctypes.POINTER(_Event), ctypes.c_int32, ctypes.c_double,
                                ctypes.POINTER(_Report)]
        L.orc_geqrf.argtypes = [i64, i64, ctypes.c_int, dp, i64, dp, ctypes.POINTER(_Event),
                                ctypes.c_int32, ctypes.c_double, ctypes.POINTER(_Report)]
        L.orc_potrs.argtypes = [i64, i64, dp, i64, dp, i64]
        L.orc_potrf_sched.argtypes = [i64, i64, ctypes.POINTER(ctypes.c_int32), dp, i64,
                                      ctypes.POINTER(_Event), ctypes.c_int32, ctypes.c_double,
                                      ctypes.POINTER(_Report)]
        u16p = ctypes.POINTER(ctypes.c_uint16)
        L.orc_round16.argtypes = [ctypes.c_double, ctypes.c_int, u16p]
        L.orc_round16.restype = ctypes.c_double
        L.orc_tile_sigma.argtypes = [ctypes.c_double, ctypes.c_int]
        L.orc_tile_sigma.restype = ctypes.c_double
        L.orc_mixed_coef.argtypes = [ctypes.c_double, i64]
        L.orc_mixed_coef.restype = ctypes.c_double
        L.orc_quantize.argtypes = [i64, i64, dp, i64, ctypes.c_int, dp, u16p, dp]
        L.orc_quantize.restype = None
        L.orc_syrk_mixed.argtypes = [i64, i64, i64, ctypes.c_int, dp, i64, dp, i64, u16p, dp]
        L.orc_syrk_mixed.restype = None
        L.orc_potrf_mixed.argtypes = [i64, i64, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, dp,
                                      i64, ctypes.POINTER(_Event), ctypes.c_int32,
                                      ctypes.c_double, ctypes.POINTER(_Report)]
        for f in ("orc_potf2", "orc_getf2", "orc_geqr2", "orc_potrf", "orc_getrf",
                  "orc_geqrf", "orc_potrs", "orc_potrf_sched", "orc_potrf_mixed"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _faults(faults):
    faults = list(faults or [])
    arr = (_Event * max(1, len(faults)))()
    for i, f in enumerate(faults):
        arr[i].step, arr[i].kind = int(f[0]), int(f[1])
        arr[i].row, arr[i].col, arr[i].delta = int(f[2]), int(f[3]), float(f[4])
    return arr, len(faults)


def _report(r):
    return {
        "detected": r.detected, "corrected": r.corrected,
        "uncorrectable": r.uncorrectable, "checksum_repaired": r.checksum_repaired,
        "info": r.info, "max_ratio": r.max_ratio, "tau": r.tau,
        "loc": [(r.loc[i].step, r.loc[i].kind, r.loc[i].row, r.loc[i].col, r.loc[i].delta)
                for i in range(r.nloc)],
    }


def _mat(A):
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    assert A.ndim == 2 and A.shape[0] == A.shape[1]
    return A


# ------------------------------------------------------------ unblocked
def potf2(A):
    """Unblocked lower Cholesky; returns (A with L in the lower triangle, info)."""
    A = _mat(A)
    info = lib().orc_potf2(A.shape[0], _dp(A), A.shape[1])
    return A, info


def getf2(A):
    """Unblocked LU with partial pivoting; returns (LU, ipiv (0-based), info)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    m, n = A.shape
    ipiv = np.zeros(min(m, n), dtype=np.int64)
    info = lib().orc_getf2(m, n, _dp(A), n, ipiv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return A, ipiv, info


def geqr2(A):
    """Unblocked Householder QR (larfg convention); returns (QR, tau)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    m, n = A.shape
    tau = np.zeros(min(m, n))
    lib().orc_geqr2(m, n, _dp(A), n, _dp(tau))
    return A, tau


# --------------------------------------------------------- blocked ABFT
def potrf(A, nb, mode=FULL, faults=(), tau_scale=1.0):
    """Blocked ABFT Cholesky.  Returns (A', info, report); A' holds L in the
    lower triangle and the untouched input in the strict upper triangle."""
    A = _mat(A)
    fa, nf = _faults(faults)
    rep = _Report()
    info = lib().orc_potrf(A.shape[0], nb, mode, _dp(A), max(1, A.shape[1]), fa, nf, tau_scale,
                           ctypes.byref(rep))
    return A, info, _report(rep)


def potrf_sched(A, nb, modes, faults=(), tau_scale=1.0):
    """Blocked ABFT Cholesky with one checksum mode per step (NONE / SINGLE /
    FULL; adaptive ABFT, Sec. 3.1.2).  Returns (A', info, report) as potrf."""
    A = _mat(A)
    n = A.shape[0]
    N = max(1, -(-n // nb))
    m = np.ascontiguousarray(np.asarray(modes, dtype=np.int32))
    if m.shape != (N,):
        raise ValueError(f"modes must have {N} entries")
    fa, nf = _faults(faults)
    rep = _Report()
    info = lib().orc_potrf_sched(n, nb, m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(A),
                                 max(1, A.shape[1]), fa, nf, tau_scale, ctypes.byref(rep))
    return A, info, _report(rep)


# ----------------------------------------- mixed precision (16-bit TMU)
BF16, FP16 = 1, 0


def round16(x, bf16=True):
    """x rounded to BF16 or FP16 (nearest, ties to even) from the format
    definitions; returns (value, 16-bit encoding)."""
    b = ctypes.c_uint16(0)
    v = lib().orc_round16(float(x), 1 if bf16 else 0, ctypes.byref(b))
    return v, b.value


def tile_sigma(m, bf16=True):
    """Per-tile scale 2^(ceil(log2 m) - e_t) of a tile with maximum |x| = m."""
    return lib().orc_tile_sigma(float(m), 1 if bf16 else 0)


def mixed_coef(tau_scale, g):
    """tau_scale * 4 * gamma_g(2^-24): the factor of the abs-checksum thresholds."""
    return lib().orc_mixed_coef(float(tau_scale), int(g))


def quantize(P, bf16=True):
    """One tile quantized: (sigma, 16-bit encodings, their values)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    r, c = P.shape
    bits = np.zeros((r, c), dtype=np.uint16)
    q = np.zeros((r, c))
    sig = ctypes.c_double(0.0)
    lib().orc_quantize(r, c, _dp(P), c, 1 if bf16 else 0, ctypes.byref(sig),
                       bits.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), _dp(q))
    return sig.value, bits, q


def syrk_mixed(P, C, g, bf16=True):
    """The mixed trailing update alone: returns (C - sigma_I sigma_J Lq_I Lq_J^T
    on the lower block triangle, the encodings of Lq, sigma per tile-row)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    C = np.array(C, dtype=np.float64, order="C", copy=True)
    m, k = P.shape
    bits = np.zeros((m, k), dtype=np.uint16)
    sig = np.zeros(-(-m // g))
    lib().orc_syrk_mixed(m, k, g, 1 if bf16 else 0, _dp(P), k, _dp(C), m,
                         bits.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), _dp(sig))
    return C, bits, sig


def potrf_mixed(A, nb, mode=FULL, bf16=True, faults=(), tau_scale=1.0, modes=None):
    """Blocked ABFT Cholesky in the mixed form (16-bit quantized TMU operands,
    FP32 panel solve, abs-checksum thresholds).  Returns (A', info, report);
    report["tau"] is the largest threshold applied to a trailing tile."""
    A = _mat(A)
    n = A.shape[0]
    N = max(1, -(-n // nb))
    m = np.full(N, mode, dtype=np.int32) if modes is None else \
        np.ascontiguousarray(np.asarray(modes, dtype=np.int32))
    fa, nf = _faults(faults)
    rep = _Report()
    info = lib().orc_potrf_mixed(n, nb, m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 1 if bf16 else 0, _dp(A), max(1, A.shape[1]), fa, nf, tau_scale,
                                 ctypes.byref(rep))
    return A, info, _report(rep)


def getrf(A, nb, mode=FULL, faults=(), tau_scale=1.0):
    """Blocked ABFT LU with partial pivoting.  Returns (LU, ipiv, info, report)."""
    A = _mat(A)
    n = A.shape[0]
    ipiv = np.zeros(n, dtype=np.int64)
    fa, nf = _faults(faults)
    rep = _Report()
    info = lib().orc_getrf(n, nb, mode, _dp(A), max(1, n),
                           ipiv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           fa, nf, tau_scale, ctypes.byref(rep))
    return A, ipiv, info, _report(rep)


def geqrf(A, nb, mode=FULL, faults=(), tau_scale=1.0):
    """Blocked ABFT Householder QR.  Returns (QR, tau, info, report)."""
    A = _mat(A)
    n = A.shape[0]
    tau = np.zeros(n)
    fa, nf = _faults(faults)
    rep = _Report()
    info = lib().orc_geqrf(n, nb, mode, _dp(A), max(1, n), _dp(tau), fa, nf, tau_scale,
                           ctypes.byref(rep))
    return A, tau, info, _report(rep)


def potrs(L, B):
    """X = L^{-T} L^{-1} B by forward and backward substitution."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    X = np.array(B, dtype=np.float64, order="C", copy=True)
    if X.ndim == 1:
        X = X[:, None]
    lib().orc_potrs(L.shape[0], X.shape[1], _dp(L), L.shape[1], _dp(X), X.shape[1])
    return X


# ------------------------------------------------------ derived helpers
def unpack_lu(LU, ipiv):
    """P, L, U with P A = L U from the packed getrf output (0-based ipiv)."""
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    perm = np.arange(n)
    for j, p in enumerate(ipiv):
        perm[[j, p]] = perm[[p, j]]
    P = np.eye(n)[perm]
    return P, L, U


def form_q(QR, tau):
    """Q = H_0 H_1 ... H_{n-1} from the packed geqrf output."""
    n = QR.shape[0]
    Q = np.eye(n)
    for j in range(n - 1, -1, -1):
        v = np.zeros(n)
        v[j] = 1.0
        v[j + 1:] = QR[j + 1:, j]
        Q -= tau[j] * np.outer(v, v @ Q)
    return Q


# ------------------------------------------------------------- adjoint
def potrf_backward(L, Lbar):
    """Cholesky adjoint (Murray 2016, "Differentiation of the Cholesky
    decomposition", symbolic form): with Phi(X) = tril(X) with its diagonal
    halved, Abar = L^{-T} Phi(L^T Lbar) L^{-1}, returned symmetrized
    (Abar + Abar^T)/2 -- the gradient with respect to a symmetric A."""
    import scipy.linalg as sl
    L = np.tril(np.asarray(L, dtype=np.float64))
    Lbar = np.tril(np.asarray(Lbar, dtype=np.float64))
    P = L.T @ Lbar
    P = np.tril(P) - 0.5 * np.diag(np.diag(P))
    Y = sl.solve_triangular(L, P.T, lower=True, trans=1).T      # Phi L^{-1}
    G = sl.solve_triangular(L, Y, lower=True, trans=1)           # L^{-T} Phi L^{-1}
    return 0.5 * (G + G.T)


def gp_loss_grad(K, y):
    """GP negative log-likelihood part loss = y^T K^{-1} y / 2 + logdet(K) / 2
    and its closed-form gradient dK = (K^{-1} - alpha alpha^T) / 2, alpha = K^{-1} y."""
    Kinv = np.linalg.inv(K)
    alpha = Kinv @ y
    sign, logdet = np.linalg.slogdet(K)
    loss = 0.5 * float(y @ alpha) + 0.5 * logdet
    return loss, 0.5 * (Kinv - np.outer(alpha, alpha))
