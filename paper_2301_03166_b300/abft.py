"""Thin Python binding of libabft.so (ctypes): argument marshalling only.

Every step of every factorization runs in the library's CUDA kernels; torch
supplies device memory (matrices and workspace) and the current stream.
There is no CPU fallback: if the compiled library is missing, or a tensor is
not on a CUDA device, the call raises.
"""
import ctypes
import os

import numpy as np
import torch

from . import build as _build

F64, F32, MIXED_BF16, MIXED_F16, F64_EMU = 0, 1, 2, 3, 4
NONE, SINGLE, FULL = 0, 1, 2
F_MEMORY, F_COMPUTE, F_ROW1D, F_COL1D, F_PANEL = 0, 1, 2, 3, 4
E_0D, E_ROW, E_COL, E_UNCORR, E_CKSUM, E_PD = 0, 1, 2, 3, 4, 5
ERR_UNCORRECTABLE, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED, ERR_TOO_LARGE = -1000, -1001, -1002, -1003, -1004
NOALLOC_SCRATCH_BYTES = 16 << 20   # ABFT_NOALLOC_SCRATCH_BYTES: abft_potrf_noalloc's built-in scratch
MAX_LOC = 64


class Fault(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("row", ctypes.c_int64), ("col", ctypes.c_int64),
                ("delta", ctypes.c_double)]


class Report(ctypes.Structure):
    _fields_ = [("detected", ctypes.c_int64), ("corrected", ctypes.c_int64),
                ("uncorrectable", ctypes.c_int64), ("checksum_repaired", ctypes.c_int64),
                ("nloc", ctypes.c_int32), ("info", ctypes.c_int32),
                ("loc", Fault * MAX_LOC), ("max_ratio", ctypes.c_double),
                ("tau", ctypes.c_double), ("ir_iters", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("backward_err", ctypes.c_double),
                ("gmres_iters", ctypes.c_int32), ("attempts", ctypes.c_int32),
                ("shift", ctypes.c_double)]


class AbftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None
_i64, _i32, _dbl, _vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
_sz = ctypes.POINTER(ctypes.c_size_t)

_SIGNATURES = {
    "abft_potrf_batched": [_i32, _vp, _i32, _i32, _dbl, _vp, _i32, _vp, _sz, _vp],
    "abft_batched_set_ctas_per_sm": [_i32],
    "abft_potrf_backward": [_i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _sz, _vp],
    "abft_potrf_backward_ex": [_i64, _i64, _i32, _vp, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _sz,
                               _vp],
    "abft_potrs_backward": [_i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp,
                            _i64, _vp, _sz, _vp],
    "abft_logdet": [_i64, _vp, _i64, _vp, _vp],
    "abft_logdet_backward": [_i64, _vp, _i64, _dbl, _vp, _i64, _vp],
    "abft_tril": [_i64, _vp, _i64, _vp],
    "abft_potrs": [_i64, _i64, _i64, _i32, _vp, _i64, _vp, _i64, _vp, _sz, _vp],
    "abft_posv_ir": [_i64, _i64, _i64, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                     _dbl, _i32, ctypes.POINTER(Fault), _i32, _dbl, ctypes.POINTER(Report), _vp,
                     _sz, _vp],
    "abft_posv_gmres_ir": [_i64, _i64, _i64, _i32, _i32, _vp, _i64, _vp, _i64, _vp, _i64, _vp,
                           _i64, _dbl, _i32, _i32, _dbl, _dbl, _i32, _i32, _i32,
                           ctypes.POINTER(Fault), _i32, _dbl, ctypes.POINTER(Report), _vp, _sz,
                           _vp],
    "abft_geqrf": [_i64, _i64, _i32, _i32, _vp, _i64, _vp, ctypes.POINTER(Fault), _i32, _dbl,
                   ctypes.POINTER(Report), _vp, _sz, _vp],
    "abft_getrf": [_i64, _i64, _i32, _i32, _vp, _i64, _vp, ctypes.POINTER(Fault), _i32, _dbl,
                   ctypes.POINTER(Report), _vp, _sz, _vp],
    "abft_potrf_noalloc": [_i64, _i64, _i32, _i32, _vp, _i64, ctypes.POINTER(Fault), _i32, _dbl,
                           ctypes.POINTER(Report), _vp],
    "abft_potrf": [_i64, _i64, _i32, _i32, _vp, _i64, ctypes.POINTER(Fault), _i32, _dbl,
                   ctypes.POINTER(Report), _vp, _sz, _vp],
    "abft_symm_emu": [_i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp],
    "abft_syrk_mixed": [_i64, _i64, _i64, _i32, _vp, _i64, _vp, _i64, _vp, _vp,
                        ctypes.POINTER(_i32), _vp, _sz, _vp],
    "abft_batched_partition": [_i32, ctypes.POINTER(_i64), _i32, ctypes.POINTER(_i32),
                               ctypes.POINTER(_dbl)],
    "abft_wait_selftest": [_i32, _i64, ctypes.POINTER(_i32), _vp, _sz, _vp],
    "abft_fp64_pipe_probe": [_i32, _i64, ctypes.POINTER(_dbl), _vp],
    "abft_potrf_sched": [_i64, _i64, _i32, ctypes.POINTER(_i32), _vp, _i64,
                         ctypes.POINTER(Fault), _i32, _dbl, ctypes.POINTER(Report), _vp, _sz, _vp],
}


def lib_path():
    return _build.LIB


def lib():
    """Load libabft.so (building it in-tree first when nvcc is available and
    the sources are newer).  Raises if the library cannot be loaded."""
    global _lib
    if _lib is None:
        if _build.stale():
            try:
                _build.build()
            except Exception as e:  # no compiler here: use what is on disk, or fail
                if not os.path.exists(_build.LIB):
                    raise RuntimeError(f"libabft.so is missing and could not be built: {e}")
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libabft.so is missing; run paper_2301_03166_b300/build.py")
        L = ctypes.CDLL(_build.LIB)
        for name, argt in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = argt
            fn.restype = ctypes.c_int
        L.abft_timing_enable.argtypes = [_i32]
        L.abft_set_lookahead.argtypes = [_i32]
        L.abft_set_lookahead.restype = ctypes.c_int
        L.abft_timing_marks.argtypes = [ctypes.POINTER(_i32), ctypes.POINTER(_i64),
                                        ctypes.POINTER(ctypes.c_double), _i32]
        L.abft_timing_marks.restype = ctypes.c_int
        L.abft_predict_step_times.argtypes = [ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), _i64,
                                              ctypes.POINTER(ctypes.c_double)]
        L.abft_predict_step_times.restype = ctypes.c_int
        L.abft_chol_step_work.argtypes = [_i64, _i64, _i32, _i64]
        L.abft_chol_step_work.restype = ctypes.c_double
        L.abft_timing_enable.restype = ctypes.c_int
        L.abft_timing_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]
        L.abft_timing_read.restype = ctypes.c_int
        L.abft_launch_count.restype = _i64
        L.abft_version.restype = ctypes.c_char_p
        L.abft_strerror.restype = ctypes.c_char_p
        L.abft_strerror.argtypes = [_i32]
        for name in ("abft_fc_single", "abft_fc_full"):
            getattr(L, name).argtypes = [_i64, _dbl, _dbl, _dbl]
            getattr(L, name).restype = _dbl
        L.abft_adaptive_modes.argtypes = [_i64, _i64, ctypes.POINTER(_dbl), _dbl,
                                          ctypes.POINTER(_dbl), ctypes.POINTER(_i32),
                                          ctypes.POINTER(_dbl)]
        L.abft_adaptive_modes.restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code):
    return lib().abft_strerror(int(code)).decode()


def _faults(faults):
    faults = list(faults or [])
    arr = (Fault * max(1, len(faults)))()
    for i, f in enumerate(faults):
        arr[i].step, arr[i].kind = int(f[0]), int(f[1])
        arr[i].row, arr[i].col, arr[i].delta = int(f[2]), int(f[3]), float(f[4])
    return arr, len(faults)


def report_dict(r):
    return {
        "detected": r.detected, "corrected": r.corrected,
        "uncorrectable": r.uncorrectable, "checksum_repaired": r.checksum_repaired,
        "info": r.info, "max_ratio": r.max_ratio, "tau": r.tau,
        "ir_iters": r.ir_iters, "backward_err": r.backward_err,
        "gmres_iters": r.gmres_iters, "attempts": r.attempts, "shift": r.shift,
        "loc": [(r.loc[i].step, r.loc[i].kind, r.loc[i].row, r.loc[i].col, r.loc[i].delta)
                for i in range(r.nloc)],
    }


def _check_matrix(A, name="A"):
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (no CPU fallback)")
    if A.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError(f"{name} must be a row-major 2-D tensor (stride(1) == 1)")


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Workspace:
    """Caller-owned device workspace reused across calls (grown on demand)."""

    def __init__(self, device=None):
        self.buf = None
        self.device = device

    def get(self, nbytes, device):
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != device:
            self.buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
        return self.buf


def potrf(A, nb, mode=FULL, dtype=F64, faults=(), tau_scale=1.0, report=True,
          workspace=None, stream=None, check=True):
    """ABFT Cholesky in place: the lower triangle of A becomes L.
    Returns (info_or_code, report dict or None)."""
    _check_matrix(A)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    L = lib()
    fa, nf = _faults(faults)
    need = ctypes.c_size_t(0)
    rc = L.abft_potrf(n, nb, dtype, mode, None, max(1, A.stride(0)), fa, nf, tau_scale,
                      None, None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, A.device)
    rep = Report() if report else None
    size = ctypes.c_size_t(ws.numel())
    rc = L.abft_potrf(n, nb, dtype, mode, ctypes.c_void_p(A.data_ptr()), max(1, A.stride(0)),
                      fa, nf, tau_scale, ctypes.byref(rep) if rep is not None else None,
                      ctypes.c_void_p(ws.data_ptr()), ctypes.byref(size), _stream(stream))
    if check and rc < 0 and rc != ERR_UNCORRECTABLE:
        raise AbftError(rc, strerror(rc))
    return rc, (report_dict(rep) if rep is not None else None)


def symm_emu(A, X, Y=None, workspace=None, stream=None):
    """Y = A X for symmetric A (lower triangle read), FP64-accurate on the BF16
    tensor cores (n a multiple of 32).  Returns Y."""
    _check_matrix(A)
    _check_matrix(X, "X")
    n, nrhs = X.shape
    if A.shape != (n, n):
        raise ValueError("A must be n x n")
    if Y is None:
        Y = torch.empty_like(X)
    L = lib()
    need = ctypes.c_size_t(0)
    rc = L.abft_symm_emu(n, nrhs, None, max(1, A.stride(0)), None, max(1, X.stride(0)), None,
                         max(1, Y.stride(0)), None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, A.device)
    size = ctypes.c_size_t(ws.numel())
    rc = L.abft_symm_emu(n, nrhs, ctypes.c_void_p(A.data_ptr()), max(1, A.stride(0)),
                         ctypes.c_void_p(X.data_ptr()), max(1, X.stride(0)),
                         ctypes.c_void_p(Y.data_ptr()), max(1, Y.stride(0)),
                         ctypes.c_void_p(ws.data_ptr()), ctypes.byref(size), _stream(stream))
    if rc != 0:
        raise AbftError(rc, strerror(rc))
    return Y


def syrk_mixed(P, C, g, dtype=MIXED_BF16, workspace=None, stream=None, sync=True):
    """The mixed-precision trailing update on its own: C -= sigma_I sigma_J
    (Pq_I Pq_J^T) on the lower block triangle (in place).  Returns (the 16-bit
    codes of Pq as a uint16 numpy array, sigma as a numpy array) when sync,
    else (Pq, sigma) as device tensors."""
    _check_matrix(P, "P")
    _check_matrix(C, "C")
    m, k = P.shape
    if C.shape != (m, m):
        raise ValueError("C must be m x m")
    Pq = torch.empty((m, k), dtype=torch.int16, device=P.device)
    sig = torch.empty(max(1, -(-m // g)), dtype=torch.float64, device=P.device)
    L = lib()
    need = ctypes.c_size_t(0)
    rc = L.abft_syrk_mixed(m, k, g, dtype, None, max(1, P.stride(0)), None, max(1, C.stride(0)),
                           None, None, None, None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, P.device)
    size = ctypes.c_size_t(ws.numel())
    tout = _i32(0)
    rc = L.abft_syrk_mixed(m, k, g, dtype, ctypes.c_void_p(P.data_ptr()), max(1, P.stride(0)),
                           ctypes.c_void_p(C.data_ptr()), max(1, C.stride(0)),
                           ctypes.c_void_p(Pq.data_ptr()), ctypes.c_void_p(sig.data_ptr()),
                           ctypes.byref(tout) if sync else None,
                           ctypes.c_void_p(ws.data_ptr()), ctypes.byref(size), _stream(stream))
    if rc != 0:
        raise AbftError(rc, strerror(rc))
    if not sync:
        return Pq, sig
    return Pq.cpu().numpy().view(np.uint16), sig.cpu().numpy()


def wait_selftest(which, limit_ns=1000000, device="cuda", stream=None):
    """Run one case of abft_wait_selftest; returns (return code, error code)."""
    L = lib()
    need = ctypes.c_size_t(0)
    rc = L.abft_wait_selftest(which, limit_ns, None, None, ctypes.byref(need), None)
    if rc < 0 and rc > ERR_UNCORRECTABLE:
        raise AbftError(rc, strerror(rc))
    ws = torch.zeros(max(256, need.value), dtype=torch.uint8, device=device)
    size = ctypes.c_size_t(ws.numel())
    err = _i32(0)
    rc = L.abft_wait_selftest(which, limit_ns, ctypes.byref(err), ctypes.c_void_p(ws.data_ptr()),
                              ctypes.byref(size), _stream(stream))
    return rc, err.value


def fp64_pipe_probe(which, iters=20000, stream=None):
    """FP64 multiply-add rate in TFLOP/s: which 0 = FMA, 1 = tensor-core MMA."""
    out = _dbl(0.0)
    rc = lib().abft_fp64_pipe_probe(which, iters, ctypes.byref(out), _stream(stream))
    if rc != 0:
        raise AbftError(rc, strerror(rc))
    return out.value


def _modes_array(modes, n, nb):
    N = max(1, -(-n // nb)) if n > 0 else 0
    m = np.ascontiguousarray(np.asarray(list(modes), dtype=np.int32))
    if m.shape != (N,):
        raise ValueError(f"modes must have {N} entries (one per step)")
    return m


def potrf_sched(A, nb, modes, dtype=F64, faults=(), tau_scale=1.0, workspace=None, stream=None,
                check=True):
    """ABFT Cholesky in place with one checksum mode per step (adaptive ABFT).
    Returns (info_or_code, report dict)."""
    _check_matrix(A)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    m = _modes_array(modes, n, nb)
    mp = m.ctypes.data_as(ctypes.POINTER(_i32))
    L = lib()
    fa, nf = _faults(faults)
    need = ctypes.c_size_t(0)
    rc = L.abft_potrf_sched(n, nb, dtype, mp, None, max(1, A.stride(0)), fa, nf, tau_scale, None,
                            None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, A.device)
    rep = Report()
    size = ctypes.c_size_t(ws.numel())
    rc = L.abft_potrf_sched(n, nb, dtype, mp, ctypes.c_void_p(A.data_ptr()), max(1, A.stride(0)),
                            fa, nf, tau_scale, ctypes.byref(rep), ctypes.c_void_p(ws.data_ptr()),
                            ctypes.byref(size), _stream(stream))
    if check and rc < 0 and rc != ERR_UNCORRECTABLE:
        raise AbftError(rc, strerror(rc))
    return rc, report_dict(rep)


def fc_single(S, mu0, mu1, mu2):
    """Fault coverage of single-side checksums for one interval (host only)."""
    return lib().abft_fc_single(int(S), float(mu0), float(mu1), float(mu2))


def fc_full(S, mu0, mu1, mu2):
    """Fault coverage of full checksums for one interval (host only)."""
    return lib().abft_fc_full(int(S), float(mu0), float(mu1), float(mu2))


def adaptive_modes(n, nb, lambdas, fc_desired, step_seconds):
    """Per-step checksum modes of adaptive ABFT (host only).  Returns
    (modes list, coverage list)."""
    N = max(0, -(-n // nb))
    lam = (_dbl * 3)(*[float(x) for x in lambdas])
    ts = np.ascontiguousarray(np.asarray(step_seconds, dtype=np.float64))
    if ts.shape != (N,):
        raise ValueError(f"step_seconds must have {N} entries")
    modes = np.zeros(max(N, 1), dtype=np.int32)
    cov = np.zeros(max(N, 1), dtype=np.float64)
    rc = lib().abft_adaptive_modes(n, nb, lam, float(fc_desired),
                                   ts.ctypes.data_as(ctypes.POINTER(_dbl)),
                                   modes.ctypes.data_as(ctypes.POINTER(_i32)),
                                   cov.ctypes.data_as(ctypes.POINTER(_dbl)))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return modes[:N].tolist(), cov[:N].tolist()


PHASES = ("pd", "pu", "tmu", "verify", "other", "solve")


def set_lookahead(on=True):
    """Look-ahead of the blocked Cholesky (next diagonal block factored on a
    side stream while the rest of the update runs); returns the previous
    setting.  Results are identical either way."""
    return bool(lib().abft_set_lookahead(1 if on else 0))


def timing_enable(on=True):
    """Per-phase CUDA-event timing inside the library (resets the totals)."""
    lib().abft_timing_enable(1 if on else 0)


def timing_read():
    ms = (ctypes.c_double * len(PHASES))()
    cnt = (ctypes.c_int64 * len(PHASES))()
    lib().abft_timing_read(ms, cnt, len(PHASES))
    return {p: (ms[i], cnt[i]) for i, p in enumerate(PHASES)}


def timing_marks():
    """Timed intervals since timing_enable: list of (phase name, iteration, ms)."""
    L = lib()
    n = L.abft_timing_marks(None, None, None, 0)
    if n <= 0:
        return []
    ph = (_i32 * n)()
    st = (_i64 * n)()
    ms = (ctypes.c_double * n)()
    L.abft_timing_marks(ph, st, ms, n)
    return [(PHASES[ph[i]], st[i], ms[i]) for i in range(n)]


def predict_step_times(T, W):
    """Per-iteration time prediction from the last four iterations (Sec. 3.2.1),
    computed by the library: pred[k] = sum_i w_i (W[k] / W[k-i]) T[k-i]."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    if T.shape != W.shape or T.ndim != 1:
        raise ValueError("T and W must be 1-D arrays of the same length")
    out = np.empty_like(T)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().abft_predict_step_times(T.ctypes.data_as(dp), W.ctypes.data_as(dp), T.size,
                                       out.ctypes.data_as(dp))
    if rc != 0:
        raise AbftError(rc, "bad arguments")
    return out


def chol_step_work(n, nb, phase, k):
    """Work of operation `phase` ('pd', 'pu', 'tmu', 'verify') at iteration k."""
    return lib().abft_chol_step_work(n, nb, PHASES.index(phase), k)


def launch_count():
    return int(lib().abft_launch_count())


def getrf(A, nb, mode=FULL, dtype=F64, faults=(), tau_scale=1.0, report=True,
          workspace=None, stream=None, check=True):
    """ABFT LU with partial pivoting in place (LAPACK getrf layout).
    Returns (info_or_code, ipiv int64 CUDA tensor (0-based), report dict or None)."""
    _check_matrix(A)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    L = lib()
    fa, nf = _faults(faults)
    need = ctypes.c_size_t(0)
    rc = L.abft_getrf(n, nb, dtype, mode, None, max(1, A.stride(0)), None, fa, nf, tau_scale,
                      None, None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, A.device)
    ipiv = torch.zeros(max(n, 1), dtype=torch.int64, device=A.device)
    rep = Report() if report else None
    size = ctypes.c_size_t(ws.numel())
    rc = L.abft_getrf(n, nb, dtype, mode, ctypes.c_void_p(A.data_ptr()), max(1, A.stride(0)),
                      ctypes.c_void_p(ipiv.data_ptr()), fa, nf, tau_scale,
                      ctypes.byref(rep) if rep is not None else None,
                      ctypes.c_void_p(ws.data_ptr()), ctypes.byref(size), _stream(stream))
    if check and rc < 0 and rc != ERR_UNCORRECTABLE:
        raise AbftError(rc, strerror(rc))
    return rc, ipiv[:n], (report_dict(rep) if rep is not None else None)


def geqrf(A, nb, mode=FULL, dtype=F64, faults=(), tau_scale=1.0, report=True,
          workspace=None, stream=None, check=True):
    """ABFT Householder QR in place (LAPACK geqrf layout).
    Returns (code, tau float64 CUDA tensor, report dict or None)."""
    _check_matrix(A)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    L = lib()
    fa, nf = _faults(faults)
    need = ctypes.c_size_t(0)
    rc = L.abft_geqrf(n, nb, dtype, mode, None, max(1, A.stride(0)), None, fa, nf, tau_scale,
                      None, None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, A.device)
    tau = torch.zeros(max(n, 1), dtype=torch.float64, device=A.device)
    rep = Report() if report else None
    size = ctypes.c_size_t(ws.numel())
    rc = L.abft_geqrf(n, nb, dtype, mode, ctypes.c_void_p(A.data_ptr()), max(1, A.stride(0)),
                      ctypes.c_void_p(tau.data_ptr()), fa, nf, tau_scale,
                      ctypes.byref(rep) if rep is not None else None,
                      ctypes.c_void_p(ws.data_ptr()), ctypes.byref(size), _stream(stream))
    if check and rc < 0 and rc != ERR_UNCORRECTABLE:
        raise AbftError(rc, strerror(rc))
    return rc, tau[:n], (report_dict(rep) if rep is not None else None)


def potrs(L, B, nb=256, dtype=F64, workspace=None, stream=None):
    """In place B := L^{-T} L^{-1} B with the lower factor L (CUDA float64)."""
    _check_matrix(L, "L")
    _check_matrix(B, "B")
    n, nrhs = B.shape
    Lb = lib()
    need = ctypes.c_size_t(0)
    rc = Lb.abft_potrs(n, nrhs, nb, dtype, None, max(1, L.stride(0)), None, max(1, B.stride(0)),
                       None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, B.device)
    size = ctypes.c_size_t(ws.numel())
    rc = Lb.abft_potrs(n, nrhs, nb, dtype, ctypes.c_void_p(L.data_ptr()), max(1, L.stride(0)),
                       ctypes.c_void_p(B.data_ptr()), max(1, B.stride(0)),
                       ctypes.c_void_p(ws.data_ptr()), ctypes.byref(size), _stream(stream))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return B


def posv_ir(A, B, nb=256, dtype=MIXED_BF16, mode=FULL, tol=1e-12, maxit=50, faults=(),
            tau_scale=1.0, L=None, X=None, workspace=None, stream=None, check=True):
    """Solve A X = B (A SPD, lower triangle read) by an ABFT Cholesky in `dtype`
    plus iterative refinement with an FP64 residual.  Returns (code, X, L, report)."""
    _check_matrix(A)
    _check_matrix(B, "B")
    n, nrhs = B.shape
    L = torch.empty_like(A) if L is None else L
    X = torch.empty_like(B) if X is None else X
    Lb = lib()
    fa, nf = _faults(faults)
    need = ctypes.c_size_t(0)
    rc = Lb.abft_posv_ir(n, nrhs, nb, dtype, mode, None, max(1, A.stride(0)), None,
                         max(1, L.stride(0)), None, max(1, B.stride(0)), None, max(1, X.stride(0)),
                         tol, maxit, fa, nf, tau_scale, None, None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, A.device)
    rep = Report()
    size = ctypes.c_size_t(ws.numel())
    rc = Lb.abft_posv_ir(n, nrhs, nb, dtype, mode, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                         ctypes.c_void_p(L.data_ptr()), L.stride(0), ctypes.c_void_p(B.data_ptr()),
                         B.stride(0), ctypes.c_void_p(X.data_ptr()), X.stride(0), tol, maxit, fa,
                         nf, tau_scale, ctypes.byref(rep), ctypes.c_void_p(ws.data_ptr()),
                         ctypes.byref(size), _stream(stream))
    if check and rc < 0 and rc != ERR_UNCORRECTABLE:
        raise AbftError(rc, strerror(rc))
    return rc, X, L, report_dict(rep)


def posv_gmres_ir(A, B, nb=256, dtype=MIXED_BF16, mode=FULL, tol=1e-12, maxit=20, m=30,
                  inner_tol=1e-6, shift=-1.0, scale=True, precond_f64=False, inner_f32=False,
                  faults=(), tau_scale=1.0, L=None, X=None, workspace=None, stream=None,
                  check=True):
    """Solve A X = B (A SPD, lower triangle read) by GMRES-based iterative
    refinement preconditioned by an ABFT Cholesky of the scaled, shifted matrix
    in `dtype` (shift < 0: automatic).  Returns (code, X, L, report)."""
    _check_matrix(A)
    _check_matrix(B, "B")
    n, nrhs = B.shape
    L = torch.empty_like(A) if L is None else L
    X = torch.empty_like(B) if X is None else X
    Lb = lib()
    fa, nf = _faults(faults)
    need = ctypes.c_size_t(0)
    rc = Lb.abft_posv_gmres_ir(n, nrhs, nb, dtype, mode, None, max(1, A.stride(0)), None,
                               max(1, L.stride(0)), None, max(1, B.stride(0)), None,
                               max(1, X.stride(0)), tol, maxit, m, inner_tol, shift, int(scale),
                               int(precond_f64), int(inner_f32), fa, nf, tau_scale, None, None,
                               ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, A.device)
    rep = Report()
    size = ctypes.c_size_t(ws.numel())
    rc = Lb.abft_posv_gmres_ir(n, nrhs, nb, dtype, mode, _ptr(A), A.stride(0), _ptr(L),
                               L.stride(0), _ptr(B), B.stride(0), _ptr(X), X.stride(0), tol,
                               maxit, m, inner_tol, shift, int(scale), int(precond_f64),
                               int(inner_f32), fa, nf, tau_scale, ctypes.byref(rep), _ptr(ws),
                               ctypes.byref(size), _stream(stream))
    if check and rc < 0 and rc != ERR_UNCORRECTABLE:
        raise AbftError(rc, strerror(rc))
    return rc, X, L, report_dict(rep)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _ws_call(fn, query_args, run_args, device, workspace):
    need = ctypes.c_size_t(0)
    rc = fn(*query_args, None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, device)
    size = ctypes.c_size_t(ws.numel())
    return run_args, ws, size


def potrf_backward(L, Lbar, nb=256, sym=True, Abar=None, workspace=None, stream=None,
                   dtype=F64):
    """Adjoint of the Cholesky factorization: Abar from L and Lbar (lower
    triangles read).  sym=True returns the symmetric gradient.  dtype F64_EMU
    runs the dominant product FP64-accurate on the BF16 tensor cores (nb 128
    or 256, n a multiple of nb)."""
    _check_matrix(L, "L")
    _check_matrix(Lbar, "Lbar")
    n = L.shape[0]
    Abar = torch.empty_like(L) if Abar is None else Abar
    Lb = lib()
    need = ctypes.c_size_t(0)
    rc = Lb.abft_potrf_backward_ex(n, nb, dtype, None, max(1, L.stride(0)), None,
                                   max(1, Lbar.stride(0)), None, max(1, Abar.stride(0)),
                                   1 if sym else 0, None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, L.device)
    size = ctypes.c_size_t(ws.numel())
    rc = Lb.abft_potrf_backward_ex(n, nb, dtype, _ptr(L), L.stride(0), _ptr(Lbar), Lbar.stride(0),
                                   _ptr(Abar), Abar.stride(0), 1 if sym else 0, _ptr(ws),
                                   ctypes.byref(size), _stream(stream))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return Abar


def potrs_backward(L, X, Xbar, Lbar, nb=256, workspace=None, stream=None):
    """For X = A^{-1} B: returns Bbar = A^{-1} Xbar and accumulates
    Lbar -= tril((Bbar X^T + X Bbar^T) L)."""
    n, nrhs = X.shape
    Bbar = torch.empty_like(X)
    Lb = lib()
    need = ctypes.c_size_t(0)
    rc = Lb.abft_potrs_backward(n, nrhs, nb, None, max(1, L.stride(0)), None, max(1, X.stride(0)),
                                None, max(1, Xbar.stride(0)), None, max(1, Bbar.stride(0)), None,
                                max(1, Lbar.stride(0)), None, ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, L.device)
    size = ctypes.c_size_t(ws.numel())
    rc = Lb.abft_potrs_backward(n, nrhs, nb, _ptr(L), L.stride(0), _ptr(X), X.stride(0), _ptr(Xbar),
                                Xbar.stride(0), _ptr(Bbar), Bbar.stride(0), _ptr(Lbar),
                                Lbar.stride(0), _ptr(ws), ctypes.byref(size), _stream(stream))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return Bbar


def logdet(L, out=None, stream=None):
    out = torch.empty((), dtype=torch.float64, device=L.device) if out is None else out
    rc = lib().abft_logdet(L.shape[0], _ptr(L), max(1, L.stride(0)), _ptr(out), _stream(stream))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return out


def logdet_backward(L, gbar, Lbar, stream=None):
    rc = lib().abft_logdet_backward(L.shape[0], _ptr(L), max(1, L.stride(0)), float(gbar),
                                    _ptr(Lbar), max(1, Lbar.stride(0)), _stream(stream))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return Lbar


def tril_(A, stream=None):
    rc = lib().abft_tril(A.shape[0], _ptr(A), max(1, A.stride(0)), _stream(stream))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return A


# ------------------------------------------------------------------ batched
import numpy as _np

_ITEM = _np.dtype([("A", "<u8"), ("lda", "<i8"), ("n", "<i4"), ("id", "<i4"), ("nb", "<i4"),
                   ("fstep", "<i4"), ("fkind", "<i4"), ("frow", "<i4"), ("fcol", "<i4"),
                   ("pad", "<i4"), ("fdelta", "<f8")])
_STATUS_FIELDS = ("info", "detected", "corrected", "uncorrectable", "ev_step", "ev_kind",
                  "ev_row", "ev_col")


class Batch:
    """Device-resident descriptors of a batch of square matrices stored back
    to back in one CUDA buffer; descriptors are ordered by decreasing n."""

    def __init__(self, buf, sizes, offsets, nb, faults=None):
        self.buf, self.sizes, self.offsets = buf, list(sizes), list(offsets)
        esz = buf.element_size()
        order = sorted(range(len(sizes)), key=lambda i: -sizes[i])
        items = _np.zeros(len(sizes), dtype=_ITEM)
        faults = faults or {}
        for slot, i in enumerate(order):
            n = int(sizes[i])
            it = items[slot]
            it["A"] = buf.data_ptr() + int(offsets[i]) * esz
            it["lda"], it["n"], it["id"] = n, n, i
            it["nb"] = nb(n) if callable(nb) else int(nb)
            f = faults.get(i)
            if f is None:
                it["fstep"] = -1
            else:
                it["fstep"], it["fkind"], it["frow"], it["fcol"], it["fdelta"] = f
        self.items = torch.from_numpy(items.view(_np.uint8)).to(buf.device)
        self.status = torch.zeros((len(sizes), len(_STATUS_FIELDS)), dtype=torch.int32,
                                  device=buf.device)

    def matrix(self, i):
        n, o = self.sizes[i], self.offsets[i]
        return self.buf[o:o + n * n].view(n, n)

    def statuses(self):
        st = self.status.cpu().numpy()
        return [dict(zip(_STATUS_FIELDS, map(int, row))) for row in st]


def set_batched_ctas_per_sm(ctas):
    """Persistent CTAs per SM of the batched launch (0: the default, the most
    that fit); returns the previous setting."""
    rc = lib().abft_batched_set_ctas_per_sm(int(ctas))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return rc


def potrf_batched(batch, mode=FULL, tau_scale=1.0, use_graph=False, workspace=None, stream=None):
    """Factor every matrix of `batch` in one persistent launch (FP64 or FP32
    according to the buffer dtype)."""
    dtype = F64 if batch.buf.dtype == torch.float64 else F32
    L = lib()
    need = ctypes.c_size_t(0)
    count = len(batch.sizes)
    rc = L.abft_potrf_batched(count, None, dtype, mode, tau_scale, None, 0, None,
                              ctypes.byref(need), None)
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    ws = (workspace or Workspace()).get(need.value, batch.buf.device)
    size = ctypes.c_size_t(ws.numel())
    rc = L.abft_potrf_batched(count, _ptr(batch.items), dtype, mode, tau_scale, _ptr(batch.status),
                              1 if use_graph else 0, _ptr(ws), ctypes.byref(size), _stream(stream))
    if rc < 0:
        raise AbftError(rc, strerror(rc))
    return batch
