"""Pins of the oracle's ABFT logic (Sec. 3.1.2): encode, carry, verify,
locate, correct, and the 0D / 1D / 2D error classes.

What fixes the expected values: a clean run must raise no flag (the carried
checksums equal the recomputed sums up to rounding); an injected error at a
known position must be located there and its size recovered; with integer
data every sum is exact, so correction restores the factor bit for bit; full
checksums correct 0D and 1D errors, single-side ones correct 0D only, and two
errors in different rows and columns of one block (2D) are uncorrectable.
"""
import numpy as np
import pytest

import oracle
from paper_2301_03166_b300 import workloads as W

U = 2.0 ** -53
FULL, SINGLE, NONE = oracle.FULL, oracle.SINGLE, oracle.NONE


def _chol(A, nb, mode, faults=()):
    L, info, rep = oracle.potrf(A, nb, mode, faults)
    assert info == 0
    return np.tril(L), rep


def _lu(A, nb, mode, faults=()):
    LU, ipiv, info, rep = oracle.getrf(A, nb, mode, faults)
    return LU, ipiv, rep


def _qr(A, nb, mode, faults=()):
    QR, tau, info, rep = oracle.geqrf(A, nb, mode, faults)
    return QR, tau, rep


@pytest.mark.parametrize("mode", [SINGLE, FULL])
@pytest.mark.parametrize("n,nb", [(100, 32), (160, 32), (257, 64)])
def test_no_false_positive(mode, n, nb):
    A = W.spd_mmt(n, seed=n)
    L, rep = _chol(A, nb, mode)
    assert rep["detected"] == 0 and rep["max_ratio"] < 1e-2
    LU, ipiv, rep = _lu(W.uniform(n, seed=n), nb, mode)
    assert rep["detected"] == 0 and rep["max_ratio"] < 1e-2
    QR, tau, rep = _qr(W.uniform(n, seed=n), nb, mode)
    assert rep["detected"] == 0 and rep["max_ratio"] < 1e-2


def test_tau_formula():
    n, nb = 100, 32
    A = W.spd_mmt(n, 1)
    _, rep = _chol(A, nb, FULL)
    assert rep["tau"] == 8.0 * U * n * nb * A.diagonal().max()


@pytest.mark.parametrize("mode", [SINGLE, FULL])
@pytest.mark.parametrize("kind", [oracle.F_MEMORY, oracle.F_COMPUTE])
def test_chol_0d_located_and_corrected(mode, kind):
    n, nb = 160, 32
    A = W.spd_mmt(n, 9)
    Lc, _ = _chol(A, nb, mode)
    f = [(2, kind, 150, 100, 1e3)]          # trailing region of step 2: rows/cols >= 96
    L, rep = _chol(A, nb, mode, f)
    assert [(e[0], e[1], e[2], e[3]) for e in rep["loc"]] == [(2, oracle.E_0D, 150, 100)]
    assert abs(rep["loc"][0][4] - 1e3) < 1e-9
    assert rep["corrected"] == 1 and rep["uncorrectable"] == 0
    assert np.abs(L - Lc).max() < 1e-11
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) <= 10 * n * U


def test_chol_no_abft_fault_corrupts():
    n, nb = 160, 32
    A = W.spd_mmt(n, 9)
    Lc, _ = _chol(A, nb, NONE)
    L, rep = _chol(A, nb, NONE, [(2, oracle.F_MEMORY, 150, 100, 1.0)])
    assert rep["detected"] == 0 and np.abs(L - Lc).max() > 1e-3


@pytest.mark.parametrize("mode", [SINGLE, FULL])
def test_chol_integer_exact_correction(mode):
    """Integer data: sums are exact, so the corrected factor is L0 bit-exactly."""
    n, nb = 64, 16
    L0 = W.integer_l0(n, 3)
    A = L0 @ L0.T
    f = [(1, oracle.F_MEMORY, 50, 33, 1000.0), (2, oracle.F_PANEL, 60, 40, 7.0)]
    L, rep = _chol(A, nb, mode, f)
    assert np.array_equal(L, L0)
    assert [(e[0], e[2], e[3]) for e in rep["loc"]] == [(1, 50, 33), (2, 60, 40)]
    assert [e[4] for e in rep["loc"]] == [1000.0, 7.0]


@pytest.mark.parametrize("mode", [SINGLE, FULL])
def test_chol_panel_fault_corrected_before_tmu(mode):
    n, nb = 160, 32
    A = W.spd_mmt(n, 12)
    Lc, _ = _chol(A, nb, mode)
    L, rep = _chol(A, nb, mode, [(1, oracle.F_PANEL, 130, 50, 1e3)])
    assert [(e[0], e[2], e[3]) for e in rep["loc"]] == [(1, 130, 50)]
    assert np.abs(L - Lc).max() < 1e-11


def test_chol_1d_row_and_col_full_vs_single():
    n, nb = 160, 32
    A = W.spd_mmt(n, 13)
    Lc, _ = _chol(A, nb, FULL)
    row = [(1, oracle.F_ROW1D, 140, 100, 50.0)]   # row 140, cols 100..127
    col = [(1, oracle.F_COL1D, 130, 70, 50.0)]    # col 70, rows 130..159
    L, rep = _chol(A, nb, FULL, row)
    assert rep["corrected"] == 28 and all(e[1] == oracle.E_ROW and e[2] == 140 for e in rep["loc"])
    assert np.abs(L - Lc).max() < 1e-10
    L, rep = _chol(A, nb, FULL, col)
    assert rep["corrected"] == 30 and all(e[1] == oracle.E_COL and e[3] == 70 for e in rep["loc"])
    assert np.abs(L - Lc).max() < 1e-10
    # single-side: a row error is a set of 0D errors in distinct columns (located
    # by the weighted checksum); a column error is not locatable.
    L, rep = _chol(A, nb, SINGLE, row)
    assert rep["corrected"] == 28 and np.abs(L - Lc).max() < 1e-10
    L, info, rep = oracle.potrf(A, nb, SINGLE, col)
    assert info != 0 or rep["uncorrectable"] > 0 or np.abs(np.tril(L) - Lc).max() > 1e-3


def test_2d_uncorrectable():
    n, nb = 160, 32
    A = W.spd_mmt(n, 14)
    f = [(1, oracle.F_MEMORY, 130, 100, 5.0), (1, oracle.F_MEMORY, 140, 110, 6.0)]
    L, info, rep = oracle.potrf(A, nb, FULL, f)
    # the 2D error is reported at its step; what later steps do with the
    # uncorrected error is not specified
    assert rep["uncorrectable"] >= 1
    assert rep["loc"][0][:4] == (1, oracle.E_UNCORR, 128, 96)


def test_faults_in_distinct_blocks_all_corrected():
    n, nb = 192, 32
    A = W.spd_mmt(n, 15)
    Lc, _ = _chol(A, nb, FULL)
    f = [(0, 0, 40, 35, 1e3), (0, 0, 100, 33, -2e2), (0, 1, 190, 180, 3.0), (3, 0, 170, 130, 1e3)]
    L, rep = _chol(A, nb, FULL, f)
    assert rep["corrected"] == 4 and rep["uncorrectable"] == 0
    assert [(e[0], e[2], e[3]) for e in rep["loc"]] == [(0, 40, 35), (0, 100, 33), (0, 190, 180), (3, 170, 130)]
    assert np.abs(L - Lc).max() < 1e-11


def test_invalid_fault_rejected():
    A = W.spd_mmt(64, 1)
    _, info, _ = oracle.potrf(A, 16, FULL, [(0, 0, 5, 40, 1.0)])   # above the diagonal block
    assert info < 0
    _, info, _ = oracle.potrf(A, 16, FULL, [(3, 0, 60, 60, 1.0)])  # last step has no TMU
    assert info < 0


# ------------------------------------------------------------------- LU
@pytest.mark.parametrize("mode", [SINGLE, FULL])
def test_lu_0d_and_panel(mode):
    n, nb = 130, 32
    A = W.uniform(n, 21)
    LUc, ipc, _ = _lu(A, nb, mode)
    f = [(1, oracle.F_MEMORY, 100, 70, 1e3), (2, oracle.F_PANEL, 70, 120, 4.0)]
    LU, ip, rep = _lu(A, nb, mode, f)
    assert [(e[0], e[2], e[3]) for e in rep["loc"]] == [(1, 100, 70), (2, 70, 120)]
    assert np.array_equal(ip, ipc) and np.abs(LU - LUc).max() < 1e-10


def test_lu_exact_with_fault():
    n, nb = 64, 16
    A, P0, L0, U0 = W.lu_exact(n, 5)
    LU, ip, rep = _lu(A, nb, FULL, [(1, 0, 40, 50, 512.0)])
    P, L, Um = oracle.unpack_lu(LU, ip)
    assert np.array_equal(L, L0) and np.array_equal(Um, U0) and rep["corrected"] == 1


def test_lu_1d():
    n, nb = 128, 32
    A = W.uniform(n, 22)
    LUc, _, _ = _lu(A, nb, FULL)
    LU, _, rep = _lu(A, nb, FULL, [(0, oracle.F_COL1D, 40, 50, 3.0)])
    assert rep["corrected"] == 24 and np.abs(LU - LUc).max() < 1e-10
    LU, _, rep = _lu(A, nb, SINGLE, [(0, oracle.F_COL1D, 40, 50, 3.0)])
    assert np.abs(LU - LUc).max() > 1e-3


# ------------------------------------------------------------------- QR
@pytest.mark.parametrize("mode", [SINGLE, FULL])
def test_qr_0d(mode):
    n, nb = 130, 32
    A = W.uniform(n, 31)
    QRc, tc, _ = _qr(A, nb, mode)
    QR, t, rep = _qr(A, nb, mode, [(1, 0, 40, 70, 1e3), (2, 1, 64, 100, -3.0)])
    assert [(e[0], e[2], e[3]) for e in rep["loc"]] == [(1, 40, 70), (2, 64, 100)]
    assert np.abs(QR - QRc).max() < 1e-10 and np.abs(t - tc).max() < 1e-12


def test_qr_1d_full():
    n, nb = 128, 32
    A = W.uniform(n, 32)
    QRc, _, _ = _qr(A, nb, FULL)
    QR, _, rep = _qr(A, nb, FULL, [(1, oracle.F_ROW1D, 40, 70, 2.0)])
    assert rep["corrected"] == 26 and np.abs(QR - QRc).max() < 1e-10


# ------------------------------------------------------ fault schedule
def test_fault_schedule_rate():
    f = W.fault_schedule(16384, 256, "cholesky")
    steps = [x[0] for x in f]
    assert all(b - a == 10 for a, b in zip(steps, steps[1:]))
    for k, kind, r, c, d in f:
        assert r >= (k + 1) * 256 and c >= (k + 1) * 256 and c // 256 <= r // 256
