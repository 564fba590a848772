"""GPU parity of the ABFT LU with partial pivoting (abft_getrf through the C
ABI) against the CPU oracle: pivots, factors, event lists (Sec. 2.1, 3.1.2)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu_getrf(A, nb, mode, faults=()):
    T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    rc, ipiv, rep = abft.getrf(T, nb, mode, faults=faults)
    torch.cuda.synchronize()
    return rc, T.cpu().numpy(), ipiv.cpu().numpy(), rep


def events(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("n,nb", [(1, 32), (31, 32), (100, 32), (128, 64), (257, 64), (300, 128),
                                  (513, 256), (700, 512)])
def test_parity_clean(n, nb, mode):
    A = W.uniform(n, seed=200 + n)
    LUo, ipo, info_o, rep_o = oracle.getrf(A, nb, mode)
    rc, LU, ip, rep = gpu_getrf(A, nb, mode)
    assert rc == 0 and info_o == 0
    assert np.array_equal(ip, ipo)
    assert np.abs(LU - LUo).max() <= 1e-12 * max(1.0, np.abs(LUo).max())
    P, L, U = oracle.unpack_lu(LU, ip)
    assert np.linalg.norm(P @ A - L @ U) / np.linalg.norm(A) <= 1e-13
    assert rep["detected"] == 0
    if mode != oracle.NONE:
        assert rep["max_ratio"] < 1e-2
        assert abs(rep["tau"] - rep_o["tau"]) <= 1e-12 * rep_o["tau"]


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.FULL])
def test_exact_plu(mode):
    n, nb = 128, 32
    A, P0, L0, U0 = W.lu_exact(n, 5)
    rc, LU, ip, rep = gpu_getrf(A, nb, mode)
    P, L, U = oracle.unpack_lu(LU, ip)
    assert rc == 0 and np.array_equal(P, P0.T) and np.array_equal(L, L0) and np.array_equal(U, U0)
    if mode != oracle.NONE:
        f = [(1, oracle.F_MEMORY, 100, 70, 512.0), (0, oracle.F_PANEL, 10, 50, 4.0)]
        rc, LU, ip, rep = gpu_getrf(A, nb, mode, f)
        P, L, U = oracle.unpack_lu(LU, ip)
        assert np.array_equal(L, L0) and np.array_equal(U, U0)
        _, _, _, rep_o = oracle.getrf(A, nb, mode, f)
        assert events(rep) == events(rep_o) and rep["corrected"] == 2


@pytest.mark.parametrize("mode", [oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("faults", [
    [(1, oracle.F_MEMORY, 100, 70, 1e3), (2, oracle.F_PANEL, 70, 120, 4.0)],
    [(1, oracle.F_COMPUTE, 150, 180, -20.0)],
    [(0, oracle.F_COL1D, 40, 50, 3.0)],
    [(0, oracle.F_ROW1D, 40, 50, 3.0)],
    [(1, oracle.F_MEMORY, 130, 100, 5.0), (1, oracle.F_MEMORY, 140, 110, 6.0)],
])
def test_error_classes_match_oracle(mode, faults):
    n, nb = 192, 32
    A = W.uniform(n, 23)
    LUo, ipo, info_o, rep_o = oracle.getrf(A, nb, mode, faults)
    rc, LU, ip, rep = gpu_getrf(A, nb, mode, faults)
    for key in ("detected", "corrected", "uncorrectable", "checksum_repaired"):
        assert rep[key] == rep_o[key], key
    if len(rep_o["loc"]) < 64:
        assert events(rep) == events(rep_o)
    if rep_o["uncorrectable"] == 0:
        assert np.array_equal(ip, ipo)
        assert np.abs(LU - LUo).max() <= 1e-10


def test_zero_pivot_info():
    A = W.uniform(96, 3)
    A[:, 40] = 0.0
    LUo, ipo, info_o, _ = oracle.getrf(A, 32, oracle.FULL)
    rc, LU, ip, rep = gpu_getrf(A, 32, oracle.FULL)
    assert info_o == 41 and rc == 41 and rep["info"] == 41
    assert np.array_equal(ip, ipo)


@pytest.mark.parametrize("n", [8192, 16384])
def test_full_size_sampled(n):
    nb = 256
    Ad = W.uniform_torch(n, seed=1001 + n, device=DEV)
    A0 = Ad.clone()
    faults = W.fault_schedule(n, nb, "lu", seed=3000 + n)
    rc, ipiv, rep = abft.getrf(Ad, nb, abft.FULL, faults=faults)
    torch.cuda.synchronize()
    assert rc == 0
    assert events(rep) == sorted((f[0], 0, f[2], f[3]) for f in faults)
    assert rep["max_ratio"] < 1e-1
    perm = np.arange(n)
    for j, p in enumerate(ipiv.cpu().numpy()):
        perm[[j, p]] = perm[[p, j]]
    r = W.rng(11)
    ii = r.integers(0, n, 200); jj = r.integers(0, n, 200)
    LU = Ad
    rows = LU[torch.as_tensor(ii, device=DEV)].cpu().numpy()
    cols = LU[:, torch.as_tensor(jj, device=DEV)].T.cpu().numpy()
    PA = A0[torch.as_tensor(perm[ii], device=DEV), torch.as_tensor(jj, device=DEV)].cpu().numpy()
    recon = np.empty(200)
    for t in range(200):
        i, j = ii[t], jj[t]
        l = rows[t].copy(); l[i] = 1.0; l[i + 1:] = 0.0
        u = cols[t].copy(); u[j + 1:] = 0.0
        recon[t] = float(np.dot(l[:min(i, j) + 1], u[:min(i, j) + 1]))
    assert np.abs(recon - PA).max() <= 1e-12 * n


@pytest.mark.parametrize("n,nb", [(64, 32), (96, 32)])
def test_growth_beyond_fixed_point_bound(n, nb):
    # Wilkinson's growth example: unit diagonal, -1 below it, ones in the last
    # column.  Partial pivoting keeps the diagonal (ties go to the first row),
    # the last column doubles at every step (u_in = 2^i), and every entry of
    # the factors is a power of two or +-1, so both sides are exact.  The
    # entries soon exceed the fixed-point bound of the verify sums (16 times
    # the largest |a| and |u| seen so far), so those tiles are summed in FP64.
    A = np.tril(-np.ones((n, n)), -1) + np.eye(n)
    A[:, -1] = 1.0
    for mode in (oracle.SINGLE, oracle.FULL):
        LUo, ipo, info_o, rep_o = oracle.getrf(A, nb, mode)
        rc, LU, ip, rep = gpu_getrf(A, nb, mode)
        assert rc == 0 and info_o == 0
        assert np.array_equal(ip, ipo) and np.array_equal(LU, LUo)
        assert LU[-1, -1] == 2.0 ** (n - 1)
        assert rep["detected"] == 0
        # an error in the growing last column, where the tile's sums run in FP64
        f = [(0, oracle.F_MEMORY, 50, n - 1, 2.0 ** 48)]
        LUo, ipo, _, rep_o = oracle.getrf(A, nb, mode, f)
        rc, LU, ip, rep = gpu_getrf(A, nb, mode, f)
        assert events(rep) == events(rep_o)
        for key in ("detected", "corrected", "uncorrectable"):
            assert rep[key] == rep_o[key], key
        if rep_o["uncorrectable"] == 0:
            assert np.array_equal(ip, ipo) and np.array_equal(LU, LUo)
