"""GPU parity of the ABFT LU whose trailing update (and its checksum
borders) runs FP64-accurate on the BF16 tensor cores (abft_getrf with
ABFT_F64_EMU) against the CPU FP64 oracle: the same pivots, factors to FP64
rounding, bit-exact event lists, exact results on dyadic data."""
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
    rc, ipiv, rep = abft.getrf(T, nb, mode, dtype=abft.F64_EMU, faults=faults)
    torch.cuda.synchronize()
    return rc, T.cpu().numpy(), ipiv.cpu().numpy(), rep


def events(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("n,nb", [(100, 32), (257, 64), (300, 128), (513, 256), (1024, 256)])
def test_parity_clean(n, nb, mode):
    A = W.uniform(n, seed=400 + n)
    LUo, ipo, info_o, rep_o = oracle.getrf(A, nb, mode)
    rc, LU, ip, rep = gpu_getrf(A, nb, mode)
    assert rc == 0 and info_o == 0
    assert np.array_equal(ip, ipo)
    assert np.abs(LU - LUo).max() <= 1e-12 * max(1.0, np.abs(LUo).max())
    P, L, U = oracle.unpack_lu(LU, ip)
    assert np.linalg.norm(P @ A - L @ U) / np.linalg.norm(A) <= 1e-14
    assert rep["detected"] == 0
    if mode != oracle.NONE:
        assert rep["max_ratio"] < 1e-2


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.FULL])
def test_exact_plu(mode):
    n, nb = 128, 32
    A, P0, L0, U0 = W.lu_exact(n, 5)
    rc, LU, ip, rep = gpu_getrf(A, nb, mode)
    P, L, U = oracle.unpack_lu(LU, ip)
    assert rc == 0 and np.array_equal(P, P0.T) and np.array_equal(L, L0) and np.array_equal(U, U0)
    if mode != oracle.NONE:
        f = [(1, oracle.F_MEMORY, 100, 70, 512.0), (0, oracle.F_PANEL, 10, 50, 4.0),
             (2, oracle.F_COMPUTE, 120, 110, 64.0)]
        rc, LU, ip, rep = gpu_getrf(A, nb, mode, f)
        P, L, U = oracle.unpack_lu(LU, ip)
        assert np.array_equal(L, L0) and np.array_equal(U, U0)
        _, _, _, rep_o = oracle.getrf(A, nb, mode, f)
        assert events(rep) == events(rep_o) and rep["corrected"] == 3


@pytest.mark.parametrize("mode", [oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("faults", [
    [(1, oracle.F_MEMORY, 100, 70, 1e3), (2, oracle.F_PANEL, 70, 120, 4.0)],
    [(1, oracle.F_COMPUTE, 150, 180, -20.0)],
    [(0, oracle.F_COL1D, 40, 50, 3.0)],
    [(0, oracle.F_ROW1D, 40, 50, 3.0)],
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
    _, ipo, info_o, _ = oracle.getrf(A, 32, oracle.FULL)
    rc, LU, ip, rep = gpu_getrf(A, 32, oracle.FULL)
    assert info_o == 41 and rc == 41 and rep["info"] == 41
    assert np.array_equal(ip, ipo)


def test_block_wider_than_256_is_unsupported():
    A = torch.eye(1024, dtype=torch.float64, device=DEV)
    with pytest.raises(abft.AbftError):
        abft.getrf(A, 512, abft.FULL, dtype=abft.F64_EMU)


def test_full_size_sampled():
    n, nb = 8192, 256
    Ad = W.uniform_torch(n, seed=1001 + n, device=DEV)
    A0 = Ad.clone()
    faults = W.fault_schedule(n, nb, "lu", seed=3000 + n)
    rc, ipiv, rep = abft.getrf(Ad, nb, abft.FULL, dtype=abft.F64_EMU, faults=faults)
    torch.cuda.synchronize()
    assert rc == 0
    assert events(rep) == sorted((f[0], 0, f[2], f[3]) for f in faults)
    perm = np.arange(n)
    for j, p in enumerate(ipiv.cpu().numpy()):
        perm[[j, p]] = perm[[p, j]]
    r = W.rng(11)
    ii = r.integers(0, n, 200); jj = r.integers(0, n, 200)
    rows = Ad[torch.as_tensor(ii, device=DEV)].cpu().numpy()
    cols = Ad[:, torch.as_tensor(jj, device=DEV)].T.cpu().numpy()
    PA = A0[torch.as_tensor(perm[ii], device=DEV), torch.as_tensor(jj, device=DEV)].cpu().numpy()
    recon = np.empty(200)
    for t in range(200):
        i, j = ii[t], jj[t]
        l = rows[t].copy(); l[i] = 1.0; l[i + 1:] = 0.0
        u = cols[t].copy(); u[j + 1:] = 0.0
        recon[t] = float(np.dot(l[:min(i, j) + 1], u[:min(i, j) + 1]))
    assert np.abs(recon - PA).max() <= 1e-12 * n
