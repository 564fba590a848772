"""GPU parity of the ABFT Householder QR whose block-reflector update runs
FP64-accurate on the BF16 tensor cores (abft_geqrf with ABFT_F64_EMU through
the C ABI) against the FP64 CPU oracle: packed R / reflectors, tau, event
lists (Sec. 2.1, 3.1.2).  The reduction V^T [C, r] over the panel rows runs in
256-row pieces: the sizes below give one, several and a ragged last piece."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U = 2.0 ** -53


def gpu_geqrf(A, nb, mode, faults=()):
    T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    rc, tau, rep = abft.geqrf(T, nb, mode, dtype=abft.F64_EMU, faults=faults)
    torch.cuda.synchronize()
    return rc, T.cpu().numpy(), tau.cpu().numpy(), rep


def events(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("n,nb", [(1, 32), (31, 32), (100, 32), (257, 64), (300, 128),
                                  (513, 256), (700, 128), (1100, 256)])
def test_parity_clean(n, nb, mode):
    A = W.uniform(n, seed=300 + n)
    QRo, tauo, _, rep_o = oracle.geqrf(A, nb, mode)
    rc, QR, tau, rep = gpu_geqrf(A, nb, mode)
    assert rc == 0
    scale = max(1.0, np.abs(QRo).max())
    assert np.abs(QR - QRo).max() <= 1e-11 * scale
    assert np.abs(tau - tauo).max() <= 1e-12
    Q = oracle.form_q(QR, tau)
    assert np.linalg.norm(A - Q @ np.triu(QR)) / np.linalg.norm(A) <= 10 * n * U
    assert rep["detected"] == 0
    if mode != oracle.NONE:
        assert rep["max_ratio"] < 1e-2
        assert abs(rep["tau"] - rep_o["tau"]) <= 1e-12 * rep_o["tau"]


@pytest.mark.parametrize("mode", [oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("faults", [
    [(1, oracle.F_MEMORY, 40, 70, 1e3), (2, oracle.F_COMPUTE, 64, 100, -3.0)],
    [(1, oracle.F_ROW1D, 40, 70, 2.0)],
    [(0, oracle.F_COL1D, 40, 50, 3.0)],
    [(1, oracle.F_MEMORY, 130, 100, 5.0), (1, oracle.F_MEMORY, 140, 110, 6.0)],
    [(0, oracle.F_COMPUTE, 300, 200, 7.0)],
])
def test_error_classes_match_oracle(mode, faults):
    n, nb = 384, 32
    A = W.uniform(n, 33)
    QRo, tauo, _, rep_o = oracle.geqrf(A, nb, mode, faults)
    rc, QR, tau, rep = gpu_geqrf(A, nb, mode, faults)
    for key in ("detected", "corrected", "uncorrectable", "checksum_repaired"):
        assert rep[key] == rep_o[key], key
    if len(rep_o["loc"]) < 64:
        assert events(rep) == events(rep_o)
    if rep_o["uncorrectable"] == 0:
        assert np.abs(QR - QRo).max() <= 1e-10 and np.abs(tau - tauo).max() <= 1e-12


def test_block_too_wide_refused():
    A = torch.zeros(600, 600, dtype=torch.float64, device=DEV)
    with pytest.raises(abft.AbftError):
        abft.geqrf(A, 512, abft.FULL, dtype=abft.F64_EMU)


def test_matches_fp64_path():
    """The tensor-core update and the FP64 one give the same factorization to
    FP64 accuracy (the same panel arithmetic, updates that differ by rounding)."""
    n, nb = 1536, 256
    Ad = W.uniform_torch(n, seed=77, device=DEV)
    A1 = Ad.clone(); A2 = Ad.clone()
    rc1, t1, _ = abft.geqrf(A1, nb, abft.FULL)
    rc2, t2, _ = abft.geqrf(A2, nb, abft.FULL, dtype=abft.F64_EMU)
    torch.cuda.synchronize()
    assert rc1 == 0 and rc2 == 0
    assert float((A1 - A2).abs().max()) <= 1e-11 * float(A1.abs().max())
    assert float((t1 - t2).abs().max()) <= 1e-12


@pytest.mark.parametrize("n", [8192, 16384])
def test_full_size_sampled(n):
    """Full size: faults located at their injected positions; sampled entries of
    R^T R equal those of A^T A (one FP64 dot product per entry on the CPU)."""
    nb = 256
    Ad = W.uniform_torch(n, seed=1002 + n, device=DEV)
    r = W.rng(13)
    ii = r.integers(0, n, 100); jj = r.integers(0, n, 100)
    Ai = Ad[:, torch.as_tensor(ii, device=DEV)].T.cpu().numpy()
    Aj = Ad[:, torch.as_tensor(jj, device=DEV)].T.cpu().numpy()
    ata = np.einsum("ij,ij->i", Ai, Aj)
    faults = W.fault_schedule(n, nb, "qr", seed=4000 + n)
    rc, tau, rep = abft.geqrf(Ad, nb, abft.FULL, dtype=abft.F64_EMU, faults=faults)
    torch.cuda.synchronize()
    assert rc == 0
    assert events(rep) == sorted((f[0], 0, f[2], f[3]) for f in faults)
    assert rep["max_ratio"] < 1e-1
    R = torch.triu(Ad)
    Ri = R[:, torch.as_tensor(ii, device=DEV)].T.cpu().numpy()
    Rj = R[:, torch.as_tensor(jj, device=DEV)].T.cpu().numpy()
    rtr = np.einsum("ij,ij->i", Ri, Rj)
    assert np.abs(rtr - ata).max() <= 1e-12 * n
