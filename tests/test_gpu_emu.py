"""GPU parity of the FP64-accurate trailing update on the BF16 tensor cores
(abft_potrf with ABFT_F64_EMU) against the CPU FP64 oracle: factors to FP64
rounding, bit-exact event lists, and exact results on integer data."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def run(A, nb, mode, faults=()):
    T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    rc, rep = abft.potrf(T, nb, mode, dtype=abft.F64_EMU, faults=faults, check=False)
    torch.cuda.synchronize()
    return rc, rep, np.tril(T.cpu().numpy())


def events(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("n,nb", [(256, 128), (700, 128), (1024, 256), (1500, 256), (2048, 256)])
def test_parity_clean(n, nb, mode):
    A = W.spd_mmt(n, seed=300 + n)
    Lo, info_o, rep_o = oracle.potrf(A, nb, mode)
    rc, rep, L = run(A, nb, mode)
    assert rc == 0 and info_o == 0 and rep["detected"] == 0
    Lo = np.tril(Lo)
    assert np.abs(L - Lo).max() <= 1e-12 * np.abs(Lo).max()
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) <= 1e-15
    if mode != oracle.NONE:
        assert rep["tau"] == rep_o["tau"] and rep["max_ratio"] < 1e-2


@pytest.mark.parametrize("mode", [oracle.SINGLE, oracle.FULL])
def test_faults_located_like_the_oracle(mode):
    n, nb = 2048, 256
    A = W.spd_mmt(n, seed=31)
    # 1D errors of 10 and 8 elements, so that every event fits the report
    faults = [(0, abft.F_MEMORY, 700, 300, 1e3), (2, abft.F_COMPUTE, 1500, 900, -3e2),
              (3, abft.F_ROW1D, 1900, 1270, 2e2), (4, abft.F_PANEL, 1800, 1100, 50.0)]
    if mode == oracle.FULL:
        faults.append((5, abft.F_COL1D, 2040, 1700, 7e2))
    Lo, info_o, rep_o = oracle.potrf(A, nb, mode, faults)
    rc, rep, L = run(A, nb, mode, faults)
    assert info_o == 0 and rc == 0 and rep_o["uncorrectable"] == 0
    assert events(rep) == [(e[0], e[1], e[2], e[3]) for e in rep_o["loc"]]
    assert np.abs(L - np.tril(Lo)).max() <= 1e-10 * np.abs(Lo).max()


def test_integer_exact():
    """Integer factors with power-of-two pivots: every slice product and the
    integer recombination are exact, so the factor is recovered bit for bit."""
    n, nb = 512, 128
    L0 = W.integer_l0(n, 3)
    A = L0 @ L0.T
    rc, rep, L = run(A, nb, oracle.FULL)
    assert rc == 0 and rep["detected"] == 0
    assert np.array_equal(L, L0)


def test_non_spd_reports_info():
    n, nb = 512, 128
    A = W.spd_mmt(n, seed=5)
    A[300, 300] = -1.0
    Lo, info_o, _ = oracle.potrf(A, nb, oracle.FULL)
    rc, rep, L = run(A, nb, oracle.FULL)
    assert rc == info_o > 0


def test_unsupported_block_size():
    A = torch.eye(512, dtype=torch.float64, device=DEV)
    with pytest.raises(abft.AbftError):
        abft.potrf(A, 512, abft.FULL, dtype=abft.F64_EMU)
