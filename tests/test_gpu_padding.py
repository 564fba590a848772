"""LU and QR (abft_getrf / abft_geqrf through the C ABI) on a matrix stored
with lda > n: the columns n .. lda-1 of every row are filled with NaN before
the call and must still be NaN afterwards (no kernel reads or writes past
column n), while the factors match the CPU oracle.  FP64 and the
FP64-accurate tensor-core update; an odd lda, so rows start unaligned."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def padded(A, ld):
    n = A.shape[0]
    buf = torch.full((n, ld), float("nan"), dtype=torch.float64, device=DEV)
    T = buf[:, :n]
    T.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return buf, T


@pytest.mark.parametrize("dtype", [abft.F64, abft.F64_EMU])
def test_getrf_padding_untouched(dtype):
    n, nb = 300, 64
    A = W.uniform(n, seed=411)
    buf, T = padded(A, n + 13)
    rc, ipiv, rep = abft.getrf(T, nb, abft.FULL, dtype=dtype)
    torch.cuda.synchronize()
    out = buf.cpu().numpy()
    assert rc == 0 and rep["detected"] == 0
    assert np.isnan(out[:, n:]).all()
    LUo, ipo, _, _ = oracle.getrf(A, nb, oracle.FULL)
    assert np.array_equal(ipiv.cpu().numpy(), ipo)
    assert np.abs(out[:, :n] - LUo).max() <= 1e-12 * max(1.0, np.abs(LUo).max())


@pytest.mark.parametrize("dtype", [abft.F64, abft.F64_EMU])
def test_geqrf_padding_untouched(dtype):
    n, nb = 300, 64
    A = W.uniform(n, seed=412)
    buf, T = padded(A, n + 13)
    rc, tau, rep = abft.geqrf(T, nb, abft.FULL, dtype=dtype)
    torch.cuda.synchronize()
    out = buf.cpu().numpy()
    assert rc == 0 and rep["detected"] == 0
    assert np.isnan(out[:, n:]).all()
    QRo, tauo, _, _ = oracle.geqrf(A, nb, oracle.FULL)
    assert np.abs(out[:, :n] - QRo).max() <= 1e-11 * max(1.0, np.abs(QRo).max())
    assert np.abs(tau.cpu().numpy() - tauo).max() <= 1e-12
