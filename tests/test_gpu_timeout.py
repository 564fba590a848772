"""The give-up path of the bounded waits (the failure path of every
persistent and cooperative kernel), made to run out on purpose-built cases
with a flag that nothing sets: the call returns ABFT_ERR_TIMEOUT with the
status block's error code, the CTA that waited frees its tensor memory, and
the GPU stays usable -- the next factorizations on it (tensor-core mixed
form; cooperative LU panel) still match the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_waits_give_up_and_the_gpu_stays_usable():
    for _ in range(3):   # TMEM freed each time: the next allocation succeeds
        assert abft.wait_selftest(0, 1_000_000) == (abft.ERR_TIMEOUT, 1)
        assert abft.wait_selftest(1, 1_000_000) == (abft.ERR_TIMEOUT, 2)
    assert abft.wait_selftest(2, 1_000_000_000) == (0, 0)
    assert abft.wait_selftest(3, 1_000_000_000) == (0, 0)
    torch.cuda.synchronize()
    # tensor-core update (TMEM, mbarrier waits) after the timeouts
    n, nb = 640, 128
    A = W.spd_mmt(n, seed=900)
    T = torch.from_numpy(A).to(DEV)
    rc, rep = abft.potrf(T, nb, abft.FULL, dtype=abft.MIXED_BF16)
    torch.cuda.synchronize()
    Lo, info, rep_o = oracle.potrf_mixed(A, nb, oracle.FULL, True)
    L = np.tril(T.cpu().numpy())
    assert rc == 0 and info == 0 and rep["detected"] == 0
    assert np.array_equal(L[nb:, :nb], np.tril(Lo)[nb:, :nb])
    # cooperative LU panel (grid barriers) after the timeouts
    Au = W.uniform(512, seed=901)
    Tu = torch.from_numpy(Au).to(DEV)
    rc, ipiv, rep = abft.getrf(Tu, 128, abft.FULL)
    torch.cuda.synchronize()
    LUo, ipo, info, _ = oracle.getrf(Au, 128, oracle.FULL)
    assert rc == 0 and np.array_equal(ipiv.cpu().numpy(), ipo)
    assert np.abs(Tu.cpu().numpy() - LUo).max() <= 1e-12 * np.abs(LUo).max()
