"""The synthetic inputs: the conditioned matrix for the largest orders has
the stated spectrum, is symmetric and dense, and is reproducible."""
import numpy as np
import torch

from paper_2301_03166_b300 import workloads as W


def test_butterfly_conditioned_matrix():
    n, kappa = 512, 1e6
    A = W.spd_kappa_butterfly_torch(n, kappa, seed=5, device="cpu").numpy()
    sig = kappa ** (-np.arange(n) / (n - 1))
    ev = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert np.abs(ev - sig).max() <= 1e-13
    assert np.array_equal(A, A.T)
    assert np.mean(np.abs(A) < 1e-14) == 0.0            # no structural zeros
    assert abs(A.trace() - sig.sum()) <= 1e-12 * sig.sum()
    B = W.spd_kappa_butterfly_torch(n, kappa, seed=5, device="cpu").numpy()
    assert np.array_equal(A, B)
    C = W.spd_kappa_butterfly_torch(n, kappa, seed=6, device="cpu").numpy()
    assert not np.allclose(A, C)
