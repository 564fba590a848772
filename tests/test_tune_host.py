"""Host logic of the batched autotuner, on the CPU: the size buckets the block
size is tuned per, the chooser built from a tuned table, and the packed layout
of the synthetic SPD batch it times (matrix i at offset sum_{k<i} n_k^2, row-major)."""
import numpy as np
import torch

from paper_2301_03166_b300 import tune


def test_bucket_boundaries():
    for (lo, hi), b in zip(tune.BUCKETS, range(len(tune.BUCKETS))):
        assert tune._bucket(lo) == b and tune._bucket(hi) == b
    assert tune._bucket(tune.BUCKETS[-1][1] + 1) == len(tune.BUCKETS) - 1


def test_chooser_maps_orders_to_their_bucket():
    table = {0: 32, 1: 64, 2: 32}
    nb = tune.chooser(table)
    assert [nb(n) for n in (32, 100, 127, 128, 255, 256, 512)] == [32, 32, 32, 64, 64, 32, 32]


def test_spd_batch_layout():
    sizes = np.array([3, 5, 1, 4])
    buf, s, offs = tune._spd_batch(sizes, torch.float64, "cpu", seed=5)
    assert list(offs) == [0, 9, 34, 35]
    assert buf.numel() == int((sizes ** 2).sum())
    for n, o in zip(sizes, offs):
        A = buf[o:o + n * n].reshape(n, n).numpy()
        assert np.allclose(A, A.T, rtol=0, atol=1e-12)
        np.linalg.cholesky(A)                           # raises unless SPD
        assert np.linalg.eigvalsh(A).min() >= 1.0 - 1e-12   # M M^T / n + I
