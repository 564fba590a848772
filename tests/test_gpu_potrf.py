"""GPU parity of the ABFT Cholesky (abft_potrf through the C ABI) against the
CPU oracle: same seeded inputs, element-by-element factors, bit-exact event
lists (step, kind, row, col), and the paper's error classes (Sec. 3.1.2)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
DEV = "cuda:0"


def gpu_potrf(A, nb, mode, faults=(), lda=None, poison_upper=False):
    n = A.shape[0]
    ld = lda or max(1, n)
    buf = torch.full((max(n, 1), ld), float("nan"), dtype=torch.float64, device=DEV)
    T = buf[:n, :n]
    if n:
        Ah = torch.from_numpy(np.ascontiguousarray(A))
        if poison_upper:
            Ah = torch.tril(Ah) + torch.triu(torch.full_like(Ah, float("nan")), 1)
        T.copy_(Ah)
    rc, rep = abft.potrf(T, nb, mode, faults=faults)
    torch.cuda.synchronize()
    return rc, rep, buf.cpu().numpy()


def events(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


def backward_err(L, A):
    return np.linalg.norm(L @ L.T - A) / np.linalg.norm(A)


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("n,nb", [(1, 32), (31, 32), (100, 32), (128, 64), (257, 64), (300, 128),
                                  (513, 256), (700, 512)])
def test_parity_clean(n, nb, mode):
    A = W.spd_mmt(n, seed=100 + n)
    Lo, info_o, rep_o = oracle.potrf(A, nb, mode)
    rc, rep, out = gpu_potrf(A, nb, mode)
    assert rc == 0 and info_o == 0
    L = np.tril(out[:n, :n])
    assert np.abs(L - np.tril(Lo)).max() <= 1e-13 * max(1.0, np.abs(Lo).max())
    assert backward_err(L, A) <= 1e-13
    assert rep["detected"] == 0 and rep_o["detected"] == 0
    if mode != oracle.NONE:
        assert rep["tau"] == rep_o["tau"]          # same threshold, bit for bit
        assert rep["max_ratio"] < 1e-2


def test_upper_triangle_and_padding_untouched():
    n, nb, ld = 200, 64, 213
    A = W.spd_mmt(n, seed=5)
    rc, rep, out = gpu_potrf(A, nb, oracle.FULL, lda=ld, poison_upper=True)
    assert rc == 0
    assert np.isnan(out[:n, :n][np.triu_indices(n, 1)]).all()
    assert np.isnan(out[:n, n:]).all()
    Lo, _, _ = oracle.potrf(A, nb, oracle.FULL)
    assert np.abs(np.tril(out[:n, :n]) - np.tril(Lo)).max() <= 1e-13


@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
def test_integer_exact(mode):
    n, nb = 128, 32
    L0 = W.integer_l0(n, 3)
    A = L0 @ L0.T
    rc, rep, out = gpu_potrf(A, nb, mode)
    assert rc == 0 and np.array_equal(np.tril(out[:n, :n]), L0)
    if mode != oracle.NONE:
        f = [(0, oracle.F_MEMORY, 100, 40, 1000.0), (0, oracle.F_PANEL, 70, 20, 7.0),
             (0, oracle.F_COMPUTE, 90, 70, -64.0)]
        rc, rep, out = gpu_potrf(A, nb, mode, f)
        assert rc == 0 and np.array_equal(np.tril(out[:n, :n]), L0)
        _, _, rep_o = oracle.potrf(A, nb, mode, f)
        assert events(rep) == events(rep_o)
        assert [e[4] for e in rep["loc"]] == [e[4] for e in rep_o["loc"]]


def test_config_n1024_fault_step3():
    """FP64 ABFT Cholesky n = 1024, block 128, A = M M^T / n + I, one seeded
    +1e3 single-element corruption in the trailing update of step 3."""
    n, nb = 1024, 128
    A = W.spd_mmt(n, seed=1000)
    r = W.rng(3000)
    row = int(r.integers(4 * nb, n)); col = int(r.integers(4 * nb, row + 1))
    if col // nb > row // nb:
        row, col = col, row
    for kind in (oracle.F_MEMORY, oracle.F_COMPUTE):
        f = [(3, kind, row, col, 1e3)]
        Lo, _, rep_o = oracle.potrf(A, nb, oracle.FULL, f)
        rc, rep, out = gpu_potrf(A, nb, oracle.FULL, f)
        assert rc == 0
        assert events(rep) == events(rep_o) == [(3, oracle.E_0D, row, col)]
        assert abs(rep["loc"][0][4] - 1e3) < 1e-9
        L = np.tril(out[:n, :n])
        assert backward_err(L, A) <= 1e-13
        assert np.abs(L - np.tril(Lo)).max() <= 1e-12


@pytest.mark.parametrize("mode", [oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("faults", [
    [(1, oracle.F_ROW1D, 140, 100, 50.0)],
    [(1, oracle.F_COL1D, 130, 70, 50.0)],
    [(1, oracle.F_MEMORY, 130, 100, 5.0), (1, oracle.F_MEMORY, 140, 110, 6.0)],
    [(1, oracle.F_PANEL, 130, 50, 1e3)],
    [(0, 0, 40, 35, 1e3), (0, 0, 100, 33, -2e2), (0, 1, 190, 180, 3.0), (3, 0, 170, 130, 1e3)],
])
def test_error_classes_match_oracle(mode, faults):
    n, nb = 192, 32
    A = W.spd_mmt(n, 13)
    Lo, info_o, rep_o = oracle.potrf(A, nb, mode, faults)
    rc, rep, out = gpu_potrf(A, nb, mode, faults)
    assert rep["info"] == info_o
    for key in ("detected", "corrected", "uncorrectable", "checksum_repaired"):
        assert rep[key] == rep_o[key], key
    if len(rep_o["loc"]) < 64:       # beyond 64 events the kept subset is unspecified
        assert events(rep) == events(rep_o)
    if info_o == 0 and rep_o["uncorrectable"] == 0:
        assert np.abs(np.tril(out[:n, :n]) - np.tril(Lo)).max() <= 1e-10


def test_not_spd_info():
    A = W.spd_mmt(300, 3)
    A[217, 217] = -5.0
    _, info_o, _ = oracle.potrf(A, 64, oracle.FULL)
    rc, rep, _ = gpu_potrf(A, 64, oracle.FULL)
    assert rc == info_o == 218 and rep["info"] == 218


@pytest.mark.parametrize("dtype", [abft.F64, abft.MIXED_BF16, abft.F64_EMU])
@pytest.mark.parametrize("pos", [0, 31, 32, 255, 256, 287, 288, 319, 511])
def test_not_spd_info_at_tile_boundaries(dtype, pos):
    """The diagonal block is factored in 32 x 32 tiles, each with a one-pivot
    look-ahead (the next pivot's reciprocal is formed while the current one's
    update runs): a negative pivot at the first or last pivot of a tile, of a
    block or of the matrix is reported at its own index (the oracle pins it,
    since d_pos = A[pos, pos] - |L[pos, :pos]|^2 < 0 and the earlier pivots
    are untouched), in every form of the trailing update."""
    n, nb = 512, 256
    A = W.spd_mmt(n, 7)
    A[pos, pos] = -5.0
    _, info_o, _ = oracle.potrf(A, nb, oracle.FULL)
    assert info_o == pos + 1
    T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    rc, rep = abft.potrf(T, nb, abft.FULL, dtype=dtype)
    torch.cuda.synchronize()
    assert rc == info_o and rep["info"] == info_o


def test_invalid_arguments():
    T = torch.eye(64, dtype=torch.float64, device=DEV)
    with pytest.raises(abft.AbftError):
        abft.potrf(T, 48)                                          # nb not a multiple of 32
    with pytest.raises(abft.AbftError):
        abft.potrf(T, 32, faults=[(0, 0, 5, 40, 1.0)])            # fault above the diagonal
    with pytest.raises(abft.AbftError):
        abft.potrf(T, 32, faults=[(1, 0, 60, 60, 1.0)])           # last step has no TMU


@pytest.mark.parametrize("n", [8192, 16384])
def test_full_size_sampled(n):
    """Full size, block 256, faults at 1 per 10 steps: every fault is located at
    its injected position; sampled entries of L L^T match A (oracle-style dot
    products in FP64 on the CPU, one entry at a time)."""
    nb = 256
    Ad = W.spd_mmt_torch(n, seed=1000 + n, device=DEV)
    A_lower_samples = None
    faults = W.fault_schedule(n, nb, "cholesky", seed=2000 + n)
    r = W.rng(7)
    ii = r.integers(0, n, 200); jj = r.integers(0, n, 200)
    ii, jj = np.maximum(ii, jj), np.minimum(ii, jj)
    A_lower_samples = Ad[torch.as_tensor(ii, device=DEV), torch.as_tensor(jj, device=DEV)].cpu().numpy()
    rc, rep = abft.potrf(Ad, nb, abft.FULL, faults=faults)
    torch.cuda.synchronize()
    assert rc == 0
    assert events(rep) == sorted((f[0], 0, f[2], f[3]) for f in faults)
    assert rep["max_ratio"] < 1e-1
    L = torch.tril(Ad)
    Li = L[torch.as_tensor(ii, device=DEV)].cpu().numpy()
    Lj = L[torch.as_tensor(jj, device=DEV)].cpu().numpy()
    recon = np.einsum("ij,ij->i", Li, Lj)
    assert np.abs(recon - A_lower_samples).max() <= 1e-13 * n


def test_n4096_every_entry_vs_oracle():
    """n = 4096, block 256, faults at 1 per 10 steps: the whole factor, not a
    sample, against the oracle's, for the FP64 update and for the FP64-accurate
    tensor-core update (the tile counts of the full-size runs: 16 block columns,
    every look-ahead split); events equal to the oracle's."""
    n, nb = 4096, 256
    A = W.spd_mmt(n, seed=1000 + n)
    faults = W.fault_schedule(n, nb, "cholesky", seed=2000 + n)
    Lo, info_o, rep_o = oracle.potrf(A, nb, oracle.FULL, faults)
    Lo = np.tril(Lo)
    for dt in (abft.F64, abft.F64_EMU):
        T = torch.from_numpy(A).to(DEV)
        rc, rep = abft.potrf(T, nb, abft.FULL, dtype=dt, faults=faults)
        torch.cuda.synchronize()
        assert rc == 0 and info_o == 0
        assert events(rep) == events(rep_o)
        assert np.abs(np.tril(T.cpu().numpy()) - Lo).max() <= 1e-12 * np.abs(Lo).max()


@pytest.mark.parametrize("mode", [oracle.SINGLE, oracle.FULL])
def test_zero_and_subnormal_entries(mode):
    # A block-diagonal SPD matrix (exact zeros between the blocks) with subnormal
    # couplings in some entries: the verify's fixed-point conversion reads zeros
    # and subnormals below one unit of its bound; the sums, the (absent) events
    # and the factor must agree with the oracle, and an error is still located.
    n, nb = 256, 64
    r = W.rng(77)
    A = np.zeros((n, n))
    for b in range(0, n, 32):
        M = r.standard_normal((32, 32))
        A[b:b + 32, b:b + 32] = M @ M.T / 32 + np.eye(32)
    idx = r.integers(0, n, size=(40, 2))
    for i, j in idx:
        if i != j:
            A[i, j] = A[j, i] = 3e-310 * (1 + (i % 3))
    assert np.all(np.linalg.eigvalsh(A) > 0)
    Lo, info_o, rep_o = oracle.potrf(A, nb, mode)
    rc, rep, L = gpu_potrf(A, nb, mode)
    assert rc == 0 and info_o == 0 and rep["detected"] == 0 and rep_o["detected"] == 0
    assert np.abs(np.tril(L) - np.tril(Lo)).max() <= 1e-13
    f = [(1, oracle.F_MEMORY, 200, 150, 1.5)]
    _, _, rep_o = oracle.potrf(A, nb, mode, f)
    rc, rep, L = gpu_potrf(A, nb, mode, f)
    assert events(rep) == events(rep_o) and rep["corrected"] == rep_o["corrected"] == 1
