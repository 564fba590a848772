"""The mixed-precision path against the oracle's mixed form (16-bit quantized
update, FP32 panel solve, abs-checksum thresholds).

* The update alone (abft_syrk_mixed): per-tile scales and 16-bit codes equal
  the oracle's bit for bit; every updated entry is within the FP32
  accumulation bound of the oracle's (products summed in FP64); entries
  outside the lower block triangle are untouched.
* The factorization: the FP32 panel solve of the first step is bit-identical;
  the whole factor is far closer to the oracle's mixed factor than either is
  to the FP64 factor; fault events equal the oracle's bit for bit, also for
  errors far below the scalar FP32 threshold that the abs-checksums replace.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U32 = 2.0 ** -24
FMTS = [(abft.MIXED_BF16, True), (abft.MIXED_F16, False)]


def gamma(k, u):
    return k * u / (1 - k * u)


@pytest.mark.parametrize("dtype,bf16", FMTS)
@pytest.mark.parametrize("m,k,g", [(300, 64, 128), (640, 128, 128), (1000, 256, 256),
                                   (520, 512, 256)])
def test_syrk_mixed_vs_oracle(dtype, bf16, m, k, g):
    r = W.rng(m + k)
    P = r.standard_normal((m, k)) * np.exp(r.uniform(-4, 0, (m, 1)))
    if m > 2 * g:
        P[g:2 * g] = 0.0                      # an all-zero tile: sigma = 1, codes 0
    C = r.standard_normal((m, m))
    Co, bits_o, sig_o = oracle.syrk_mixed(P, C, g, bf16)
    Cd = torch.from_numpy(C).to(DEV)
    bits, sig = abft.syrk_mixed(torch.from_numpy(P).to(DEV), Cd, g, dtype)
    Cg = Cd.cpu().numpy()
    assert np.array_equal(sig, sig_o)
    assert np.array_equal(bits, bits_o)
    mask = (np.arange(m)[None, :] // g) <= (np.arange(m)[:, None] // g)
    assert np.array_equal(Cg[~mask], C[~mask])
    # |sum_32 - sum_exact| <= 2 gamma_k(u32) sum |q||q| (the 2 allows an
    # accumulation that truncates), plus the FP64 sum of the oracle and one
    # rounding of the subtraction
    Q = np.zeros((m, k))
    for I in range(-(-m // g)):
        _, _, Q[I * g:(I + 1) * g] = oracle.quantize(P[I * g:(I + 1) * g], bf16)
    sc = sig_o[np.arange(m) // g]
    absprod = np.outer(sc, sc) * (np.abs(Q) @ np.abs(Q).T)
    bound = (2 * gamma(k, U32) + gamma(k, 2.0 ** -53)) * absprod + 2.0 ** -52 * np.abs(Co)
    err = np.abs(Cg - Co)
    assert np.all(err[mask] <= bound[mask]), (err[mask] / np.maximum(bound[mask], 1e-300)).max()


def run(A, nb, mode, dtype, faults=()):
    T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    rc, rep = abft.potrf(T, nb, mode, dtype=dtype, faults=faults)
    torch.cuda.synchronize()
    return rc, np.tril(T.cpu().numpy()), rep


def ev(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


@pytest.mark.parametrize("dtype,bf16", FMTS)
@pytest.mark.parametrize("mode", [abft.SINGLE, abft.FULL])
@pytest.mark.parametrize("n,nb", [(300, 128), (640, 128), (1000, 256)])
def test_potrf_mixed_vs_oracle(dtype, bf16, mode, n, nb):
    A = W.spd_mmt(n, seed=700 + n)
    rc, L, rep = run(A, nb, mode, dtype)
    Lo, info, rep_o = oracle.potrf_mixed(A, nb, mode, bf16)
    Lo = np.tril(Lo)
    assert rc == 0 and info == 0
    assert ev(rep) == ev(rep_o) == []
    # step 0: FP64 diagonal block, then the FP32 panel solve, bit for bit
    assert np.abs(L[:nb, :nb] - Lo[:nb, :nb]).max() <= 1e-14
    assert np.array_equal(L[nb:, :nb], Lo[nb:, :nb])
    # later steps: the FP32 tensor-core sums differ from the oracle's FP64
    # sums only at the FP32 level; the 16-bit quantization itself is shared
    L64, _, _ = oracle.potrf(A, nb, oracle.FULL)
    L64 = np.tril(L64)
    # (measured: 0.01-0.05 of the quantization's own effect; FP16's effect is 8x smaller)
    assert np.linalg.norm(L - Lo) <= 0.15 * np.linalg.norm(Lo - L64)
    # thresholds: the abs-checksums agree to FP32 accumulation; clean margins
    assert abs(rep["tau"] - rep_o["tau"]) <= 1e-4 * rep_o["tau"]
    assert rep["max_ratio"] < 0.05


@pytest.mark.parametrize("dtype,bf16", FMTS)
@pytest.mark.parametrize("mode", [abft.SINGLE, abft.FULL])
def test_small_faults_located_like_the_oracle(dtype, bf16, mode):
    """Trailing-matrix errors of 1e-2 at n = 2048: below the scalar FP32 bound
    8 u32 n g max a_ii (about 0.5) by more than an order of magnitude, above
    the per-column thresholds; located, classified and corrected exactly as by
    the oracle.  (The panel check keeps the scalar bound: its error is 3.)"""
    n, nb = 2048, 256
    A = W.spd_mmt(n, seed=1000)
    assert 8 * U32 * n * nb * A.diagonal().max() > 0.2
    faults = [(2, abft.F_MEMORY, 1500, 1000, 1e-2), (4, abft.F_COMPUTE, 2000, 1300, -2e-2),
              (3, abft.F_PANEL, 1700, 800, 3.0)]
    if mode == abft.FULL:
        faults.append((5, abft.F_ROW1D, 1900, 1780, 5e-2))   # 12 entries to the tile's end
    rc, L, rep = run(A, nb, mode, dtype, faults)
    Lo, info, rep_o = oracle.potrf_mixed(A, nb, mode, bf16, faults=faults)
    assert rc == 0 and info == 0
    assert ev(rep) == ev(rep_o)
    assert len(ev(rep)) == (3 if mode == abft.SINGLE else 3 + 12)
    for e, eo in zip(rep["loc"], rep_o["loc"]):
        assert abs(e[4] - eo[4]) <= 1e-6
    assert rep["corrected"] == rep_o["corrected"] and rep["uncorrectable"] == 0
    assert rep["tau"] < 5e-3
    Lo = np.tril(Lo)
    assert np.linalg.norm(L - Lo) <= 0.3 * np.linalg.norm(Lo - np.linalg.cholesky(A))


def test_n4096_mixed_vs_oracle():
    """n = 4096, block 256 (16 block columns, the look-ahead splits of the
    full-size runs), BF16, faults at 1 per 10 steps: events equal to the mixed
    oracle's, the first panel bit for bit, the factor within the same fraction
    of the quantization's own effect as at the smaller orders."""
    n, nb = 4096, 256
    A = W.spd_mmt(n, seed=1000 + n)
    faults = W.fault_schedule(n, nb, "cholesky", seed=2000 + n)
    rc, L, rep = run(A, nb, abft.FULL, abft.MIXED_BF16, faults)
    Lo, info, rep_o = oracle.potrf_mixed(A, nb, oracle.FULL, True, faults=faults)
    Lo = np.tril(Lo)
    assert rc == 0 and info == 0
    assert ev(rep) == ev(rep_o) and len(ev(rep)) == len(faults)
    assert np.array_equal(L[nb:, :nb], Lo[nb:, :nb])
    L64 = np.linalg.cholesky(A)
    assert np.linalg.norm(L - Lo) <= 0.3 * np.linalg.norm(Lo - L64)
