"""Pins of the oracle's mixed-precision form (16-bit quantized trailing update
with FP32 accumulation, FP32 panel solve, abs-checksum thresholds), each
against something other than the oracle itself: a hand-worked quantization,
exact enumeration of the 16-bit formats, numpy's FP16 conversion (a library
special case), exact integer and dyadic cases, LAPACK, and a float32
simulation of the accumulation that the thresholds must cover."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_2301_03166_b300 import workloads as W
from tests.golden.read import load

U32 = 2.0 ** -24


# ------------------------------------------------------------ quantization
@pytest.mark.parametrize("bf16,tag", [(True, "BF16"), (False, "FP16")])
def test_quantize_golden_2x2(bf16, tag):
    g = load("mixed_quant_2x2.txt")
    s, bits, q = oracle.quantize(g["P"], bf16)
    assert s == g["SIGMA_" + tag][0][0]
    assert np.array_equal(q, g["Q_" + tag])
    assert np.array_equal(bits, g["CODE_" + tag].astype(np.uint16))


def test_sigma_power_of_two_maximum():
    """A tile maximum that is an exact power of two maps to 2^e_t exactly;
    one ulp above it moves to the next power."""
    assert oracle.tile_sigma(0.5, True) == 0.5          # 0.5 / 0.5 = 1 = 2^0
    assert oracle.tile_sigma(0.5, False) == 2.0 ** -15  # 0.5 / 2^-15 = 2^14
    up = np.nextafter(0.5, 1.0)
    assert oracle.tile_sigma(up, True) == 1.0
    assert oracle.tile_sigma(up, False) == 2.0 ** -14
    assert oracle.tile_sigma(3.0, True) == 4.0
    assert oracle.tile_sigma(0.0, True) == 1.0 and oracle.tile_sigma(0.0, False) == 1.0
    s, _, q = oracle.quantize(np.array([[0.5, -0.25], [0.125, 0.0]]), True)
    assert s == 0.5 and np.array_equal(q, [[1.0, -0.5], [0.25, 0.0]])


def _format(bf16):
    """All finite non-negative values of the format with their codes, decoded
    from the definition (sign, biased exponent, fraction) in exact rationals."""
    ebits, fbits = (8, 7) if bf16 else (5, 10)
    bias = (1 << (ebits - 1)) - 1
    vals = []
    for e in range((1 << ebits) - 1):
        for f in range(1 << fbits):
            if e == 0:
                v = Fraction(f, 1 << fbits) * Fraction(2) ** (1 - bias)
            else:
                v = (1 + Fraction(f, 1 << fbits)) * Fraction(2) ** (e - bias)
            vals.append((v, (e << fbits) | f))
    return vals, ebits, fbits


def _nearest(x, vals, ebits, fbits):
    """Brute-force round to nearest, ties to the even code, overflow to inf."""
    a = Fraction(abs(x))
    sign = 0x8000 if x < 0 or (x == 0 and np.signbit(x)) else 0
    lo = max((p for p in vals if p[0] <= a), key=lambda p: p[0])
    hi = [p for p in vals if p[0] >= a]
    top = vals[-1][0]
    if not hi:   # above the largest finite value: its half-way point rounds to inf (odd code)
        spacing = top - vals[-2][0]
        if a >= top + spacing / 2:
            return sign | (((1 << ebits) - 1) << fbits)
        return sign | vals[-1][1]
    hi = min(hi, key=lambda p: p[0])
    dl, dh = a - lo[0], hi[0] - a
    pick = lo if dl < dh else hi if dh < dl else (lo if lo[1] % 2 == 0 else hi)
    return sign | pick[1]


@pytest.mark.parametrize("bf16", [True, False])
def test_round16_vs_enumeration(bf16):
    vals, ebits, fbits = _format(bf16)
    r = W.rng(31 if bf16 else 32)
    xs = list(r.standard_normal(150) * 10.0 ** r.integers(-6, 4, 150))
    # exact ties between neighbours, subnormal range, the top of the range
    for i in r.integers(1, len(vals) - 1, 60):
        xs.append(float((vals[i][0] + vals[i + 1][0]) / 2))
        xs.append(-float((vals[i - 1][0] + vals[i][0]) / 2))
    sub = float(vals[1][0])
    xs += [sub * 0.5, sub * 1.5, sub * 0.49, sub * 3.0, float(vals[-1][0]) * 1.001,
           float(vals[-1][0]) * 0.9999, 0.0]
    for x in xs:
        v, code = oracle.round16(x, bf16)
        assert code == _nearest(x, vals, ebits, fbits), (x, code)


def test_fp16_vs_numpy():
    """numpy converts float64 to float16 with one rounding to nearest even."""
    r = W.rng(33)
    x = np.concatenate([r.standard_normal(4000) * 10.0 ** r.integers(-9, 5, 4000),
                        r.uniform(-1, 1, 1000) * 2.0 ** -24])
    want = x.astype(np.float16)
    for xi, wi in zip(x, want):
        v, code = oracle.round16(float(xi), False)
        assert code == int(wi.view(np.uint16)) and (v == float(wi))


# ------------------------------------------------------- the update alone
def test_syrk_mixed_dyadic_exact():
    """Entries that are exact after scaling: the scales cancel and the update
    equals C - P P^T exactly, on the lower block triangle only."""
    r = W.rng(34)
    m, k, g = 300, 64, 128
    P = r.integers(-8, 9, (m, k)) / 16.0
    C = r.integers(-50, 51, (m, m)).astype(np.float64)
    for bf16 in (True, False):
        Cn, bits, sig = oracle.syrk_mixed(P, C, g, bf16)
        full = C - P @ P.T
        mask = (np.arange(m)[None, :] // g) <= (np.arange(m)[:, None] // g)
        assert np.array_equal(Cn[mask], full[mask])
        assert np.array_equal(Cn[~mask], C[~mask])
        assert all(s == (0.5 if bf16 else 2.0 ** -15) for s in sig)


@pytest.mark.parametrize("bf16,u", [(True, 2.0 ** -8), (False, 2.0 ** -11)])
def test_syrk_mixed_quantization_bound(bf16, u):
    """Random panel: each operand carries one relative rounding of at most u,
    so every entry is within (2u + u^2) (|P||P|^T) of C - P P^T, and further
    from it than FP64 rounding (the operands really are 16-bit)."""
    r = W.rng(35)
    m, k, g = 384, 128, 128
    P = r.standard_normal((m, k)) * np.exp(r.uniform(-3, 0, (m, 1)))
    C = r.standard_normal((m, m))
    Cn, _, _ = oracle.syrk_mixed(P, C, g, bf16)
    ref = C - P @ P.T
    bound = (2 * u + u * u) * (np.abs(P) @ np.abs(P).T) + 1e-13 * np.abs(C)
    mask = (np.arange(m)[None, :] // g) <= (np.arange(m)[:, None] // g)
    assert np.all(np.abs(Cn - ref)[mask] <= bound[mask])
    assert np.abs(Cn - ref)[mask].max() > 1e3 * 2.0 ** -53 * np.abs(ref).max()


# ----------------------------------------------------- the factorization
@pytest.mark.parametrize("bf16", [True, False])
@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
@pytest.mark.parametrize("n", [256, 300])
def test_potrf_mixed_integer_exact(bf16, mode, n):
    """Integer L0: the FP32 panel solve, the power-of-two scales, the 16-bit
    operands and every sum are exact, so the factor is L0 bit for bit."""
    L0 = W.integer_l0(n, 3)
    A = L0 @ L0.T
    L, info, rep = oracle.potrf_mixed(A, 128, mode, bf16)
    assert info == 0 and np.array_equal(np.tril(L), L0)
    assert rep["detected"] == 0
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))


@pytest.mark.parametrize("bf16,u", [(True, 2.0 ** -8), (False, 2.0 ** -11)])
def test_potrf_mixed_vs_lapack(bf16, u):
    n, nb = 512, 128
    A = W.spd_mmt(n, seed=36)
    L, info, rep = oracle.potrf_mixed(A, nb, oracle.FULL, bf16)
    L = np.tril(L)
    Lf = np.linalg.cholesky(A)
    assert info == 0 and rep["detected"] == 0
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) <= 4 * u
    # the first block column is the FP64 diagonal block and the FP32 panel
    # solve: FP32 values within the FP32 solve's error of the FP64 factor
    L0, _, _ = oracle.potrf(A, nb, oracle.FULL)
    assert np.abs(L[:nb, :nb] - np.tril(L0)[:nb, :nb]).max() <= 1e-14
    X = L[nb:, :nb]
    assert np.array_equal(X, X.astype(np.float32).astype(np.float64))
    Xr = sl.solve_triangular(L[:nb, :nb], A[nb:, :nb].T, lower=True).T
    assert np.abs(X - Xr).max() <= 64 * nb * U32 * np.abs(Xr).max()
    # the later columns carry the 16-bit update's error, above FP64 rounding
    assert np.abs(L - Lf)[nb:, nb:].max() > 1e-9


def _fp32_relation_gap(P, g, bf16):
    """The checksum relation of one mixed update computed as a tensor core
    would at best: every dot product of 16-bit operands summed in float32,
    p in order (each product is exact in float32).  Returns, per tile-row I
    and column j, |1^T (Lq_I Lq_J^T)_32 - (t32_I Lq_J^T)_32| and the
    abs-checksum sigma_I sigma_J (1^T |Lq_I|) |Lq_J|^T."""
    m, k = P.shape
    nt = -(-m // g)
    sig = np.zeros(nt)
    Q = np.zeros((m, k))
    for I in range(nt):
        sig[I], _, Q[I * g:(I + 1) * g] = oracle.quantize(P[I * g:(I + 1) * g], bf16)
    Q32 = Q.astype(np.float32)
    acc = np.zeros((m, m), dtype=np.float32)
    for p in range(k):
        acc = (acc + np.outer(Q32[:, p], Q32[:, p])).astype(np.float32)
    gaps, absc = [], []
    for I in range(nt):
        rows = slice(I * g, min(m, (I + 1) * g))
        t32 = Q[rows].sum(axis=0).astype(np.float32)
        ta = np.abs(Q[rows]).sum(axis=0)
        cacc = np.zeros(m, dtype=np.float32)
        for p in range(k):
            cacc = (cacc + t32[p] * Q32[:, p]).astype(np.float32)
        sc = sig[I] * sig[np.arange(m) // g]
        data = acc[rows].astype(np.float64).sum(axis=0)
        gaps.append(sc * np.abs(data - cacc.astype(np.float64)))
        absc.append(sc * (np.abs(Q) @ ta))
    return np.array(gaps), np.array(absc)


@pytest.mark.parametrize("bf16", [True, False])
def test_threshold_covers_fp32_accumulation(bf16):
    """coef |c| (coef = 4 gamma_g(2^-24)) bounds the relation gap that FP32
    accumulation leaves, with room to spare, while the FP64 threshold alone
    would flag clean columns (the abs-checksum term is needed)."""
    r = W.rng(37 if bf16 else 38)
    m, k, g = 512, 128, 128
    P = r.standard_normal((m, k)) * 0.05
    gaps, absc = _fp32_relation_gap(P, g, bf16)
    coef = oracle.mixed_coef(1.0, k)
    assert coef == 4.0 * (k * U32 / (1 - k * U32))
    assert np.max(gaps / (coef * absc)) < 0.25
    tau64 = 8 * 2.0 ** -53 * 4096 * g * 2.0
    assert gaps.max() > tau64


def test_potrf_mixed_fault_below_scalar_threshold():
    """An error of 1e-2 at n = 2048: far below the scalar FP32 bound
    8 u32 n g max a_ii (about 0.5 here) that a threshold without abs-checksums
    would need, yet flagged, located and corrected in both checksum modes."""
    n, nb = 2048, 256
    A = W.spd_mmt(n, seed=1000)
    scalar = 8 * U32 * n * nb * A.diagonal().max()
    assert scalar > 0.1
    f = (2, oracle.F_MEMORY, 1500, 1000, 1e-2)
    Lc, _, rep_c = oracle.potrf_mixed(A, nb, oracle.FULL, True)
    assert rep_c["detected"] == 0 and rep_c["tau"] < 0.5e-2
    for mode in (oracle.FULL, oracle.SINGLE):
        L, info, rep = oracle.potrf_mixed(A, nb, mode, True, faults=[f])
        assert info == 0
        assert [(e[0], e[1], e[2], e[3]) for e in rep["loc"]] == [(2, oracle.E_0D, 1500, 1000)]
        assert abs(rep["loc"][0][4] - 1e-2) < 1e-6
        assert np.abs(np.tril(L) - np.tril(Lc)).max() < 1e-12
