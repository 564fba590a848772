"""The adaptive-ABFT oracle (fault-coverage formulas, mode policy, per-step
checksum schedule) pinned against Monte Carlo simulation of the fault model,
closed forms, and the unprotected factorization of the corrupted matrix."""
import math

import numpy as np
import pytest

import oracle
from oracle import adaptive as ad
from paper_2301_03166_b300 import workloads as W


def monte_carlo(S, mu0, mu1, mu2, trials, seed):
    """Fraction of intervals in which single-side / full checksums correct every
    error: Poisson counts per type, blocks drawn uniformly."""
    r = np.random.default_rng(seed)
    k0 = r.poisson(mu0, trials)
    k1 = r.poisson(mu1, trials)
    k2 = r.poisson(mu2, trials)
    single = full = 0
    for a, b, c in zip(k0, k1, k2):
        if c:
            continue
        blocks = r.integers(0, S, a + b)
        distinct0 = len(set(blocks[:a].tolist())) == a
        distinct = len(set(blocks.tolist())) == a + b
        single += int(b == 0 and distinct0)
        full += int(distinct)
    return single / trials, full / trials


def literal_fc_single(S, mu0, mu1, mu2):
    """The formula with the product printed up to i = k (not used: pins the reading)."""
    s = 0.0
    for k in range(0, 60):
        w = math.exp(-mu0) * mu0 ** k / math.factorial(k)
        p = 1.0
        for i in range(k + 1):
            p *= (S - i) / S
        s += w * p
    return s * math.exp(-mu1 - mu2)


@pytest.mark.parametrize("S,mu0,mu1,mu2", [(4, 1.0, 0.0, 0.0), (16, 2.0, 0.5, 0.0),
                                           (9, 0.7, 0.3, 0.05), (64, 5.0, 1.0, 0.0)])
def test_fc_matches_monte_carlo(S, mu0, mu1, mu2):
    trials = 200000
    ms, mf = monte_carlo(S, mu0, mu1, mu2, trials, seed=S)
    fs, ff = ad.fc_single(S, mu0, mu1, mu2), ad.fc_full(S, mu0, mu1, mu2)
    for p, q in ((fs, ms), (ff, mf)):
        sd = math.sqrt(max(p * (1 - p), 1e-12) / trials)
        assert abs(p - q) <= 5 * sd + 1e-12, (p, q)


def test_product_reading_is_the_one_the_simulation_supports():
    S, mu0 = 4, 1.0
    ms, _ = monte_carlo(S, mu0, 0.0, 0.0, 200000, seed=7)
    lit = literal_fc_single(S, mu0, 0.0, 0.0)
    sd = math.sqrt(ms * (1 - ms) / 200000)
    assert abs(ad.fc_single(S, mu0, 0.0, 0.0) - ms) <= 5 * sd
    assert abs(lit - ms) > 20 * sd


def test_closed_forms():
    for mu0, mu1, mu2 in ((0.3, 0.0, 0.0), (1.2, 0.4, 0.1)):
        # one block: at most one error may strike
        assert ad.fc_single(1, mu0, mu1, mu2) == pytest.approx(
            math.exp(-mu0) * (1 + mu0) * math.exp(-mu1 - mu2), rel=1e-14)
        assert ad.fc_full(1, mu0, mu1, mu2) == pytest.approx(
            math.exp(-mu0 - mu1) * (1 + mu0 + mu1) * math.exp(-mu2), rel=1e-14)
        # very many blocks: only the uncorrectable types matter
        S = 10 ** 12
        assert ad.fc_single(S, mu0, mu1, mu2) == pytest.approx(math.exp(-mu1 - mu2), rel=1e-9)
        assert ad.fc_full(S, mu0, mu1, mu2) == pytest.approx(math.exp(-mu2), rel=1e-9)
    # no errors expected: full coverage
    assert ad.fc_single(256, 0.0, 0.0, 0.0) == 1.0 and ad.fc_full(256, 0.0, 0.0, 0.0) == 1.0


def test_full_equals_single_of_the_merged_process():
    """The sum of two independent Poisson counts is Poisson(mu0 + mu1), so
    FC_full(mu0, mu1) = FC_single(mu0 + mu1, 0) with the same 2D factor."""
    for S, mu0, mu1, mu2 in ((16, 2.0, 0.5, 0.1), (1024, 7.0, 3.0, 0.0), (3, 0.4, 0.9, 0.2)):
        assert ad.fc_full(S, mu0, mu1, mu2) == pytest.approx(ad.fc_single(S, mu0 + mu1, 0.0, mu2),
                                                             rel=1e-12)
        assert ad.fc_full(S, mu0, mu1, mu2) >= ad.fc_single(S, mu0, mu1, mu2)
        assert ad.fc_full(S, 0.0, mu1, mu2) == pytest.approx(ad.fc_single(S, mu1, 0.0, mu2),
                                                             rel=1e-12)


def test_policy():
    n, nb = 4096, 256
    T = [0.001 * (k + 1) for k in range(16)]
    modes, cov = ad.adaptive_modes(n, nb, (0.0, 0.0, 0.0), 0.999999, T)
    assert modes == [ad.NONE] * 16 and cov == [1.0] * 16
    # 0D errors only: single-side checksums suffice while two errors in one
    # block stay unlikely enough
    modes, cov = ad.adaptive_modes(n, nb, (1.0, 0.0, 0.0), 0.999999, T)
    assert all(m == ad.SINGLE for m in modes)
    # 1D errors need full checksums
    modes, cov = ad.adaptive_modes(n, nb, (1.0, 1e-4, 0.0), 0.999999, T)
    assert modes[0] == ad.SINGLE and modes[-1] == ad.FULL
    k = modes.index(ad.FULL)
    assert all(m == ad.FULL for m in modes[k:]) and all(c >= 0.999999 for c in cov)


def _chol_matrix(n, seed):
    return W.spd_mmt(n, seed=seed)


def test_uniform_schedule_equals_fixed_mode():
    n, nb = 256, 32
    A = _chol_matrix(n, 1)
    f = [(2, oracle.F_MEMORY, 200, 100, 1e3), (4, oracle.F_COL1D, 250, 170, 5e2)]
    for mode in (oracle.NONE, oracle.SINGLE, oracle.FULL):
        L1, i1, r1 = oracle.potrf(A.copy(), nb, mode, f)
        L2, i2, r2 = oracle.potrf_sched(A.copy(), nb, [mode] * (n // nb), f)
        assert i1 == i2 and np.array_equal(L1, L2) and r1["loc"] == r2["loc"]


def test_fault_in_unchecked_step_is_absorbed():
    """An error that strikes while no checksum is kept is not detected, and
    the result is the Cholesky factor of the matrix with that error."""
    n, nb = 256, 32
    A = _chol_matrix(n, 2)
    modes = [oracle.NONE, oracle.NONE, oracle.NONE, oracle.FULL, oracle.FULL,
             oracle.SINGLE, oracle.SINGLE, oracle.SINGLE]
    i, j, d = 230, 140, 0.25
    L, info, rep = oracle.potrf_sched(A.copy(), nb, modes, [(2, oracle.F_MEMORY, i, j, d)])
    assert info == 0 and rep["detected"] == 0
    Ae = A.copy()
    Ae[i, j] += d
    Ae[j, i] += d
    assert np.abs(np.tril(L) - np.linalg.cholesky(Ae)).max() <= 1e-12


def test_checked_steps_after_a_switch_correct_errors():
    """Checking resumes with fresh checksums (step 3), a 1D column error is
    corrected at a full step (needs the re-encoded row sums), and a 0D error
    at a single-side step after full ones."""
    n, nb = 256, 32
    A = _chol_matrix(n, 3)
    modes = [oracle.NONE, oracle.SINGLE, oracle.SINGLE, oracle.FULL, oracle.FULL,
             oracle.SINGLE, oracle.NONE, oracle.NONE]
    f = [(3, oracle.F_COL1D, 200, 170, 3e2), (5, oracle.F_MEMORY, 250, 200, 1e3)]
    L, info, rep = oracle.potrf_sched(A.copy(), nb, modes, f)
    Lc, _, _ = oracle.potrf(A.copy(), nb, oracle.NONE)
    assert info == 0 and rep["uncorrectable"] == 0
    assert {e[0] for e in rep["loc"]} == {3, 5}
    assert np.abs(np.tril(L) - np.tril(Lc)).max() <= 1e-9
