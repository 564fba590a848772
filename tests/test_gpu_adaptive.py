"""GPU parity of the per-step checksum schedule (abft_potrf_sched, adaptive
ABFT) against the oracle's schedule: element-by-element factors and bit-exact
event lists, for schedules that start, stop, strengthen and weaken checking,
with errors injected at checked and unchecked steps."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N_, S_, F_ = oracle.NONE, oracle.SINGLE, oracle.FULL


def events(rep):
    return [(e[0], e[1], e[2], e[3]) for e in rep["loc"]]


def run(A, nb, modes, faults=(), dtype=abft.F64):
    T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    rc, rep = abft.potrf_sched(T, nb, modes, dtype=dtype, faults=faults)
    torch.cuda.synchronize()
    return rc, rep, np.tril(T.cpu().numpy())


SCHEDULES = [
    [N_, N_, S_, S_, F_, F_, S_, N_],
    [F_, N_, F_, S_, N_, S_, F_, F_],
    [S_, F_, N_, N_, N_, F_, F_, S_],
]


@pytest.mark.parametrize("modes", SCHEDULES)
def test_schedule_parity_with_faults(modes):
    n, nb = 1024, 128
    A = W.spd_mmt(n, seed=21)
    # deltas far above the threshold (~1e-9 here) but small enough that an
    # error absorbed at an unchecked step keeps A positive definite (its
    # eigenvalues are >= 1)
    faults = [(1, abft.F_MEMORY, 700, 300, 0.05),
              (3, abft.F_COL1D, 1010, 600, 0.02),      # 1D errors of 14 and 16 elements:
              (4, abft.F_MEMORY, 1000, 800, -0.04),    # every event fits the report
              (5, abft.F_ROW1D, 950, 880, 0.03)]
    Lo, info_o, rep_o = oracle.potrf_sched(A.copy(), nb, modes, faults)
    rc, rep, L = run(A, nb, modes, faults)
    # a 1D column error at a single-side step cannot be located: reported as
    # uncorrectable by both
    assert info_o == 0 and rc == (abft.ERR_UNCORRECTABLE if rep_o["uncorrectable"] else 0)
    assert events(rep) == [(e[0], e[1], e[2], e[3]) for e in rep_o["loc"]]
    assert rep["detected"] == rep_o["detected"] and rep["corrected"] == rep_o["corrected"]
    assert rep["uncorrectable"] == rep_o["uncorrectable"]
    assert np.abs(L - np.tril(Lo)).max() <= 1e-12 * np.abs(Lo).max()


def test_uniform_schedule_is_the_fixed_mode_run():
    n, nb = 777, 128
    A = W.spd_mmt(n, seed=22)
    faults = [(2, abft.F_MEMORY, 700, 500, 0.1)]
    for mode in (N_, S_, F_):
        T = torch.from_numpy(A).to(DEV)
        rc1, rep1 = abft.potrf(T, nb, mode, faults=faults)
        L1 = T.cpu().numpy()
        rc2, rep2, L2 = run(A, nb, [mode] * 7, faults)
        assert rc1 == rc2 and events(rep1) == events(rep2)
        assert np.array_equal(np.tril(L1), L2)


def test_unchecked_error_is_absorbed_like_the_oracle():
    n, nb = 512, 64
    A = W.spd_mmt(n, seed=23)
    modes = [N_, N_, N_, F_, F_, S_, S_, S_]
    f = [(2, abft.F_MEMORY, 450, 300, 0.125)]
    Lo, _, rep_o = oracle.potrf_sched(A.copy(), nb, modes, f)
    rc, rep, L = run(A, nb, modes, f)
    assert rc == 0 and rep["detected"] == 0 == rep_o["detected"]
    Ae = A.copy()
    Ae[450, 300] += 0.125
    Ae[300, 450] += 0.125
    assert np.abs(L - np.linalg.cholesky(Ae)).max() <= 1e-12 * np.abs(L).max()


@pytest.mark.parametrize("dtype", [abft.MIXED_BF16, abft.MIXED_F16])
def test_mixed_schedule_locates_like_the_oracle(dtype):
    n, nb = 1024, 128
    A = W.spd_mmt(n, seed=24)
    modes = [S_, N_, F_, F_, S_, N_, S_, F_]
    faults = [(2, abft.F_COL1D, 1000, 600, 0.5), (4, abft.F_MEMORY, 1000, 800, 0.5),
              (5, abft.F_MEMORY, 990, 800, 0.5)]
    Lo, _, rep_o = oracle.potrf_sched(A.copy(), nb, modes, faults)
    rc, rep, L = run(A, nb, modes, faults, dtype)
    assert rc == 0 and rep_o["uncorrectable"] == 0
    assert events(rep) == [(e[0], e[1], e[2], e[3]) for e in rep_o["loc"]]
    # 16-bit trailing update: the factor agrees to the mixed-precision level
    assert np.abs(L - np.tril(Lo)).max() <= 5e-2 * np.abs(Lo).max()


def test_policy_schedule_runs():
    """Modes from the adaptive policy for a rising 0D / 1D error rate drive
    the factorization: steps the policy leaves unchecked raise no flag."""
    n, nb = 2048, 256
    A = W.spd_mmt(n, seed=25)
    steps = (n + nb - 1) // nb
    T = [1e-3 * (steps - k) ** 2 / steps ** 2 for k in range(steps)]
    modes, cov = abft.adaptive_modes(n, nb, (2.0, 2e-3, 0.0), 0.999999, T)
    assert modes[0] == F_ and modes[-1] == S_ and min(cov) >= 0.999999
    rc, rep, L = run(A, nb, modes)
    assert rc == 0 and rep["detected"] == 0
    assert np.abs(L @ L.T - A).max() <= 1e-13 * np.abs(A).max() * n
