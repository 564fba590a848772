"""Look-ahead of the blocked Cholesky (Sec. 2.1, Fig. example-lu (b)): the
next diagonal block is factored on a side stream while the rest of the
trailing update runs.  Every kernel does the same arithmetic in either
schedule, so factors, reports and return codes must be bit-identical with
look-ahead on and off, for every update precision, checksum mode and kind of
injected error, including ragged last blocks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def run(A, nb, mode, dtype, faults, lookahead):
    prev = abft.set_lookahead(lookahead)
    try:
        T = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
        rc, rep = abft.potrf(T, nb, mode, dtype=dtype, faults=faults, check=False)
        torch.cuda.synchronize()
        return rc, rep, T.cpu().numpy()
    finally:
        abft.set_lookahead(prev)


def same(a, b):
    rc1, rep1, L1 = a
    rc2, rep2, L2 = b
    diffs = []
    if rc1 != rc2:
        diffs.append(f"rc {rc1} != {rc2}")
    if not np.array_equal(L1, L2):
        bad = np.argwhere(L1 != L2)
        diffs.append(f"{len(bad)} entries differ, first {bad[:4].tolist()}, "
                     f"max |diff| {np.abs(L1 - L2).max():.3e}")
    for key in ("detected", "corrected", "uncorrectable", "checksum_repaired", "tau",
                "max_ratio", "info"):
        if rep1[key] != rep2[key]:
            diffs.append(f"{key} {rep1[key]} != {rep2[key]}")
    if rep1["loc"] != rep2["loc"]:
        diffs.append(f"events {rep1['loc']} != {rep2['loc']}")
    assert not diffs, "; ".join(diffs)


# (step, kind, row, col, delta) for n = 1500, nb = 256: errors in the
# look-ahead block column and in the rest of the update, off-diagonal blocks;
# the 1D errors are short so that every event fits the report
FAULTS = [(0, abft.F_MEMORY, 700, 300, 2.0),        # look-ahead column (block 1)
          (1, abft.F_COMPUTE, 600, 520, -2.5),      # look-ahead column (block 2)
          (1, abft.F_MEMORY, 1100, 900, 3.0),       # rest
          (2, abft.F_COMPUTE, 1400, 1300, 2.75),    # rest
          (2, abft.F_COL1D, 1490, 1100, 2.0),       # rest (10 rows; FULL mode only)
          (3, abft.F_ROW1D, 1300, 1270, 2.5),       # look-ahead column (block 4, 10 columns)
          (4, abft.F_MEMORY, 1450, 1290, -2.0)]     # last step: no split


@pytest.mark.parametrize("dtype", [abft.F64, abft.MIXED_BF16, abft.MIXED_F16, abft.F64_EMU])
@pytest.mark.parametrize("mode", [oracle.NONE, oracle.SINGLE, oracle.FULL])
def test_lookahead_is_bit_identical(dtype, mode):
    n, nb = 1500, 256
    A = W.spd_mmt(n, seed=61)
    faults = [] if mode == oracle.NONE else \
        [f for f in FAULTS if mode == oracle.FULL or f[1] != abft.F_COL1D]
    on = run(A, nb, mode, dtype, faults, True)
    off = run(A, nb, mode, dtype, faults, False)
    same(on, off)
    assert on[0] == 0


@pytest.mark.parametrize("n,nb", [(1024, 128), (777, 128), (2048, 256)])
def test_lookahead_fp64_matches_oracle(n, nb):
    A = W.spd_mmt(n, seed=62 + n)
    # step 1 in the look-ahead column (block 2), step 2 in the rest (block 4 or
    # the last block)
    faults = [(1, abft.F_MEMORY, n - 5, 2 * nb + 3, 2.0),
              (2, abft.F_COMPUTE, n - 1, min(4 * nb + 1, n - 2), -1.5)]
    Lo, info_o, rep_o = oracle.potrf(A, nb, oracle.FULL, faults)
    rc, rep, L = run(A, nb, oracle.FULL, abft.F64, faults, True)
    assert rc == info_o == 0
    assert [tuple(e[:4]) for e in rep["loc"]] == [tuple(e[:4]) for e in rep_o["loc"]]
    assert np.abs(np.tril(L) - np.tril(Lo)).max() <= 1e-12 * np.abs(Lo).max()


def test_lookahead_non_spd_info():
    """A non-positive pivot found by the look-ahead PD stops the factorization
    with the same info as the sequential schedule."""
    n, nb = 1024, 128
    A = W.spd_mmt(n, seed=63)
    A[600, 600] = -5.0
    on = run(A, nb, oracle.FULL, abft.F64, [], True)
    off = run(A, nb, oracle.FULL, abft.F64, [], False)
    assert on[0] == off[0] > 0


def test_set_lookahead_returns_previous():
    prev = abft.set_lookahead(False)
    try:
        assert abft.set_lookahead(True) is False
        assert abft.set_lookahead(True) is True
    finally:
        abft.set_lookahead(prev)
