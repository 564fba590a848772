"""Host-side helpers of bench.py (no GPU): the energy arithmetic and the
LAPACK CPU baseline on a small matrix."""
import importlib.util
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    saved = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test",
                                                      os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = saved
    return mod


def test_energy_joules(bench):
    # counter in mJ: 4 J over 2 calls = 2 J per call; missing or non-increasing -> None
    assert bench.BoardEnergy.joules(1000.0, 5000.0, 2) == 2.0
    assert bench.BoardEnergy.joules(None, 5000.0, 1) is None
    assert bench.BoardEnergy.joules(5000.0, 5000.0, 1) is None
    assert bench.BoardEnergy.joules(1000.0, 5000.0, 0) is None


def test_energy_reader_without_gpu(bench):
    # no CUDA device here: the reader must report "unavailable", not raise
    assert bench.BoardEnergy("cpu").read() is None


def test_lapack_baseline_factors(bench):
    rng = np.random.default_rng(7)
    m = rng.standard_normal((200, 200))
    a = m @ m.T / 200 + np.eye(200)
    a0 = a.copy()
    t, threads, name = bench.lapack_baseline(a)
    assert t > 0 and threads >= 1 and "dpotrf" in name
    assert np.array_equal(a, a0)   # the caller's matrix is not touched
