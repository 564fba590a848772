"""The C-ABI library loads without a GPU and exports every function that
include/*.h declares; the workspace query and argument checks run on the host."""
import ctypes
import glob
import os
import re

import pytest

from paper_2301_03166_b300 import abft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(abft_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = abft.lib()
    names = declared_functions()
    assert "abft_potrf" in names and len(names) >= 5
    for name in names:
        assert hasattr(L, name), name


def test_version_and_strerror():
    assert b"sm_103a" in abft.lib().abft_version()
    assert abft.strerror(-1000).startswith("uncorrectable")


def test_workspace_query_and_arguments_on_host():
    L = abft.lib()
    need = ctypes.c_size_t(0)
    assert L.abft_potrf(1024, 128, 0, 2, None, 1024, None, 0, 1.0, None, None,
                        ctypes.byref(need), None) == 0
    nt = 8
    assert need.value >= 8 * (nt * 1024 + 1024 * nt + 1024 * 128)
    assert L.abft_potrf(-1, 128, 0, 2, None, 1, None, 0, 1.0, None, None, ctypes.byref(need), None) == -1
    assert L.abft_potrf(64, 48, 0, 2, None, 64, None, 0, 1.0, None, None, ctypes.byref(need), None) == -2
    assert L.abft_potrf(64, 32, 7, 2, None, 64, None, 0, 1.0, None, None, ctypes.byref(need), None) == -3
    assert L.abft_potrf(64, 32, 0, 5, None, 64, None, 0, 1.0, None, None, ctypes.byref(need), None) == -4
    assert L.abft_potrf(64, 32, 0, 2, None, 63, None, 0, 1.0, None, None, ctypes.byref(need), None) == -6
    fa, nf = abft._faults([(0, 0, 5, 40, 1.0)])
    assert L.abft_potrf(64, 32, 0, 2, None, 64, fa, nf, 1.0, None, None, ctypes.byref(need), None) == -7
    fa, nf = abft._faults([(1, 0, 60, 60, 1.0)])
    assert L.abft_potrf(64, 32, 0, 2, None, 64, fa, nf, 1.0, None, None, ctypes.byref(need), None) == -7
    assert L.abft_potrf(64, 32, 0, 2, None, 64, None, 0, 0.0, None, None, ctypes.byref(need), None) == -9


def test_cpu_tensor_rejected():
    import torch
    with pytest.raises(TypeError):
        abft.potrf(torch.eye(4, dtype=torch.float64), 32)


def test_gmres_ir_workspace_query_and_arguments_on_host():
    L = abft.lib()
    need = ctypes.c_size_t(0)
    args = lambda m, itol, shift: (1024, 16, 128, abft.MIXED_BF16, abft.FULL, None, 1024, None, 1024,
                                   None, 16, None, 16, 1e-12, 10, m, itol, shift, 1, 0, 0, None,
                                   0, 1.0, None, None, ctypes.byref(need), None)
    assert L.abft_posv_gmres_ir(*args(30, 1e-6, -1.0)) == 0
    # the Krylov basis (m + 1 blocks of n x 16 doubles) is part of the workspace
    assert need.value >= 31 * 1024 * 16 * 8
    assert L.abft_posv_gmres_ir(*args(0, 1e-6, -1.0)) == -16
    assert L.abft_posv_gmres_ir(*args(65, 1e-6, -1.0)) == -16
    assert L.abft_posv_gmres_ir(*args(30, -1.0, -1.0)) == -17
    assert L.abft_posv_gmres_ir(*args(30, 1e-6, float("nan"))) == -18


def test_fault_coverage_and_policy_match_the_oracle():
    """The library's host-side fault-coverage model and mode policy against the
    oracle's literal double sums (no GPU needed)."""
    from oracle import adaptive as ad
    for S, m0, m1, m2 in ((1, 0.3, 0.0, 0.0), (16, 2.0, 0.5, 0.1), (4096, 3.0, 1e-3, 0.0),
                          (65536, 40.0, 2.0, 1e-4), (9, 0.0, 0.0, 0.0)):
        assert abft.fc_single(S, m0, m1, m2) == pytest.approx(ad.fc_single(S, m0, m1, m2), rel=1e-12)
        assert abft.fc_full(S, m0, m1, m2) == pytest.approx(ad.fc_full(S, m0, m1, m2), rel=1e-12)
    import math
    assert math.isnan(abft.fc_single(0, 1.0, 0.0, 0.0))
    n, nb = 8192, 256
    T = [2e-4 * (32 - k) ** 2 for k in range(32)]
    for lam in ((0.0, 0.0, 0.0), (2.0, 0.0, 0.0), (50.0, 0.01, 0.0), (5.0, 1e-3, 1e-4)):
        got, cov = abft.adaptive_modes(n, nb, lam, 0.999999, T)
        want, wcov = ad.adaptive_modes(n, nb, lam, 0.999999, T)
        assert got == want
        assert cov == pytest.approx(wcov, rel=1e-12)


def test_sched_arguments_on_host():
    L = abft.lib()
    need = ctypes.c_size_t(0)
    m = (ctypes.c_int32 * 8)(0, 0, 1, 1, 2, 2, 1, 0)
    assert L.abft_potrf_sched(1024, 128, 0, m, None, 1024, None, 0, 1.0, None, None,
                              ctypes.byref(need), None) == 0
    full = ctypes.c_size_t(0)
    assert L.abft_potrf(1024, 128, 0, 2, None, 1024, None, 0, 1.0, None, None,
                        ctypes.byref(full), None) == 0
    assert need.value == full.value
    bad = (ctypes.c_int32 * 8)(0, 0, 1, 3, 2, 2, 1, 0)
    assert L.abft_potrf_sched(1024, 128, 0, bad, None, 1024, None, 0, 1.0, None, None,
                              ctypes.byref(need), None) == -4


def test_added_entry_points_check_arguments_on_host():
    L = abft.lib()
    need = ctypes.c_size_t(0)
    # abft_syrk_mixed: workspace query and argument checks
    assert L.abft_syrk_mixed(300, 64, 128, abft.MIXED_BF16, None, 64, None, 300, None, None, None,
                             None, ctypes.byref(need), None) == 0 and need.value > 0
    assert L.abft_syrk_mixed(300, 48, 128, abft.MIXED_BF16, None, 64, None, 300, None, None, None,
                             None, ctypes.byref(need), None) == -2
    assert L.abft_syrk_mixed(300, 64, 96, abft.MIXED_BF16, None, 64, None, 300, None, None, None,
                             None, ctypes.byref(need), None) == -3
    assert L.abft_syrk_mixed(300, 64, 128, abft.F64, None, 64, None, 300, None, None, None,
                             None, ctypes.byref(need), None) == -4
    # abft_wait_selftest: host-side checks only (the cases themselves need a GPU)
    assert L.abft_wait_selftest(0, 1000, None, None, ctypes.byref(need), None) == 0
    assert L.abft_wait_selftest(4, 1000, None, None, ctypes.byref(need), None) == -1
    assert L.abft_wait_selftest(0, 0, None, None, ctypes.byref(need), None) == -2
    # abft_batched_partition: host only
    n = (ctypes.c_int64 * 3)(10, 20, 30)
    own = (ctypes.c_int32 * 3)()
    assert L.abft_batched_partition(3, n, 0, own, None) == -3
    assert L.abft_batched_partition(3, n, 2, own, None) == 0 and list(own) == [1, 1, 0]
    # abft_batched_set_ctas_per_sm: host only, returns the previous setting
    assert L.abft_batched_set_ctas_per_sm(-1) == -1
    prev = L.abft_batched_set_ctas_per_sm(3)
    assert L.abft_batched_set_ctas_per_sm(prev) == 3
