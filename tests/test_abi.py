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
                                   None, 16, None, 16, 1e-12, 10, m, itol, shift, 1, 0, None, 0,
                                   1.0, None, None, ctypes.byref(need), None)
    assert L.abft_posv_gmres_ir(*args(30, 1e-6, -1.0)) == 0
    # the Krylov basis (m + 1 blocks of n x 16 doubles) is part of the workspace
    assert need.value >= 31 * 1024 * 16 * 8
    assert L.abft_posv_gmres_ir(*args(0, 1e-6, -1.0)) == -16
    assert L.abft_posv_gmres_ir(*args(65, 1e-6, -1.0)) == -16
    assert L.abft_posv_gmres_ir(*args(30, -1.0, -1.0)) == -17
    assert L.abft_posv_gmres_ir(*args(30, 1e-6, float("nan"))) == -18
