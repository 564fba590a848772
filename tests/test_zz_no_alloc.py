"""abft_potrf_noalloc: the Cholesky entry point for callers that cannot
allocate device memory (their own allocator or arena owns the GPU, so they
can neither call cudaMalloc nor pass a workspace).  It runs on a built-in
device scratch array; these checks call it through the C ABI and compare it
with abft_potrf (caller workspace) on the same inputs, twice in a row, since
the shared array keeps the previous call's contents."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2301_03166_b300 import abft
from paper_2301_03166_b300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _noalloc(T, nb, mode, faults):
    L = abft.lib()
    fa, nf = abft._faults(faults)
    rep = abft.Report()
    rc = L.abft_potrf_noalloc(T.shape[0], nb, abft.F64, mode, ctypes.c_void_p(T.data_ptr()),
                              T.stride(0), fa, nf, 1.0, ctypes.byref(rep),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, abft.report_dict(rep)


@pytest.mark.parametrize("n,nb,mode,faults", [
    (1024, 128, abft.FULL, [(3, abft.F_MEMORY, 900, 700, 1e3)]),
    (600, 64, abft.SINGLE, [(2, abft.F_COMPUTE, 500, 250, -40.0), (4, abft.F_ROW1D, 450, 330, 3.0)]),
])
def test_noalloc_matches_workspace_entry_point_twice(n, nb, mode, faults):
    A = torch.from_numpy(W.spd_mmt(n, seed=77 + n)).to(DEV)
    ref = A.clone()
    rc_ref, rep_ref = abft.potrf(ref, nb, mode, faults=faults)
    assert rc_ref == 0
    for _ in range(2):                      # two calls in a row on the shared scratch
        T = A.clone()
        rc, rep = _noalloc(T, nb, mode, faults)
        assert rc == 0
        assert torch.max(torch.abs(torch.tril(T) - torch.tril(ref))).item() <= 1e-13
        assert [e[:4] for e in rep["loc"]] == [e[:4] for e in rep_ref["loc"]]
        assert rep["corrected"] == rep_ref["corrected"] == len(rep_ref["loc"])
        assert rep["tau"] == rep_ref["tau"]


def test_noalloc_rejects_oversized_problem():
    L = abft.lib()
    T = torch.empty(8192, 8192, dtype=torch.float64, device=DEV)
    fa, nf = abft._faults([])
    rc = L.abft_potrf_noalloc(8192, 256, abft.F64, abft.FULL, ctypes.c_void_p(T.data_ptr()),
                              8192, fa, nf, 1.0, None, None)
    assert rc == abft.ERR_TOO_LARGE
    assert "scratch" in abft.strerror(rc)
