"""The allocation-free sizing entry point, checked against the oracle.

gsofa_row_counts_noalloc serves callers that cannot allocate device memory
when they need the factor sizes (for example a solver that reserved the
device's free memory up front, or a loop where cudaMalloc would synchronise
the device).  It must give exactly the per-row sizes and fill counts of the oracle
(and so of the regular entry point), call after call: its scratch array is shared and
keeps the previous call's contents, so two calls in a row are compared.
This file is collected last so a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_device

pytestmark = pytest.mark.gpu


def _noalloc(lib, A, rp, ci):
    import torch
    n = A.n
    nL = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    nU = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    fc = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.gsofa_row_counts_noalloc(n, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
                                      ctypes.c_void_p(nL.data_ptr()), ctypes.c_void_p(nU.data_ptr()),
                                      ctypes.c_void_p(fc.data_ptr()), ctypes.c_void_p(st))
    assert rc == 0, rc
    torch.cuda.synchronize()
    return nL[:n].cpu().numpy(), nU[:n].cpu().numpy(), fc[:n].cpu().numpy()


@pytest.mark.parametrize("which", ["grid3d_32", "random_small", "banded", "banded_max_n", "empty"])
def test_noalloc_counts_match_oracle(which):
    """Per-row sizes and fill counts equal the oracle's, on two calls in a row.
    banded_max_n is the largest accepted order, where the frontier overflow lists
    of a full grid of CTAs do not fit the fixed scratch and the launch uses fewer
    CTAs; empty is n = 0."""
    import paper_2007_00840_gb300 as gs
    from paper_2007_00840_gb300._lib import GSOFA_NOALLOC_MAX_N
    lib = gs.load()
    A = {"grid3d_32": lambda: synth.config(1),
         "random_small": lambda: synth.random_pattern(300, 0.02, seed=77, diag=False),
         "banded": lambda: synth.banded(20000, 200, seed=5),
         "banded_max_n": lambda: synth.banded(GSOFA_NOALLOC_MAX_N, 300, seed=6),
         "empty": lambda: synth.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), "empty")}[which]()
    rp, ci = to_device(A)
    if A.n == 0:
        ci = rp  # any valid device pointer; no column is read
    o = oracle.symbolic(A, nthreads=16)
    want = (o["nnzL"], o["nnzU"], oracle.fill_count(A, o["nnzL"], o["nnzU"]))
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        got = _noalloc(lib, A, rp, ci)
        for g, w in zip(got, want):
            assert np.array_equal(g, np.asarray(w, np.int32))


def test_noalloc_rejects_oversize_and_bad_input():
    import torch
    import paper_2007_00840_gb300 as gs
    from paper_2007_00840_gb300._lib import GSOFA_E_INVAL, GSOFA_NOALLOC_MAX_N
    lib = gs.load()
    A = synth.grid2d(8, 0.7, seed=1)
    rp, ci = to_device(A)
    out = torch.zeros(A.n, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(out.data_ptr())
    rc = lib.gsofa_row_counts_noalloc(GSOFA_NOALLOC_MAX_N + 1, ctypes.c_void_p(rp.data_ptr()),
                                      ctypes.c_void_p(ci.data_ptr()), p, p, p, None)
    assert rc == GSOFA_E_INVAL
    bad = torch.from_numpy(np.where(np.arange(A.nnz) == 5, A.n + 3, A.colidx).astype(np.int32)).cuda()
    rc = lib.gsofa_row_counts_noalloc(A.n, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(bad.data_ptr()),
                                      p, p, p, None)
    assert rc == GSOFA_E_INVAL
    # and a valid call right after still matches
    got = _noalloc(lib, A, rp, ci)
    h = gs.symbolic_device(rp, ci).to_host()
    assert np.array_equal(got[0], np.diff(h.L_rowptr)) and np.array_equal(got[2], h.fill_count)
