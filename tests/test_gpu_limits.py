"""GPU parity at the size limits of the label encodings, and the bounded host
waits: a wait that runs out reports GSOFA_E_TIMEOUT and leaves the library
usable (no GPU fault is involved: the kernel simply finishes later)."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_rows_equal, assert_same, check_supernode_rule, oracle_full, run_gpu, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [65533, 65534])
def test_label_width_boundary(n):
    """n = 65,533 is the largest order with 16-bit labels (every source on chip,
    U through labels); n = 65,534 switches to 32-bit labels, a shared-memory tier
    below the on-chip limit and the class-ordered global tier above it."""
    A = synth.banded(n, 24, seed=n)
    h = run_gpu(A)
    rows = np.unique(np.concatenate([np.arange(n - 48, n), np.arange(0, n, 991), np.arange(0, 16)])).astype(np.int32)
    assert_rows_equal(h, oracle.symbolic(A, rows=rows, nthreads=16), rows)
    fc = oracle.fill_count(A, np.diff(h.L_rowptr), np.diff(h.U_rowptr))
    assert np.array_equal(h.fill_count, fc)
    check_supernode_rule(h)
    # both traversal kernels over every source give the same rows
    h2 = run_gpu(A, frontier_order=2)
    for k in ("L_rowptr", "L_colidx", "U_rowptr", "U_colidx", "super_start"):
        assert np.array_equal(getattr(h, k), getattr(h2, k)), k


def test_bounded_wait_times_out_and_library_recovers(monkeypatch):
    import torch
    import paper_2007_00840_gb300 as gs
    A = synth.config(1)
    rp, ci = to_device(A)
    monkeypatch.setenv("GSOFA_TIMEOUT_S", "0.000001")
    with pytest.raises(gs.GsofaError) as ei:
        gs.symbolic_device(rp, ci)
    assert ei.value.code == -5  # GSOFA_E_TIMEOUT
    torch.cuda.synchronize()   # the abandoned work completes; nothing faulted
    monkeypatch.delenv("GSOFA_TIMEOUT_S")
    assert_same(gs.symbolic_device(rp, ci).to_host(), oracle_full(A, nthreads=16))
