"""Host frontier spill (the external frontier management of Section 6): when
the device budget cannot hold one whole class-kernel slot, each slot's log
(level overflow and L row) lives in pinned host memory that the kernel reads
and writes directly, and only the visited bitmaps take device memory.  The
result is unchanged: bit-exact against the oracle."""
import numpy as np
import pytest

import synth
from tests.gpu_util import assert_same, oracle_full_cached, run_gpu, to_device

pytestmark = pytest.mark.gpu


def _slot_bytes(n):
    cap = (n + 1023) // 1024 * 1024
    return cap // 8 + cap // 256 + 4 * cap


def test_budget_below_one_slot_spills_to_host():
    import paper_2007_00840_gb300 as gs
    A = synth.grid2d_nd(300, 0.8, seed=5)          # n = 90,000: every source in the class kernel
    budget = 2 * (_slot_bytes(A.n) // 2)            # the slot budget (half of it) holds no whole slot
    with pytest.raises(gs.GsofaError) as ei:
        run_gpu(A, frontier_order=2, mem_budget_bytes=budget, host_spill=-1)
    assert ei.value.code == -2                      # GSOFA_E_NOMEM without the host logs
    h = run_gpu(A, frontier_order=2, mem_budget_bytes=budget)    # automatic: host logs
    assert_same(h, oracle_full_cached(("nd300", 5), A))


def test_forced_host_logs_global_bitmaps():
    """Host logs at full concurrency on an order whose bitmaps are in global memory."""
    A = synth.grid2d_nd(400, 0.8, seed=3)          # n = 160,000
    o = oracle_full_cached(("nd400", 3), A)
    assert_same(run_gpu(A, host_spill=1), o)
    assert_same(run_gpu(A, host_spill=1, team_sources=64), o)
    for k, B in enumerate((synth.random_pattern(300, 0.02, seed=24, diag=False), synth.banded(2500, 30, seed=22))):
        assert_same(run_gpu(B, frontier_order=2, host_spill=1), oracle_full_cached(("spill", k), B))


def test_served_request_refused_without_spill_completes_with_it():
    import torch
    import paper_2007_00840_gb300 as gs
    A = synth.grid2d_nd(300, 0.8, seed=5)
    dev = to_device(A)
    n, nnz = A.n, A.nnz
    # the server's projection of this request without its slots (device input)
    est = min(64 * nnz + 16 * n, n * (n + 1))
    base = 96 * n + 8 * est + (1 << 20)
    cap = base + _slot_bytes(n) // 2                 # room for half a slot
    srv = gs.Server(mem_cap_bytes=cap, streams=2, opts=gs.options(host_spill=-1))
    with pytest.raises(gs.GsofaError) as ei:
        srv.submit(*dev)
    assert ei.value.code == -2
    srv.close()
    srv = gs.Server(mem_cap_bytes=cap, streams=2)
    r, _ = srv.wait(srv.submit(*dev))
    torch.cuda.synchronize()
    assert_same(r.to_host(), oracle_full_cached(("nd300", 5), A))
    st = srv.stats()
    assert st["completed"] == 1 and st["peak_mem_in_use"] <= cap
    srv.close()
