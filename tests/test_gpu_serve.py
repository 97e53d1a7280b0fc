"""Served path (gsofa_server_*): continuous batching gives the same result as
running each pattern alone, bit for bit, and the oracle's result."""
import time

import numpy as np
import pytest

import synth
from tests.gpu_util import assert_same, oracle_full, to_device

pytestmark = pytest.mark.gpu

FIELDS = ("L_rowptr", "L_colidx", "U_rowptr", "U_colidx", "fill_count", "super_start")


def _pool():
    mats = [synth.batch_mix_one(m, seed=1000 + m, n_lo=200, n_hi=4000) for m in range(20)]
    mats.append(synth.grid2d(30, 0.7, seed=3))
    mats.append(synth.random_pattern(50, 0.05, seed=9, diag=False))
    mats.append(synth.grid2d_nd(300, 0.8, seed=5))   # n = 90,000: single-matrix global tier
    return mats


@pytest.mark.parametrize("streams,max_batch", [(3, 16), (2, 512)])
def test_served_equal_alone_and_oracle(streams, max_batch):
    import torch
    import paper_2007_00840_gb300 as gs
    pool = _pool()
    dev = [to_device(A) for A in pool]
    alone = [gs.symbolic_device(rp, ci).to_host() for rp, ci in dev]
    torch.cuda.synchronize()
    for A, h in zip(pool, alone):
        if A.n <= 5000:
            assert_same(h, oracle_full(A))
    rng = np.random.default_rng(11)
    srv = gs.Server(streams=streams, max_batch=max_batch)
    tickets = []
    for i in range(240):
        k = int(rng.integers(0, len(pool)))
        if i % 5 == 0:
            t = srv.submit(pool[k].rowptr, pool[k].colidx)      # host input
        else:
            t = srv.submit(*dev[k])                              # device-resident input
        tickets.append((t, k))
        if i % 7 == 0:
            time.sleep(0.0005)
    for t, k in tickets:
        r, lat = srv.wait(t)
        h = r.to_host()
        for f in FIELDS:
            assert np.array_equal(getattr(h, f), getattr(alone[k], f)), (k, f)
        assert lat > 0
    st = srv.stats()
    assert st["completed"] == 240 and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    assert st["batches"] >= 2
    srv.close()


def test_admission_cap_busy_and_oversize():
    import torch
    import paper_2007_00840_gb300 as gs
    pool = _pool()[:6]
    dev = [to_device(A) for A in pool]
    alone = [gs.symbolic_device(rp, ci).to_host() for rp, ci in dev]
    torch.cuda.synchronize()
    # a cap that admits about one request at a time still completes everything
    srv = gs.Server(mem_cap_bytes=64 << 20, streams=2, queue_capacity=8)
    tickets = []
    busy = 0
    for i in range(40):
        k = i % len(pool)
        try:
            tickets.append((srv.submit(*dev[k]), k))
        except gs.GsofaError as e:
            assert e.code == -6      # GSOFA_E_BUSY: pending queue full
            busy += 1
    for t, k in tickets:
        r, _ = srv.wait(t)
        h = r.to_host()
        for f in FIELDS:
            assert np.array_equal(getattr(h, f), getattr(alone[k], f))
    assert busy > 0
    # a request that alone exceeds the cap is refused at submission
    big = synth.grid2d(400, 0.7, seed=1)
    with pytest.raises(gs.GsofaError) as ei:
        srv.submit(*to_device(big))
    assert ei.value.code == -2
    assert srv.stats()["peak_mem_in_use"] <= 64 << 20
    srv.close()


def test_space_budget_admission():
    """A request whose default global-tier slots exceed the memory cap is admitted
    with fewer slots (the concurrent-source budget of Section 5, Eq. 1) instead of
    being refused, and its result is unchanged."""
    import torch
    import paper_2007_00840_gb300 as gs
    big = synth.grid2d_nd(300, 0.8, seed=5)   # n = 90,000: global tier
    dev = to_device(big)
    alone = gs.symbolic_device(*dev).to_host()
    small = [synth.batch_mix_one(m, seed=50 + m, n_lo=200, n_hi=2000) for m in range(6)]
    sdev = [to_device(A) for A in small]
    salone = [gs.symbolic_device(*d).to_host() for d in sdev]
    torch.cuda.synchronize()
    cap = 1536 << 20
    srv = gs.Server(mem_cap_bytes=cap, streams=2)
    t_big = srv.submit(*dev)
    tickets = [srv.submit(*d) for d in sdev]
    r, _ = srv.wait(t_big)
    h = r.to_host()
    for f in FIELDS:
        assert np.array_equal(getattr(h, f), getattr(alone, f)), f
    for t, a in zip(tickets, salone):
        r, _ = srv.wait(t)
        h = r.to_host()
        for f in FIELDS:
            assert np.array_equal(getattr(h, f), getattr(a, f)), f
    st = srv.stats()
    assert st["completed"] == 7 and st["failed"] == 0
    assert st["peak_mem_in_use"] <= cap
    srv.close()
