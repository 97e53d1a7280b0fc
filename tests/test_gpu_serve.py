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
    st = srv.stats()
    assert st["peak_mem_in_use"] <= 64 << 20
    # device memory the served work actually held (pool high-water mark, slots, input copies)
    assert 0 < st["peak_device_bytes"] <= 64 << 20, st["peak_device_bytes"]
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
    assert 0 < st["peak_device_bytes"] <= cap, st["peak_device_bytes"]
    srv.close()


def test_served_workload_every_result_exact():
    """The served workload's pool (the 512-matrix mix and four 512^2 ND grids):
    each distinct pattern run alone equals the oracle, and every result of a
    stream of 1,500 requests through the benchmark's server shape (2 streams,
    batches of up to 512, 150 GiB cap) equals its pattern run alone."""
    import torch
    import paper_2007_00840_gb300 as gs
    from tests.gpu_util import oracle_full_cached
    small, big = synth.served_pool()
    pool = small + big
    dev = [to_device(A) for A in pool]
    alone = [gs.symbolic_device(rp, ci) for rp, ci in dev]
    torch.cuda.synchronize()
    hosts = gs.results_to_host(alone)
    for k, (A, h) in enumerate(zip(pool, hosts)):
        key = ("config", 3, k) if k < len(small) else ("served_big", k - len(small))
        assert_same(h, oracle_full_cached(key, A)), k
    del hosts
    nreq = 1500
    which, arrivals = synth.served_choices(nreq, len(small), len(big))
    srv = gs.Server(streams=2, max_batch=512, mem_cap_bytes=150 << 30)
    tickets = []
    t0 = time.perf_counter()
    for i in range(nreq):
        due = t0 + arrivals[i] * 0.0015  # about 670 requests/s
        while time.perf_counter() < due:
            pass
        tickets.append(srv.submit(*dev[int(which[i])]))
    bad = []
    for i, t in enumerate(tickets):
        r, _ = srv.wait(t)
        a = alone[int(which[i])]
        for f in FIELDS:
            if not torch.equal(getattr(r, f), getattr(a, f)):
                bad.append((i, int(which[i]), f))
                break
    st = srv.stats()
    srv.close()
    assert not bad, bad[:10]
    assert st["completed"] == nreq and st["failed"] == 0
    assert st["batches"] >= 2


def test_served_malformed_request_fails_alone():
    """A malformed pattern batched with valid ones fails with GSOFA_E_INVAL on its
    own; every valid request of the same batch completes exactly as it would alone."""
    import torch
    import paper_2007_00840_gb300 as gs
    pool = _pool()[:8]
    dev = [to_device(A) for A in pool]
    alone = [gs.symbolic_device(rp, ci).to_host() for rp, ci in dev]
    torch.cuda.synchronize()
    A = pool[2]
    bad = A.colidx.copy()
    bad[len(bad) // 2] = A.n + 11          # a column outside [0, n)
    bad_dev = (dev[2][0], torch.from_numpy(bad).cuda())
    srv = gs.Server(streams=1, max_batch=64)
    # a large request first keeps the slot busy so the rest are batched together
    tickets = [(srv.submit(*to_device(synth.grid2d_nd(200, 0.8, seed=3))), None)]
    for i in range(24):
        if i == 9:
            tickets.append((srv.submit(*bad_dev), "bad"))
        k = i % len(pool)
        tickets.append((srv.submit(*dev[k]), k))
    for t, k in tickets:
        if k == "bad":
            with pytest.raises(gs.GsofaError) as ei:
                srv.wait(t)
            assert ei.value.code == -1
            continue
        r, _ = srv.wait(t)
        if k is None:
            continue
        h = r.to_host()
        for f in FIELDS:
            assert np.array_equal(getattr(h, f), getattr(alone[k], f)), (k, f)
        if pool[k].n <= 5000:
            assert_same(h, oracle_full(pool[k]))
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == len(tickets) - 1
    srv.close()
