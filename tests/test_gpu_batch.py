"""GPU parity of the batched path (gsofa_batch) against the oracle, bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import assert_rows_equal, assert_same, oracle_full, oracle_full_cached, to_device

pytestmark = pytest.mark.gpu


def _batch(mats, **opt):
    import torch
    import paper_2007_00840_gb300 as gs
    dev = [to_device(A) for A in mats]
    res = gs.batch_device(dev, opts=gs.options(**opt) if opt else None)
    torch.cuda.synchronize()
    return [r.to_host() for r in res]


def _mix(seed, count):
    rng = np.random.default_rng(seed)
    mats = []
    for k in range(count):
        kind = k % 4
        if kind == 0:
            mats.append(synth.near_square_grid(int(rng.integers(20, 900)), 0.7, seed=seed * 100 + k))
        elif kind == 1:
            mats.append(synth.banded(int(rng.integers(30, 1500)), int(rng.integers(3, 40)), seed=seed * 100 + k))
        elif kind == 2:
            mats.append(synth.random_pattern(int(rng.integers(2, 80)), 0.06, seed=seed * 100 + k, diag=bool(k % 3)))
        else:
            mats.append(synth.grid2d(int(rng.integers(3, 25)), 0.6, seed=seed * 100 + k))
    return mats


def test_batch_mixed_sizes_exact():
    mats = _mix(1, 48)
    mats.insert(5, synth.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), "empty"))
    mats.insert(9, synth._csr_from_pairs(1, np.array([0]), np.array([0]), "one"))
    got = _batch(mats)
    for A, h in zip(mats, got):
        assert_same(h, oracle_full(A))


def test_batch_with_global_tier_member():
    big = synth.grid2d_nd(400, 0.8, seed=3)          # n = 160,000: labels do not fit on chip
    mats = _mix(2, 12)
    mats.insert(3, big)
    got = _batch(mats)
    for A, h in zip(mats, got):
        if A is big:
            rows = np.concatenate([np.arange(big.n - 40, big.n), np.arange(0, big.n, 997)]).astype(np.int32)
            assert_rows_equal(h, oracle.symbolic(big, rows=rows, nthreads=8), rows)
        else:
            assert_same(h, oracle_full(A))


def test_batch_replay_autotune_and_alone_equal():
    """Same batch twice (graph replay), with the autotuner, and each matrix alone: identical."""
    import torch
    import paper_2007_00840_gb300 as gs
    mats = _mix(3, 40)
    dev = [to_device(A) for A in mats]
    r1 = [r.to_host() for r in gs.batch_device(dev)]
    r2 = [r.to_host() for r in gs.batch_device(dev)]
    r3 = [r.to_host() for r in gs.batch_device(dev, opts=gs.options(autotune=1))]
    r4 = [r.to_host() for r in gs.batch_device(dev, opts=gs.options(work_chunk=3, list_capacity=64))]
    r5 = [r.to_host() for r in gs.batch_device(dev, opts=gs.options(frontier_order=1))]
    r6 = [r.to_host() for r in gs.batch_device(dev, opts=gs.options(frontier_order=2))]
    r7 = [r.to_host() for r in gs.batch_device(dev, opts=gs.options(frontier_order=1, expand_mode=1))]
    r8 = [r.to_host() for r in gs.batch_device(dev, opts=gs.options(frontier_order=1, expand_mode=3,
                                                                      list_capacity=64))]
    r9 = [r.to_host() for r in gs.batch_device(dev, opts=gs.options(frontier_order=1, expand_mode=2))]
    r10 = gs.results_to_host(gs.batch_device(dev))  # adjacent arrays copied as spans
    torch.cuda.synchronize()
    for k, (A, (rp, ci)) in enumerate(zip(mats, dev)):
        alone = gs.symbolic_device(rp, ci).to_host()
        for r in (r1[k], r2[k], r3[k], r4[k], r5[k], r6[k], r7[k], r8[k], r9[k], r10[k]):
            for key in ("L_rowptr", "L_colidx", "U_rowptr", "U_colidx", "fill_count", "super_start"):
                assert np.array_equal(getattr(r, key), getattr(alone, key)), (k, key)
        assert_same(alone, oracle_full(A))


def test_batch_invalid_member_rejected():
    import torch
    import paper_2007_00840_gb300 as gs
    mats = _mix(4, 10)
    dev = [to_device(A) for A in mats]
    bad = mats[6].colidx.copy()
    bad[-1] = mats[6].n + 7
    dev[6] = (dev[6][0], torch.from_numpy(bad).cuda())
    with pytest.raises(gs.GsofaError) as ei:
        gs.batch_device(dev)
    assert ei.value.code == -1
    # still usable afterwards
    got = [r.to_host() for r in gs.batch_device([to_device(A) for A in mats[:3]])]
    for A, h in zip(mats[:3], got):
        assert_same(h, oracle_full(A))


def test_batch_workload_512():
    """The 512-matrix mix at full size, autotuned as the benchmark runs it: every
    member against the oracle on every row, with fill counts and supernodes."""
    mats = synth.config(3)
    got = _batch(mats, autotune=1)  # the configuration the benchmark times
    for k, (A, h) in enumerate(zip(mats, got)):
        assert_same(h, oracle_full_cached(("config", 3, k), A)), k
