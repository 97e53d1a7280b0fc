"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Every output is integer/index data, so the bar is exact equality: L and U row
pointers and sorted columns, fill counts and the supernode partition.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.common import brute_ge, load_paper_example, pattern_from_result
from tests.gpu_util import assert_same, oracle_full, oracle_full_cached, run_gpu, to_device

pytestmark = pytest.mark.gpu


def test_paper_example():
    A, facts = load_paper_example()
    h = run_gpu(A)
    assert_same(h, oracle_full(A))
    assert h.L_colidx[h.L_rowptr[8]:h.L_rowptr[9]].tolist() == facts["row8_L"]
    assert h.U_colidx[h.U_rowptr[8]:h.U_rowptr[9]].tolist() == facts["row8_U"]


@pytest.mark.parametrize("tier", ["smem", "global"])
def test_random_small(tier):
    opt = {} if tier == "smem" else {"smem_max_source": -1}
    for t in range(60):
        n = 5 + (t * 7) % 90
        A = synth.random_pattern(n, [0.03, 0.08, 0.2][t % 3], seed=7000 + t, diag=bool(t % 4))
        h = run_gpu(A, **opt)
        assert_same(h, oracle_full(A))
        if n <= 40:
            P = pattern_from_result(n, h.L_rowptr, h.L_colidx, h.U_rowptr, h.U_colidx)
            assert np.array_equal(P, brute_ge(A))


def test_adversarial_shapes():
    cases = []
    n = 300
    # star: vertex 0 connected both ways to everyone (dense first row/column)
    r = np.concatenate([np.zeros(n), np.arange(n), np.arange(n)])
    c = np.concatenate([np.arange(n), np.zeros(n), np.arange(n)])
    cases.append(synth._csr_from_pairs(n, r, c, "star0"))
    # chain ordered high -> low (forces many maxId revisits)
    r = np.concatenate([np.arange(1, n), np.arange(n)])
    c = np.concatenate([np.arange(0, n - 1), np.arange(n)])
    cases.append(synth._csr_from_pairs(n, r, c, "chain_down"))
    r = np.concatenate([np.arange(0, n - 1), np.arange(n)])
    c = np.concatenate([np.arange(1, n), np.arange(n)])
    cases.append(synth._csr_from_pairs(n, r, c, "chain_up"))
    # empty rows, no diagonal, isolated vertices
    A = synth.random_pattern(200, 0.02, seed=3, diag=False)
    cases.append(A)
    # rows longer than 32 entries (warp-cooperative expansion) and a dense last row
    rng = np.random.default_rng(5)
    rr, cc = [], []
    for i in range(400):
        k = 60 if i % 37 == 0 else 3
        cols = rng.choice(400, size=k, replace=False)
        rr += [i] * k
        cc += cols.tolist()
    rr += [399] * 400
    cc += list(range(400))
    cases.append(synth._csr_from_pairs(400, np.array(rr), np.array(cc), "bigdeg"))
    # one row, two rows, dense block
    cases.append(synth._csr_from_pairs(1, np.array([0]), np.array([0]), "n1"))
    cases.append(synth.CSR(1, np.array([0, 0], np.int32), np.zeros(0, np.int32), "n1_empty"))
    cases.append(synth._csr_from_pairs(2, np.array([0, 1]), np.array([1, 0]), "n2_swap"))
    cases.append(synth.random_pattern(70, 1.0, seed=1))
    for A in cases:
        for opt in ({}, {"smem_max_source": -1}, {"fill_first": 1}, {"expand_mode": 2},
                    {"expand_mode": 2, "fill_first": 1, "list_capacity": 32}):
            h = run_gpu(A, **opt)
            assert_same(h, oracle_full(A)), (A.name, opt)


def test_frontier_orders_and_autotune():
    """Breadth-first, class-ordered and autotuned frontier orders give the same rows."""
    cases = [synth.grid2d(40, 0.7, seed=21), synth.banded(2500, 30, seed=22),
             synth.grid2d_nd(60, 0.8, seed=23, leaf=16), synth.random_pattern(300, 0.02, seed=24, diag=False)]
    for A in cases:
        o = oracle_full(A)
        for opt in ({"frontier_order": 1}, {"frontier_order": 2}, {"autotune": 1}, {"autotune": 1},
                    {"expand_mode": 2}, {"expand_mode": 2, "label_bits": 32}, {"label_bits": 32, "fill_first": 1},
                    {"expand_mode": 1}, {"expand_mode": 3, "label_bits": 32}):
            assert_same(run_gpu(A, **opt), o), (A.name, opt)


def test_worklist_schedule_exact():
    """The shared-memory tier without level barriers (schedule = 2) gives the same rows."""
    rng = np.random.default_rng(5)
    rr, cc = [], []
    for i in range(400):  # a few rows with more than 8 neighbours (read from the CSR)
        k = 40 if i % 53 == 0 else 3
        cols = rng.choice(400, size=k, replace=False)
        rr += [i] * k
        cc += cols.tolist()
    cases = [synth.config(0), synth.grid2d(40, 0.7, seed=21), synth.banded(2500, 30, seed=22),
             synth.random_pattern(300, 0.02, seed=24, diag=False), synth.random_pattern(20, 0.3, seed=5),
             synth._csr_from_pairs(400, np.array(rr), np.array(cc), "bigdeg"), load_paper_example()[0]]
    for A in cases:
        assert_same(run_gpu(A, schedule=2), oracle_full(A)), A.name
        assert_same(run_gpu(A, schedule=2, threads_per_source=256), oracle_full(A)), A.name
    A = synth.config(1)
    assert_same(run_gpu(A, schedule=2), oracle_full(A, nthreads=16))


def _class_order_case_list():
    n = 300
    r = np.concatenate([np.zeros(n), np.arange(n), np.arange(n)])
    c = np.concatenate([np.arange(n), np.zeros(n), np.arange(n)])
    star = synth._csr_from_pairs(n, r, c, "star0")
    r = np.concatenate([np.arange(1, n), np.arange(n)])
    c = np.concatenate([np.arange(0, n - 1), np.arange(n)])
    chain = synth._csr_from_pairs(n, r, c, "chain_down")
    rng = np.random.default_rng(5)
    rr, cc = [], []
    for i in range(400):
        k = 60 if i % 37 == 0 else (9 if i % 5 == 0 else 3)   # rows past one 8-entry record
        cols = rng.choice(400, size=k, replace=False)
        rr += [i] * k
        cc += cols.tolist()
    bigdeg = synth._csr_from_pairs(400, np.array(rr), np.array(cc), "bigdeg")
    return [synth.grid2d_nd(60, 0.8, seed=23, leaf=16), synth.grid2d_nd(200, 0.8, seed=3),
            synth.random_pattern(300, 0.02, seed=24, diag=False), synth.random_pattern(40, 0.3, seed=5),
            star, chain, bigdeg, synth.grid2d(40, 0.7, seed=21), synth.banded(2500, 30, seed=22),
            synth.banded(40000, 30, seed=25),   # past 32,768 rows: 32-bit records, rows past 8 entries
            load_paper_example()[0]]


def _class_order_run(A, **opt):
    import torch
    import paper_2007_00840_gb300 as gs
    rp, ci = to_device(A)
    r = gs.symbolic_device(rp, ci, opts=gs.options(frontier_order=2, collect_stats=1, **opt))
    torch.cuda.synchronize()
    return r.stats, r.to_host()


def test_clean_head_retirement():
    """Class order with runs of clean class heads (heads whose neighbours are all
    reached already) retired together: off, adaptive, before every class, with
    and CTA teams.  Same rows as the oracle, and class order expands every reached
    vertex below the source exactly once, so the expansion and scanned-entry counts
    equal the oracle's minimum-work counts (Dijkstra order, Section 8)."""
    for A in _class_order_case_list():
        o = oracle_full(A)
        for opt in ({"clean_heads": -1}, {"clean_heads": 0}, {"clean_heads": 1}, {"clean_heads": 2},
                    {"clean_heads": 2, "team_sources": 64}, {"clean_heads": 1, "team_sources": 8}):
            st, h = _class_order_run(A, **opt)
            assert_same(h, o), (A.name, opt)
            assert st["vertices_expanded"] == int(o["vscan"].sum()), (A.name, opt)
            assert st["edges_scanned"] == int(o["escan"].sum()), (A.name, opt)
    # bitmaps in global memory (orders past the shared-memory bitmap limit)
    A = synth.grid2d_nd(400, 0.8, seed=3)          # n = 160,000
    o = oracle_full_cached(("nd400", 3), A)
    for opt in ({"clean_heads": -1}, {"clean_heads": 0}, {"clean_heads": 2}, {"clean_heads": 2, "team_sources": 256}):
        st, h = _class_order_run(A, **opt)
        assert_same(h, o), opt
        assert st["vertices_expanded"] == int(o["vscan"].sum()), opt


def test_empty_matrix():
    A = synth.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), "empty")
    h = run_gpu(A)
    assert h.n == 0 and h.nnz_L == 0 and h.nnz_U == 0
    assert h.super_start.tolist() == [0]


def test_grids_and_chunk_sizes():
    A = synth.grid2d(40, 0.7, seed=9)
    o = oracle_full(A)
    for opt in ({}, {"threads_per_source": 128}, {"threads_per_source": 1024}, {"smem_max_source": 512},
                {"smem_max_source": -1, "max_concurrent": 7}):
        assert_same(run_gpu(A, **opt), o)
    for chunk in (1, 16, 64, 256):
        h = run_gpu(A, chunk_size=chunk)
        o2 = oracle.supernodes(o["nnzU"], o["L_rowptr"], o["L_colidx"], chunk)
        assert np.array_equal(h.super_start, o2), chunk
    A = synth.grid2d_nd(48, 0.8, seed=4, leaf=16)
    assert_same(run_gpu(A), oracle_full(A))
    A = synth.banded(3000, 40, seed=12)
    assert_same(run_gpu(A), oracle_full(A))


def test_workload_grid2d_64():
    """Plain 64x64 5-point grid, natural order, p = 0.7 (first workload), all rows."""
    A = synth.config(0)
    o = oracle_full(A)
    assert_same(run_gpu(A), o)
    assert_same(run_gpu(A, fill_first=1), o)
    assert_same(run_gpu(A, smem_max_source=-1), o)


def test_workload_grid3d_32():
    """32^3 7-point grid + extra entry per row (the benchmark workload), all rows, bench launch config."""
    A = synth.config(1)
    o = oracle_full(A, nthreads=16)
    h = run_gpu(A)
    assert_same(h, o)
    assert h.nnz_L + h.nnz_U == int(o["L_rowptr"][-1] + o["U_rowptr"][-1])
    assert_same(run_gpu(A, expand_mode=2), o)
    assert_same(run_gpu(A, expand_mode=1), o)


def test_workload_nd_1m_full():
    """1024^2 nested-dissection grid (n = 1,048,576) at full size, in the launch
    configuration the benchmark times: every row of L and U, the fill counts and
    the whole supernode partition against the oracle."""
    A = synth.config(2)
    h = run_gpu(A)
    o = oracle_full_cached(("config", 2), A)
    assert_same(h, o)
    assert h.nnz_L + h.nnz_U == int(o["L_rowptr"][-1] + o["U_rowptr"][-1])


def test_invalid_csr_is_rejected():
    import torch
    import paper_2007_00840_gb300 as gs
    A = synth.grid2d(8, 0.7, seed=1)
    bad = A.colidx.copy()
    bad[10] = A.n + 5
    with pytest.raises(gs.GsofaError) as ei:
        gs.symbolic_device(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(bad).cuda())
    assert ei.value.code == -1 and ei.value.detail >= 0
    uns = A.colidx.copy()
    r = int(A.rowptr[20])
    uns[r], uns[r + 1] = uns[r + 1], uns[r]
    with pytest.raises(gs.GsofaError):
        gs.symbolic_device(torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(uns).cuda())
    # the library still works afterwards
    assert_same(run_gpu(A), oracle_full(A))


def test_host_entry_point():
    import paper_2007_00840_gb300 as gs
    A = synth.config(0)
    h = gs.symbolic_host(A.rowptr, A.colidx)
    assert_same(h, oracle_full(A))
    h2 = gs.symbolic_host(A.rowptr, A.colidx)   # reuses the pinned block
    assert_same(h2, oracle_full(A))


def test_repeatable_and_stream():
    import torch
    import paper_2007_00840_gb300 as gs
    A = synth.grid2d(30, 0.6, seed=2)
    rp, ci = to_device(A)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r1 = gs.symbolic_device(rp, ci, stream=s)
        r2 = gs.symbolic_device(rp, ci, stream=s)
    s.synchronize()
    h1, h2 = r1.to_host(), r2.to_host()
    assert np.array_equal(h1.L_colidx, h2.L_colidx) and np.array_equal(h1.U_colidx, h2.U_colidx)
    assert_same(h1, oracle_full(A))


def test_stats_are_reported():
    A = synth.config(0)
    h = run_gpu(A, collect_stats=1)
    o = oracle_full(A)
    assert h.stats["ms_traverse"] > 0
    # the label-correcting traversal expands at least the vertices Dijkstra expands
    assert h.stats["vertices_expanded"] >= int(o["vscan"].sum())
    assert h.stats["edges_scanned"] >= int(o["escan"].sum())
