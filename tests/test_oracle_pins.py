"""Pins for the CPU oracle (no GPU).

Each test checks ``oracle/`` against something other than itself: boolean
Gaussian elimination (Section 2.1), the paper's worked example (Sections 1,
2.1, 2.2, 4, 5), a closed form, structural invariants, the elimination tree of
symmetric patterns (Section 2.1) and numeric LU modulo a prime.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from tests.common import (brute_ge, dense_pattern, etree_cholesky_rows, load_paper_example,
                          numeric_lu_pattern_modp, pattern_from_result, t3_supernodes_dense)
from tests.model_maxid import maxid_levels


def oracle_pattern(A):
    r = oracle.symbolic(A)
    return pattern_from_result(A.n, r["L_rowptr"], r["L_colidx"], r["U_rowptr"], r["U_colidx"]), r


def csr_from_dense(P, name="dense"):
    r, c = np.nonzero(P)
    return synth._csr_from_pairs(P.shape[0], r, c, name)


# --------------------------------------------------------- brute force GE --

@pytest.mark.parametrize("n", [1, 2, 3])
def test_exhaustive_small(n):
    offd = [(i, j) for i in range(n) for j in range(n) if i != j]
    for bits in range(1 << len(offd)):
        for diag in (True, False):
            P = np.zeros((n, n), bool)
            for b, (i, j) in enumerate(offd):
                if bits >> b & 1:
                    P[i, j] = True
            if diag:
                np.fill_diagonal(P, True)
            A = csr_from_dense(P)
            got, _ = oracle_pattern(A)
            assert np.array_equal(got, brute_ge(A)), (n, bits, diag)


def test_exhaustive_n4():
    n = 4
    offd = [(i, j) for i in range(n) for j in range(n) if i != j]
    for bits in range(1 << len(offd)):
        P = np.eye(n, dtype=bool)
        for b, (i, j) in enumerate(offd):
            if bits >> b & 1:
                P[i, j] = True
        A = csr_from_dense(P)
        got, _ = oracle_pattern(A)
        assert np.array_equal(got, brute_ge(A)), bits


def test_random_up_to_24():
    rng = np.random.default_rng(1234)
    for t in range(1500):
        n = int(rng.integers(5, 25))
        dens = float(rng.choice([0.05, 0.1, 0.15, 0.25, 0.4]))
        A = synth.random_pattern(n, dens, seed=t, diag=bool(t % 3))
        got, _ = oracle_pattern(A)
        assert np.array_equal(got, brute_ge(A)), (t, n, dens)


def test_random_larger_sparse():
    for t in range(40):
        n = 60 + 7 * t
        A = synth.random_pattern(n, 2.5 / n, seed=10_000 + t)
        got, _ = oracle_pattern(A)
        assert np.array_equal(got, brute_ge(A)), t


def test_grids_against_ge():
    for k, p in [(6, 0.7), (7, 0.5), (9, 0.8)]:
        A = synth.grid2d(k, p, seed=k)
        got, _ = oracle_pattern(A)
        assert np.array_equal(got, brute_ge(A))
    A = synth.grid2d_nd(12, 0.8, seed=5, leaf=8)
    got, _ = oracle_pattern(A)
    assert np.array_equal(got, brute_ge(A))
    A = synth.banded(150, 9, seed=3)
    got, _ = oracle_pattern(A)
    assert np.array_equal(got, brute_ge(A))


# -------------------------------------------------------- worked example --

def test_paper_example_row8_and_fills():
    A, facts = load_paper_example()
    r = oracle.symbolic(A)
    L8 = r["L_colidx"][r["L_rowptr"][8]:r["L_rowptr"][9]].tolist()
    U8 = r["U_colidx"][r["U_rowptr"][8]:r["U_rowptr"][9]].tolist()
    assert L8 == facts["row8_L"]
    assert U8 == facts["row8_U"]
    P, _ = oracle_pattern(A)
    Adense = dense_pattern(A)
    for i, j in facts["fill"]:
        assert P[i, j] and not Adense[i, j], (i, j)
    for i, c in facts["nnzU"]:
        assert r["nnzU"][i] == c
    for i, j in facts["L_nonzero"]:
        assert P[i, j]
    for i, j in facts["L_zero"]:
        assert not P[i, j]
    # the brute-force elimination agrees on the whole example
    assert np.array_equal(P, brute_ge(A))


def test_paper_example_supernodes():
    A, facts = load_paper_example()
    r = oracle.full(A, chunk=4)
    nnzU = r["nnzU"]
    bitmap = [0] + [int(nnzU[s] == nnzU[s - 1] - 1) for s in range(1, 4)]
    assert bitmap == facts["phase1_bitmap_rows0_3"]
    leaders = [s for s in range(4) if bitmap[s] == 0]
    assert leaders == facts["leaders_rows0_3"]
    ss = r["super_start"].tolist()
    assert [s for s in ss if s <= 4] == facts["supernodes_rows0_3"]


def test_paper_example_traversal_trace():
    """Level-synchronous maxId model reproduces Fig. 6 and ends at the oracle's labels."""
    A, facts = load_paper_example()
    lab, hist, after1, L, U = maxid_levels(A, 8)
    assert hist == facts["frontiers"]
    for v, m in facts["maxid_after_iter1"].items():
        assert after1[v] == m
    for v, m in facts["maxid_final"].items():
        assert lab[v] == m
    assert L == facts["row8_L"] and U == facts["row8_U"]


def test_visit_once_variant_misses_fill_84():
    """Section 4: fill2 with parallel thresholds and visit-once marks loses (8, 4)."""
    A, facts = load_paper_example()
    # thread on frontier 7 explores vertex 4 before the path 8->2->3->4 arrives
    _, _, _, L, _ = maxid_levels(A, 8, order=lambda f: -f, visit_once=True)
    assert 4 not in L
    _, _, _, L2, _ = maxid_levels(A, 8, order=lambda f: -f, visit_once=False)
    assert 4 in L2


def test_model_matches_oracle_on_random():
    """The level-synchronous label-correcting model gives the oracle's rows."""
    for t in range(60):
        A = synth.random_pattern(40, 0.06, seed=500 + t)
        r = oracle.symbolic(A)
        for s in range(0, A.n, 3):
            _, _, _, L, U = maxid_levels(A, s)
            assert L == r["L_colidx"][r["L_rowptr"][s]:r["L_rowptr"][s + 1]].tolist()
            assert U == r["U_colidx"][r["U_rowptr"][s]:r["U_rowptr"][s + 1]].tolist()


# ------------------------------------------------------------ closed form --

@pytest.mark.parametrize("k", [3, 4, 5, 6, 8, 16, 64])
def test_full_grid_closed_form(k):
    """k x k 5-point grid, natural order, all entries: L(i,:) = {i-1} in the
    first grid row and [i-k, i) after it, U = L^T + I, so
    nnz(L+U) = n + 2((k-1) + (n-k)k)."""
    n = k * k
    A = synth.grid2d(k, 1.0, seed=0)
    r = oracle.symbolic(A)
    assert int(r["L_rowptr"][-1] + r["U_rowptr"][-1]) == n + 2 * ((k - 1) + (n - k) * k)
    for i in range(n):
        L = r["L_colidx"][r["L_rowptr"][i]:r["L_rowptr"][i + 1]].tolist()
        assert L == ([i - 1] if 0 < i < k else list(range(i - k, i)) if i >= k else [])


# ------------------------------------------------------------- invariants --

def test_containment_and_transpose():
    for t in range(30):
        A = synth.random_pattern(50, 0.05, seed=900 + t, diag=bool(t % 2))
        P, _ = oracle_pattern(A)
        Ad = dense_pattern(A) | np.eye(A.n, dtype=bool)
        assert np.all(P[Ad])
        At = csr_from_dense(dense_pattern(A).T)
        Pt, _ = oracle_pattern(At)
        assert np.array_equal(Pt, P.T)


def test_no_fill_cases():
    n = 40
    rng = np.random.default_rng(7)
    low = np.tril(rng.random((n, n)) < 0.3) | np.eye(n, dtype=bool)
    for M in (low, low.T):
        P, _ = oracle_pattern(csr_from_dense(M))
        assert np.array_equal(P, M)
    tri = np.eye(n, dtype=bool) | np.eye(n, k=1, dtype=bool) | np.eye(n, k=-1, dtype=bool)
    P, _ = oracle_pattern(csr_from_dense(tri))
    assert np.array_equal(P, tri)
    rev = np.eye(n, dtype=bool)
    rev[-1, :] = True
    rev[:, -1] = True
    P, _ = oracle_pattern(csr_from_dense(rev))
    assert np.array_equal(P, rev)


def test_dense_fill_cases():
    n = 30
    arrow = np.eye(n, dtype=bool)
    arrow[0, :] = True
    arrow[:, 0] = True
    P, _ = oracle_pattern(csr_from_dense(arrow))
    assert P.all()
    P, _ = oracle_pattern(csr_from_dense(np.ones((n, n), bool)))
    assert P.all()


def test_symmetric_matches_elimination_tree():
    for t in range(25):
        A0 = synth.random_pattern(60, 0.04, seed=300 + t)
        S = dense_pattern(A0)
        S = S | S.T | np.eye(A0.n, dtype=bool)
        A = csr_from_dense(S)
        r = oracle.symbolic(A)
        rows = etree_cholesky_rows(A)
        P, _ = oracle_pattern(A)
        assert np.array_equal(np.tril(P, -1), np.triu(P, 1).T)   # L = U^T off the diagonal
        for i in range(A.n):
            assert r["L_colidx"][r["L_rowptr"][i]:r["L_rowptr"][i + 1]].tolist() == rows[i]
    A = synth.grid2d(20, 1.0, 0)
    rows = etree_cholesky_rows(A)
    r = oracle.symbolic(A)
    for i in range(A.n):
        assert r["L_colidx"][r["L_rowptr"][i]:r["L_rowptr"][i + 1]].tolist() == rows[i]


def test_numeric_lu_mod_prime():
    for t in range(12):
        A = synth.random_pattern(14, 0.15, seed=40 + t)
        P, _ = oracle_pattern(A)
        N = numeric_lu_pattern_modp(A, seed=t)
        assert np.all(P[N])            # numeric pattern is always inside the symbolic one
        assert np.array_equal(P, N)    # and equal to it with overwhelming probability


# -------------------------------------------------------------- supernodes --

def test_supernodes_vs_dense_t3():
    for t in range(40):
        n = 30 + t
        A = synth.random_pattern(n, 0.08, seed=2000 + t)
        r = oracle.full(A, chunk=16)
        P = brute_ge(A)
        assert r["super_start"].tolist() == t3_supernodes_dense(P, chunk=16)


def test_supernode_rows_share_structure():
    A = synth.grid2d(24, 0.8, seed=11)
    r = oracle.full(A)
    U = [set(r["U_colidx"][r["U_rowptr"][i]:r["U_rowptr"][i + 1]].tolist()) for i in range(A.n)]
    ss = r["super_start"]
    assert ss[0] == 0 and ss[-1] == A.n and np.all(np.diff(ss) > 0) and np.all(np.diff(ss) <= 128)
    for a, b in zip(ss[:-1], ss[1:]):
        assert a // 128 == (b - 1) // 128           # no supernode crosses a chunk boundary
        for s in range(a + 1, b):
            assert U[s] == U[s - 1] - {s - 1}


def test_fill_count():
    A, _ = load_paper_example()
    r = oracle.full(A)
    # row 8: 3 fills; row 1: 1 fill (1,5); row 0 none
    assert r["fill_count"][8] == 3 and r["fill_count"][1] == 1 and r["fill_count"][0] == 0
    A = synth.random_pattern(30, 0.1, seed=5, diag=False)
    r = oracle.full(A)
    P = brute_ge(A)
    Ad = dense_pattern(A) | np.eye(A.n, dtype=bool)
    assert np.array_equal(r["fill_count"], (P & ~Ad).sum(axis=1))


def test_empty_and_tiny():
    A = synth.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32))
    r = oracle.full(A)
    assert r["super_start"].tolist() == [0]
    A = synth.CSR(1, np.array([0, 0], np.int32), np.zeros(0, np.int32))
    r = oracle.full(A)
    assert r["U_colidx"].tolist() == [0] and r["L_colidx"].size == 0


def test_row_subset_matches_full():
    A = synth.config(0)
    full = oracle.symbolic(A, nthreads=4)
    rows = np.array([4095, 0, 17, 2048, 1000], np.int32)
    sub = oracle.symbolic(A, rows=rows)
    for q, i in enumerate(rows):
        assert sub["L_colidx"][sub["L_rowptr"][q]:sub["L_rowptr"][q + 1]].tolist() == \
            full["L_colidx"][full["L_rowptr"][i]:full["L_rowptr"][i + 1]].tolist()
        assert sub["U_colidx"][sub["U_rowptr"][q]:sub["U_rowptr"][q + 1]].tolist() == \
            full["U_colidx"][full["U_rowptr"][i]:full["U_rowptr"][i + 1]].tolist()


def _reach_below(A, i):
    """Vertices below i that a search from row i can pass through: reachable
    from i when only vertices below i may be intermediates (plain graph search)."""
    seen = set(int(w) for w in A.colidx[A.rowptr[i]:A.rowptr[i + 1]] if w != i)
    stack = [w for w in seen if w < i]
    reach = set(stack)
    while stack:
        v = stack.pop()
        for w in A.colidx[A.rowptr[v]:A.rowptr[v + 1]]:
            w = int(w)
            if w == i or w in seen:
                continue
            seen.add(w)
            if w < i:
                reach.add(w)
                stack.append(w)
    return reach


def test_scan_counts_are_the_reach_below_the_row():
    """The per-row work counts behind the roofline's algorithmic bytes:
    V_scan(i) = |reach below i| (each such vertex is expanded exactly once by the
    label-ordered search) and E_scan(i) = the sum of their row lengths; the L row
    is a subset of that reach."""
    cases = [synth.random_pattern(n, d, seed=900 + n, diag=bool(n % 2))
             for n, d in ((12, 0.2), (30, 0.08), (45, 0.05), (60, 0.03))]
    cases += [synth.grid2d(7, 0.7, seed=3), synth.banded(80, 6, seed=4), load_paper_example()[0]]
    for A in cases:
        o = oracle.symbolic(A)
        deg = np.diff(A.rowptr)
        for i in range(A.n):
            R = _reach_below(A, i)
            assert o["vscan"][i] == len(R), (A.name, i)
            assert o["escan"][i] == int(sum(deg[v] for v in R)), (A.name, i)
            Li = set(o["L_colidx"][o["L_rowptr"][i]:o["L_rowptr"][i + 1]].tolist())
            assert Li <= R
