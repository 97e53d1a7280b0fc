"""Independent reference routines used by the tests to pin the oracle.

None of these share code with ``oracle/`` or with the CUDA library: each is a
different route to the same fill pattern (or a property of it).
"""
from __future__ import annotations

import os

import numpy as np

from synth import CSR, _csr_from_pairs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------- fixture --

def load_paper_example():
    """Parse tests/golden/paper_example.txt -> (CSR, facts dict)."""
    path = os.path.join(GOLDEN, "paper_example.txt")
    n = None
    rows, cols = [], []
    facts: dict = {"fill": []}
    mode = None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("n "):
                n = int(line.split()[1])
                continue
            if line == "edges":
                mode = "edges"
                continue
            if line == "end":
                mode = None
                continue
            if mode == "edges":
                src, rest = line.split(":")
                for c in rest.split():
                    rows.append(int(src))
                    cols.append(int(c))
                continue
            key, *vals = line.split()
            if key == "fill":
                facts["fill"].append((int(vals[0]), int(vals[1])))
            elif key in ("nnzU", "L_nonzero", "L_zero"):
                facts.setdefault(key, []).append(tuple(int(v) for v in vals))
            elif key.startswith("maxid"):
                facts[key] = {int(a): int(b) for a, b in (v.split(":") for v in vals)}
            elif key == "frontiers":
                facts[key] = [sorted(int(x) for x in v.strip("{}").split(",")) for v in vals]
            else:
                facts[key] = [int(v) for v in vals]
    assert n is not None
    rows += list(range(n))
    cols += list(range(n))
    return _csr_from_pairs(n, np.array(rows), np.array(cols), "paper_example"), facts


# ------------------------------------------------- boolean elimination pin --

def dense_pattern(A: CSR) -> np.ndarray:
    P = np.zeros((A.n, A.n), dtype=bool)
    r = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    P[r, A.colidx] = True
    return P


def brute_ge(A: CSR) -> np.ndarray:
    """Filled pattern by boolean Gaussian elimination without pivoting (Section 2.1).

    Eliminating pivot k applies row k to every later row i with a nonzero in
    column k; row i gains row k's nonzeros right of column k.  Pivots are
    taken as nonzero, so the diagonal is always present.
    """
    P = dense_pattern(A)
    n = A.n
    np.fill_diagonal(P, True)
    for k in range(n):
        tgt = np.nonzero(P[k + 1:, k])[0] + k + 1
        if tgt.size:
            P[np.ix_(tgt, np.arange(k + 1, n))] |= P[k, k + 1:]
    return P


def pattern_from_result(n, L_rowptr, L_colidx, U_rowptr, U_colidx) -> np.ndarray:
    P = np.zeros((n, n), dtype=bool)
    for i in range(n):
        P[i, L_colidx[L_rowptr[i]:L_rowptr[i + 1]]] = True
        P[i, U_colidx[U_rowptr[i]:U_rowptr[i + 1]]] = True
    return P


def t3_supernodes_dense(P: np.ndarray, chunk: int = 128) -> list:
    """Greedy T3 partition from a dense filled pattern (Definition 1)."""
    n = P.shape[0]
    nnzU = [int(P[s, s:].sum()) for s in range(n)]
    starts = []
    r = 0
    for s in range(n):
        join = s > 0 and s % chunk != 0 and nnzU[s] == nnzU[s - 1] - 1 and P[s, r]
        if not join:
            starts.append(s)
            r = s
    return starts + [n]


# ----------------------------------------------------- elimination tree pin --

def etree_cholesky_rows(A: CSR) -> list:
    """Row structures of the Cholesky factor of a symmetric pattern.

    Textbook route (Liu, "The role of elimination trees in sparse
    factorization", 1990): build the elimination tree with path-compressed
    ancestors, then row i of L is the union of the tree paths from each j < i
    with A(i, j) != 0 up towards i.
    """
    n = A.n
    parent = [-1] * n
    ancestor = [-1] * n
    for i in range(n):
        for j in A.row(i):
            j = int(j)
            if j >= i:
                continue
            while j != -1 and j < i:
                nxt = ancestor[j]
                ancestor[j] = i
                if nxt == -1:
                    parent[j] = i
                j = nxt
    rows = []
    mark = [-1] * n
    for i in range(n):
        mark[i] = i
        s = []
        for j in A.row(i):
            j = int(j)
            if j >= i:
                continue
            while mark[j] != i:
                s.append(j)
                mark[j] = i
                j = parent[j]
                if j == -1:
                    break
        rows.append(sorted(s))
    return rows


# ------------------------------------------------ numeric LU (mod prime) pin --

def numeric_lu_pattern_modp(A: CSR, seed: int, p: int = 2_147_483_647) -> np.ndarray:
    """Pattern of L+U from LU without pivoting on random values mod a prime.

    By the Schwartz-Zippel lemma, with random values the numeric pattern equals
    the symbolic one with high probability; it is always a subset of it.
    The diagonal gets values too (nonzero pivots are assumed; a zero pivot
    raises).
    """
    rng = np.random.default_rng(seed)
    n = A.n
    M = np.zeros((n, n), dtype=object)
    P = dense_pattern(A)
    np.fill_diagonal(P, True)
    vals = rng.integers(1, p, size=(n, n))
    for i in range(n):
        for j in range(n):
            if P[i, j]:
                M[i, j] = int(vals[i, j])
    for k in range(n):
        piv = M[k, k] % p
        if piv == 0:
            raise ZeroDivisionError("zero pivot")
        inv = pow(int(piv), p - 2, p)
        for i in range(k + 1, n):
            if M[i, k] % p:
                l = (M[i, k] * inv) % p
                M[i, k] = l
                for j in range(k + 1, n):
                    if M[k, j] % p:
                        M[i, j] = (M[i, j] - l * M[k, j]) % p
    out = np.vectorize(lambda x: x % p != 0)(M).astype(bool)
    np.fill_diagonal(out, True)
    return out
