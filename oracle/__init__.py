"""CPU oracle for gSoFa symbolic LU (arXiv 2007.00840).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA path.

Functions
---------
``symbolic(A, rows=None, nthreads=1)``
    Per-row L/U patterns by the minimax-label (fill2 / bottleneck Dijkstra)
    search of ``oracle.c`` - Theorem 1 (Section 2.1) written out per row.
``supernodes(nnzU, L_rowptr, L_colidx, chunk=128)``
    Greedy T3 partition (Definition 1, Section 2.2; chunk-limited as in
    Section 5).
``fill_count(A, nnzL, nnzU)``
    Entries of row i of L+U that are not in A (the emitted diagonal counts as
    present): nnzL + nnzU - |A(i,:) U {i}|.
``full(A)``
    Everything above for all rows.

Parity is pinned by the ``-m "not gpu"`` tests: boolean Gaussian elimination
by brute force, the paper's worked example, a closed form for the full grid,
invariants (containment, transposition, triangular/arrowhead/dense cases) and
the elimination-tree structure of symmetric patterns.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32 = ctypes.c_int32
            lib.oracle_run.restype = P
            lib.oracle_run.argtypes = [i32, P, P, i32, P, i32]
            lib.oracle_counts.restype = None
            lib.oracle_counts.argtypes = [P, P, P, P, P]
            lib.oracle_rows.restype = None
            lib.oracle_rows.argtypes = [P, P, P, P, P]
            lib.oracle_free.restype = None
            lib.oracle_free.argtypes = [P]
            lib.oracle_supernodes.restype = i32
            lib.oracle_supernodes.argtypes = [i32, P, P, P, i32, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr_arrays(A):
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(A.colidx, dtype=np.int32)
    if colidx.size == 0:
        colidx = np.zeros(1, dtype=np.int32)
    return int(A.n), rowptr, colidx


def symbolic(A, rows=None, nthreads: int = 1) -> dict:
    """L/U patterns of the requested rows (default: all rows, in order).

    Returns a dict with int64 ``L_rowptr``/``U_rowptr`` (len(rows)+1), int32
    ``L_colidx``/``U_colidx`` (sorted per row, U holds the diagonal), int32
    ``nnzL``/``nnzU`` and int64 ``vscan``/``escan`` per requested row.
    """
    lib = _load()
    n, rowptr, colidx = _csr_arrays(A)
    if rows is None:
        rows = np.arange(n, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    m = int(rows.size)
    h = lib.oracle_run(n, _ptr(rowptr), _ptr(colidx), m, _ptr(rows if m else np.zeros(1, np.int32)),
                       int(max(1, nthreads)))
    if not h:
        raise MemoryError("oracle_run failed")
    try:
        nnzL = np.zeros(max(m, 1), np.int32)
        nnzU = np.zeros(max(m, 1), np.int32)
        vscan = np.zeros(max(m, 1), np.int64)
        escan = np.zeros(max(m, 1), np.int64)
        lib.oracle_counts(h, _ptr(nnzL), _ptr(nnzU), _ptr(vscan), _ptr(escan))
        nnzL, nnzU, vscan, escan = nnzL[:m], nnzU[:m], vscan[:m], escan[:m]
        Lptr = np.zeros(m + 1, np.int64)
        Uptr = np.zeros(m + 1, np.int64)
        Lcol = np.zeros(max(int(nnzL.sum()), 1), np.int32)
        Ucol = np.zeros(max(int(nnzU.sum()), 1), np.int32)
        lib.oracle_rows(h, _ptr(Lptr), _ptr(Lcol), _ptr(Uptr), _ptr(Ucol))
    finally:
        lib.oracle_free(h)
    return {
        "rows": rows, "L_rowptr": Lptr, "L_colidx": Lcol[:int(Lptr[-1])],
        "U_rowptr": Uptr, "U_colidx": Ucol[:int(Uptr[-1])],
        "nnzL": nnzL, "nnzU": nnzU, "vscan": vscan, "escan": escan,
    }


def supernodes(nnzU, L_rowptr, L_colidx, chunk: int = 128) -> np.ndarray:
    """T3 supernode partition: int32 array of supernode first rows, then n."""
    lib = _load()
    nnzU = np.ascontiguousarray(nnzU, dtype=np.int32)
    n = int(nnzU.size)
    Lptr = np.ascontiguousarray(L_rowptr, dtype=np.int64)
    Lcol = np.ascontiguousarray(L_colidx, dtype=np.int32)
    if Lcol.size == 0:
        Lcol = np.zeros(1, np.int32)
    out = np.zeros(n + 1, np.int32)
    ns = lib.oracle_supernodes(n, _ptr(nnzU if n else np.zeros(1, np.int32)), _ptr(Lptr),
                               _ptr(Lcol), int(chunk), _ptr(out))
    return out[:ns + 1].copy()


def fill_count(A, nnzL, nnzU) -> np.ndarray:
    """nnzL + nnzU - |A(i,:) U {i}| for every row."""
    n = int(A.n)
    deg = np.diff(np.asarray(A.rowptr, dtype=np.int64))
    has_diag = np.zeros(n, bool)
    r = np.repeat(np.arange(n), deg)
    has_diag[r[np.asarray(A.colidx) == r]] = True
    a = deg + (~has_diag).astype(np.int64)
    return (np.asarray(nnzL, np.int64) + np.asarray(nnzU, np.int64) - a).astype(np.int32)


def full(A, nthreads: int = 1, chunk: int = 128) -> dict:
    """All rows: L/U CSR, counts, fill counts, supernodes, scan statistics."""
    r = symbolic(A, None, nthreads)
    r["fill_count"] = fill_count(A, r["nnzL"], r["nnzU"])
    r["super_start"] = supernodes(r["nnzU"], r["L_rowptr"], r["L_colidx"], chunk)
    r["n"] = int(A.n)
    return r
