"""Helpers for the GPU parity tests: run the CUDA path and compare with the oracle."""
from __future__ import annotations

import numpy as np

import oracle


def to_device(A):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.rowptr)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.colidx)).cuda())


def run_gpu(A, **opt):
    import torch
    import paper_2007_00840_gb300 as gs
    rp, ci = to_device(A)
    r = gs.symbolic_device(rp, ci, opts=gs.options(**opt) if opt else None)
    torch.cuda.synchronize()
    return r.to_host()


def host_cores() -> int:
    import os
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def oracle_full(A, nthreads=8):
    return oracle.full(A, nthreads=nthreads)


_ORACLE_CACHE = {}


def oracle_full_cached(key, A):
    """oracle.full(A) on all host cores, kept for the session under `key` (the
    batch and served tests compare the same seeded patterns)."""
    r = _ORACLE_CACHE.get(key)
    if r is None:
        r = oracle.full(A, nthreads=host_cores())
        _ORACLE_CACHE[key] = r
    return r


def assert_rows_equal(h, o, rows=None):
    """Bit-exact comparison of L/U rows (all rows, or the oracle's row subset)."""
    if rows is None:
        assert np.array_equal(h.L_rowptr, o["L_rowptr"]), "L_rowptr"
        assert np.array_equal(h.U_rowptr, o["U_rowptr"]), "U_rowptr"
        assert np.array_equal(h.L_colidx, o["L_colidx"]), "L_colidx"
        assert np.array_equal(h.U_colidx, o["U_colidx"]), "U_colidx"
        return
    for q, i in enumerate(rows):
        gl = h.L_colidx[h.L_rowptr[i]:h.L_rowptr[i + 1]]
        ol = o["L_colidx"][o["L_rowptr"][q]:o["L_rowptr"][q + 1]]
        assert np.array_equal(gl, ol), f"L row {i}"
        gu = h.U_colidx[h.U_rowptr[i]:h.U_rowptr[i + 1]]
        ou = o["U_colidx"][o["U_rowptr"][q]:o["U_rowptr"][q + 1]]
        assert np.array_equal(gu, ou), f"U row {i}"


def assert_same(h, o):
    assert_rows_equal(h, o)
    assert np.array_equal(h.fill_count, o["fill_count"]), "fill_count"
    assert np.array_equal(h.super_start, o["super_start"]), "super_start"


def check_supernode_rule(h, chunk=128):
    """The GPU partition obeys T3 on the GPU's own rows (valid at any size)."""
    n = h.n
    ss = h.super_start
    assert ss[0] == 0 and ss[-1] == n and np.all(np.diff(ss) > 0)
    nnzU = np.diff(h.U_rowptr)
    start = np.zeros(n, bool)
    start[ss[:-1]] = True
    r = 0
    for s in range(n):
        if s % chunk == 0 or s == 0:
            assert start[s], s
            r = s
            continue
        Ls = h.L_colidx[h.L_rowptr[s]:h.L_rowptr[s + 1]]
        join = nnzU[s] == nnzU[s - 1] - 1 and np.searchsorted(Ls, r) < Ls.size and Ls[np.searchsorted(Ls, r)] == r
        assert start[s] == (not join), s
        if start[s]:
            r = s
