"""The seeded input generators: workload sizes, structure and determinism.

These hold none of the method's arithmetic; they fix the inputs both the
oracle and the CUDA path are run on, so the workloads stay what the design
states (5-point / 7-point grids, nested dissection, the 512-matrix mix)."""
import numpy as np
import pytest

import synth


def _valid_csr(A):
    rp, ci = A.rowptr, A.colidx
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    assert ci.size == 0 or (ci.min() >= 0 and ci.max() < A.n)
    for i in range(0, A.n, max(1, A.n // 257)):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0), i  # sorted, no duplicates


def _offsets(A):
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return A.colidx.astype(np.int64) - rows


def test_workload_sizes_and_determinism():
    for k, (n, nnz) in enumerate([(4096, 15348), (32768, 180383)]):
        A, B = synth.config(k), synth.config(k)
        assert (A.n, A.nnz) == (n, nnz)
        assert np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.colidx, B.colidx)
        _valid_csr(A)


def test_grid_workloads_structure():
    A = synth.config(0)  # 64 x 64, 5-point, natural order
    off = _offsets(A)
    assert set(np.unique(off).tolist()) <= {-64, -1, 0, 1, 64}
    assert np.count_nonzero(off == 0) == A.n  # every diagonal present
    assert np.count_nonzero(off != 0) < 4 * A.n  # off-diagonals thinned (p = 0.7)
    B = synth.config(1)  # 32^3, 7-point plus one extra entry per row within +-1024
    offb = _offsets(B)
    assert np.count_nonzero(offb == 0) == B.n
    assert np.abs(offb).max() <= 1024
    grid = np.isin(offb, [-1024, -32, -1, 1, 32, 1024])
    assert np.count_nonzero(~grid & (offb != 0)) >= 0.9 * B.n  # the extra entries (rare collisions redrawn)


def test_nested_dissection_permutation():
    k = 40
    perm = synth.nd_permutation(k, leaf=16)
    assert np.array_equal(np.sort(perm), np.arange(k * k))
    # the top separator (the middle column) is numbered last
    mid = (k - 1) // 2
    col = np.arange(k) * k + mid
    assert set(perm[col].tolist()) == set(range(k * k - k, k * k))
    A = synth.grid2d_nd(k, 0.8, seed=1, leaf=16)
    _valid_csr(A)
    assert np.all(np.diff(A.rowptr) <= 5)


@pytest.mark.slow
def test_nd_workload_size():
    A = synth.config(2)
    assert (A.n, A.nnz) == (1048576, 4401650)
    _valid_csr(A)


def test_batch_mix_recipe():
    mats = synth.batch_mix(24, seed=synth.config_seed(3))
    for m, A in enumerate(mats):
        _valid_csr(A)
        assert 500 <= A.n <= 20000
        deg = np.diff(A.rowptr)
        off = _offsets(A)
        assert np.count_nonzero(off == 0) == A.n
        if m % 2 == 1:  # banded: 4-12 entries per row with the diagonal, within the band
            assert deg.max() <= 12 and np.abs(off).max() <= 256
        else:           # near-square grid: 5-point offsets of width ceil(sqrt(n))
            w = int(np.ceil(np.sqrt(A.n)))
            assert set(np.unique(off).tolist()) <= {-w, -1, 0, 1, w}
    full = synth.config(3)
    assert len(full) == 512 and all(500 <= A.n <= 20000 for A in full)
