"""Seeded synthetic sparsity patterns (CSR, int32, pattern only).

This module is the one piece shared by the CPU oracle side and the CUDA side:
it draws input matrices and nothing else.  It contains none of the symbolic
factorisation arithmetic.

Randomness is counter based: every decision is a pure function of
(seed, a, b) through the SplitMix64 finaliser (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), so a pattern
does not depend on the order in which it is built and any single entry can be
recomputed on its own.

Workloads (stand-ins for the paper's SuiteSparse matrices, Table 1, which are
not available here; they span its range of structural symmetry 0-1 and
nnz/n of 4-13):

* ``grid2d(k, p)``          2D 5-point stencil, natural row-major order
* ``grid3d_extra(k, p)``    3D 7-point stencil + one random entry per row
* ``grid2d_nd(k, p)``       2D 5-point stencil renumbered by geometric
                            nested dissection (separators last)
* ``banded(n, b)``          4-12 random entries per row inside a band
* ``near_square_grid(n, p)``  2D grid of width ceil(sqrt(n)), last row partial
* ``batch_mix(count)``      the many-matrix mix (half grids, half banded)
* ``config(k)``             the five benchmark workloads by index
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSR", "splitmix64", "hash3", "unif", "grid2d", "grid3d_extra", "grid2d_nd",
    "nd_permutation", "banded", "near_square_grid", "batch_mix", "random_pattern",
    "config_seed", "config", "CONFIG_NAMES", "served_pool", "served_choices",
]

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


@dataclass
class CSR:
    """Square sparsity pattern in CSR form (int32 row pointers and columns)."""

    n: int
    rowptr: np.ndarray  # int32[n+1]
    colidx: np.ndarray  # int32[nnz], sorted and unique inside each row
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row(self, i: int) -> np.ndarray:
        return self.colidx[self.rowptr[i]:self.rowptr[i + 1]]


def splitmix64(x):
    """SplitMix64 finaliser applied to uint64 values (wraps modulo 2**64)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def hash3(seed: int, a, b):
    """64-bit hash of the counter triple (seed, a, b)."""
    a = np.asarray(a, dtype=np.int64).astype(np.uint64)
    b = np.asarray(b, dtype=np.int64).astype(np.uint64)
    with np.errstate(over="ignore"):
        s = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
        return splitmix64(splitmix64(s ^ a) ^ b)


def unif(seed: int, a, b):
    """Uniform double in [0, 1) from the top 53 bits of ``hash3``."""
    h = hash3(seed, a, b)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def config_seed(k: int) -> int:
    """Seed of workload index k (0-based): golden-ratio constant times (k+1)."""
    return (0x9E3779B97F4A7C15 * (k + 1)) & 0xFFFFFFFFFFFFFFFF


# --------------------------------------------------------------------------
# CSR assembly helpers
# --------------------------------------------------------------------------

def _csr_from_candidates(n: int, cand: np.ndarray, keep: np.ndarray, name: str) -> CSR:
    """Rows given as an (n, m) candidate table already sorted along axis 1."""
    counts = keep.sum(axis=1).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = cand[keep].astype(np.int32)
    return CSR(n, rowptr.astype(np.int32), colidx, name)


def _csr_from_pairs(n: int, rows: np.ndarray, cols: np.ndarray, name: str) -> CSR:
    """Build a CSR from (row, col) pairs, sorting and removing duplicates."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * np.int64(n) + cols
    key = np.unique(key)
    r = key // n
    c = key % n
    counts = np.bincount(r, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr.astype(np.int32), c.astype(np.int32), name)


# --------------------------------------------------------------------------
# Stencil grids
# --------------------------------------------------------------------------

def grid2d(k: int, p: float, seed: int, name: str = "") -> CSR:
    """k x k 5-point stencil, vertex v = y*k + x (natural row-major order).

    The diagonal is always present; every directed off-diagonal stencil entry
    (v, w) is kept independently iff unif(seed, v, w) < p, so the pattern is
    structurally nonsymmetric for p < 1.
    """
    n = k * k
    v = np.arange(n, dtype=np.int64)
    x, y = v % k, v // k
    offs = [(-k, y > 0), (-1, x > 0), (0, np.ones(n, bool)), (1, x < k - 1), (k, y < k - 1)]
    cand = np.stack([v + o for o, _ in offs], axis=1)
    exists = np.stack([m for _, m in offs], axis=1)
    keep = exists.copy()
    off = np.ones_like(exists)
    off[:, 2] = False
    u = unif(seed, np.broadcast_to(v[:, None], cand.shape), np.where(exists, cand, 0))
    keep &= (~off) | (u < p)
    return _csr_from_candidates(n, cand, keep, name or f"grid2d_{k}x{k}_p{p}")


def grid3d_extra(k: int, p: float, seed: int, extra_range: int = 1024, tries: int = 64,
                 name: str = "") -> CSR:
    """k^3 7-point stencil (v = x + k*y + k*k*z) plus one extra entry per row.

    Diagonal always present; each directed off-diagonal stencil entry kept iff
    unif(seed, v, w) < p.  The extra entry sits at offset d drawn uniformly
    from [-extra_range, extra_range] \\ {0}; a draw that falls outside [0, n) or
    onto an entry already present is redrawn with the next counter, up to
    ``tries`` times (counter c uses hash3(seed ^ 0x5EED, v, c)).
    """
    n = k * k * k
    v = np.arange(n, dtype=np.int64)
    x, y, z = v % k, (v // k) % k, v // (k * k)
    kk = k * k
    offs = [(-kk, z > 0), (-k, y > 0), (-1, x > 0), (0, np.ones(n, bool)),
            (1, x < k - 1), (k, y < k - 1), (kk, z < k - 1)]
    cand = np.stack([v + o for o, _ in offs], axis=1)
    exists = np.stack([m for _, m in offs], axis=1)
    off = np.ones_like(exists)
    off[:, 3] = False
    u = unif(seed, np.broadcast_to(v[:, None], cand.shape), np.where(exists, cand, 0))
    keep = exists & ((~off) | (u < p))

    # extra entry: first valid draw among `tries` counters
    span = 2 * extra_range
    c = np.arange(tries, dtype=np.int64)
    h = hash3(seed ^ 0x5EED, np.broadcast_to(v[:, None], (n, tries)),
              np.broadcast_to(c[None, :], (n, tries)))
    r = (h % np.uint64(span)).astype(np.int64)           # 0 .. span-1
    d = np.where(r < extra_range, r - extra_range, r - extra_range + 1)
    col = v[:, None] + d
    valid = (col >= 0) & (col < n)
    present = np.zeros((n, tries), bool)
    for j in range(cand.shape[1]):
        present |= keep[:, j:j + 1] & (cand[:, j:j + 1] == col)
    valid &= ~present
    has = valid.any(axis=1)
    first = np.argmax(valid, axis=1)
    extra = col[np.arange(n), first]

    rows = np.concatenate([np.broadcast_to(v[:, None], cand.shape)[keep], v[has]])
    cols = np.concatenate([cand[keep], extra[has]])
    return _csr_from_pairs(n, rows, cols, name or f"grid3d_{k}^3_p{p}_extra{extra_range}")


def nd_permutation(k: int, leaf: int = 64) -> np.ndarray:
    """Geometric nested dissection of a k x k grid.

    Returns perm with perm[original] = new index, original = y*k + x.
    A box is split along its longer side (x on a tie) at
    mid = lo + (len - 1) // 2; the low half is numbered first, then the high
    half, then the separator line (in increasing coordinate order).  Boxes with
    at most ``leaf`` vertices are numbered row-major.
    """
    perm = np.empty(k * k, dtype=np.int64)
    nxt = [0]

    def number(ids: np.ndarray) -> None:
        m = ids.size
        perm[ids] = np.arange(nxt[0], nxt[0] + m)
        nxt[0] += m

    def rec(x0: int, x1: int, y0: int, y1: int) -> None:
        w, h = x1 - x0, y1 - y0
        if w <= 0 or h <= 0:
            return
        if w * h <= leaf:
            ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
            number((ys * k + xs).ravel())
            return
        if w >= h:
            mid = x0 + (w - 1) // 2
            rec(x0, mid, y0, y1)
            rec(mid + 1, x1, y0, y1)
            number(np.arange(y0, y1, dtype=np.int64) * k + mid)
        else:
            mid = y0 + (h - 1) // 2
            rec(x0, x1, y0, mid)
            rec(x0, x1, mid + 1, y1)
            number(mid * k + np.arange(x0, x1, dtype=np.int64))

    rec(0, k, 0, k)
    assert nxt[0] == k * k
    return perm


def grid2d_nd(k: int, p: float, seed: int, leaf: int = 64, name: str = "") -> CSR:
    """k x k 5-point stencil renumbered by geometric nested dissection.

    Entries are kept by the hash of the ORIGINAL grid pair (so the kept set
    does not depend on the ordering), then both indices are permuted.
    """
    n = k * k
    o = np.arange(n, dtype=np.int64)
    x, y = o % k, o // k
    offs = [(-k, y > 0), (-1, x > 0), (1, x < k - 1), (k, y < k - 1)]
    rows = [o]
    cols = [o]
    for dv, m in offs:
        w = o + dv
        keep = m & (unif(seed, o, np.where(m, w, 0)) < p)
        rows.append(o[keep])
        cols.append(w[keep])
    perm = nd_permutation(k, leaf)
    r = perm[np.concatenate(rows)]
    c = perm[np.concatenate(cols)]
    return _csr_from_pairs(n, r, c, name or f"grid2d_nd_{k}x{k}_p{p}")


def near_square_grid(n: int, p: float, seed: int, name: str = "") -> CSR:
    """5-point stencil on a grid of width w = ceil(sqrt(n)), row-major, last row partial."""
    w = int(math.ceil(math.sqrt(n)))
    v = np.arange(n, dtype=np.int64)
    x = v % w
    offs = [(-w, v - w >= 0), (-1, x > 0), (0, np.ones(n, bool)),
            (1, (x < w - 1) & (v + 1 < n)), (w, v + w < n)]
    cand = np.stack([v + o for o, _ in offs], axis=1)
    exists = np.stack([m for _, m in offs], axis=1)
    off = np.ones_like(exists)
    off[:, 2] = False
    u = unif(seed, np.broadcast_to(v[:, None], cand.shape), np.where(exists, cand, 0))
    keep = exists & ((~off) | (u < p))
    return _csr_from_candidates(n, cand, keep, name or f"nsgrid_{n}_p{p}")


def banded(n: int, b: int, seed: int, kmin: int = 4, kmax: int = 12, tries: int = 32,
           name: str = "") -> CSR:
    """Banded random pattern: row i holds the diagonal plus k-1 distinct entries.

    k ~ U{kmin..kmax} (k counts the diagonal).  Off-diagonal columns are drawn
    with counters c = 0..tries-1 as i + d, d uniform in [-b, b]; draws that
    leave [0, n), hit the diagonal or repeat an earlier draw are skipped; the
    first k-1 accepted draws are kept (rows near the matrix edge may get fewer).
    """
    v = np.arange(n, dtype=np.int64)
    kk = kmin + (hash3(seed ^ 0xB0, v, 0) % np.uint64(kmax - kmin + 1)).astype(np.int64)
    c = np.arange(tries, dtype=np.int64)
    h = hash3(seed ^ 0xB1, np.broadcast_to(v[:, None], (n, tries)),
              np.broadcast_to(c[None, :], (n, tries)))
    d = (h % np.uint64(2 * b + 1)).astype(np.int64) - b
    col = v[:, None] + d
    ok = (col >= 0) & (col < n) & (d != 0)
    # first occurrence of each column inside the row
    order = np.argsort(col, axis=1, kind="stable")
    sc = np.take_along_axis(col, order, axis=1)
    dup_sorted = np.zeros_like(ok)
    dup_sorted[:, 1:] = sc[:, 1:] == sc[:, :-1]
    dup = np.zeros_like(ok)
    np.put_along_axis(dup, order, dup_sorted, axis=1)
    acc = ok & ~dup
    cum = np.cumsum(acc, axis=1)
    take = acc & (cum <= (kk - 1)[:, None])
    rows = np.concatenate([v, np.broadcast_to(v[:, None], (n, tries))[take]])
    cols = np.concatenate([v, col[take]])
    return _csr_from_pairs(n, rows, cols, name or f"banded_{n}_b{b}")


def batch_mix(count: int, seed: int, n_lo: int = 500, n_hi: int = 20000) -> list:
    """The many-matrix mix: n log-uniform in [n_lo, n_hi]; even m -> grid, odd m -> banded.

    Grids: near-square 5-point, natural order, p = 0.7.  Banded: bandwidth
    log-uniform in [8, 256], 4-12 entries per row including the diagonal.
    Matrix m uses sub-seed hash3(seed, m, 7).
    """
    out = []
    for m in range(count):
        u = float(unif(seed, m, 1))
        n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
        sub = int(hash3(seed, m, 7))
        if m % 2 == 0:
            out.append(near_square_grid(n, 0.7, sub, name=f"mix{m}_grid{n}"))
        else:
            ub = float(unif(seed, m, 2))
            b = int(round(math.exp(math.log(8) + ub * (math.log(256) - math.log(8)))))
            out.append(banded(n, b, sub, name=f"mix{m}_band{n}_b{b}"))
    return out


def random_pattern(n: int, density: float, seed: int, diag: bool = True) -> CSR:
    """Dense-table random pattern for small tests: (i, j) kept iff unif < density."""
    i = np.repeat(np.arange(n, dtype=np.int64), n)
    j = np.tile(np.arange(n, dtype=np.int64), n)
    keep = unif(seed, i, j) < density
    if diag:
        keep |= i == j
    return _csr_from_pairs(n, i[keep], j[keep], f"rand_{n}_{density}")


CONFIG_NAMES = [
    "grid2d_64x64_p0.7",
    "grid3d_32^3_p0.6_extra1024",
    "grid2d_nd_1024x1024_p0.8",
    "batch512_mix",
    "served_poisson_mix",
]


def config(k: int):
    """Workload k (0-based): 0,1,2 -> CSR; 3 -> list of 512 CSR."""
    s = config_seed(k)
    if k == 0:
        return grid2d(64, 0.7, s, name=CONFIG_NAMES[0])
    if k == 1:
        return grid3d_extra(32, 0.6, s, 1024, name=CONFIG_NAMES[1])
    if k == 2:
        return grid2d_nd(1024, 0.8, s, name=CONFIG_NAMES[2])
    if k == 3:
        return batch_mix(512, s)
    raise ValueError("workload 4 is a request stream; see served_request()")


def served_request(idx: int, big_n_side: int = 512, big_frac: float = 0.02, seed: int | None = None) -> CSR:
    """Request ``idx`` of the served stream: the batch mix w.p. 1-big_frac, else an ND grid.

    Per-request seed is derived from the request index.
    """
    s = config_seed(4) if seed is None else seed
    u = float(unif(s, idx, 11))
    sub = int(hash3(s, idx, 12))
    if u < big_frac:
        return grid2d_nd(big_n_side, 0.8, sub, name=f"req{idx}_nd{big_n_side}")
    m = int(hash3(s, idx, 13) % np.uint64(1 << 30))
    return batch_mix_one(m, sub)


def served_pool(big_count: int = 4, big_n_side: int = 512):
    """Finite pool behind the served request stream: the 512-matrix mix (drawn
    with probability 0.98) and ``big_count`` ND grids of side ``big_n_side``
    (probability 0.02).  Returns (small, big), two lists of CSR."""
    small = config(3)
    big = [grid2d_nd(big_n_side, 0.8, seed=config_seed(4) + j, name=f"served_nd{big_n_side}_{j}")
           for j in range(big_count)]
    return small, big


def served_choices(count: int, n_small: int, n_big: int, seed: int = 4, big_frac: float = 0.02):
    """Pool index of each of ``count`` requests (small pool first, then big) and
    the Poisson arrival offsets in units of the mean inter-arrival time."""
    rng = np.random.default_rng(seed)
    which = np.where(rng.random(count) < big_frac, n_small + rng.integers(0, n_big, count),
                     rng.integers(0, n_small, count))
    arrivals = np.cumsum(rng.exponential(1.0, count))
    return which, arrivals


def batch_mix_one(m: int, seed: int, n_lo: int = 500, n_hi: int = 20000) -> CSR:
    """One member of the mix with its own seed (parity of m picks grid or banded)."""
    u = float(unif(seed, m, 1))
    n = int(round(math.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))))
    sub = int(hash3(seed, m, 7))
    if m % 2 == 0:
        return near_square_grid(n, 0.7, sub, name=f"grid{n}")
    ub = float(unif(seed, m, 2))
    b = int(round(math.exp(math.log(8) + ub * (math.log(256) - math.log(8)))))
    return banded(n, b, sub, name=f"band{n}_b{b}")
