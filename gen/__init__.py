"""Seeded synthetic CSR inputs shared by the oracle tests, the GPU tests and the benchmark.

This module draws random structure and values only; it holds none of the
SpGEMM arithmetic.  Every generator is deterministic in its seed (numpy PCG64),
so the same arrays come out on x86 and on Arm.

Workloads (the paper evaluates on SuiteSparse / HipMCL matrices, Table 2, which
are not available here; these synthetic matrices stand in for them):

* ``er``: Erdos-Renyi, exactly ``d`` distinct uniform-random columns per row.
* ``er_batch``: many independent ER products, n log-uniform, d uniform.
* ``rmat``: R-MAT graph (recursive quadrant choice), randomly permuted,
  symmetrised, self-loops added, duplicates removed, column-stochastic.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Host CSR matrix: int64 row pointers, int32 column indices (sorted and
    duplicate-free within each row), float32/float64 values."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def astype(self, dtype) -> "CSR":
        return CSR(self.nrows, self.ncols, self.rowptr, self.col, self.val.astype(dtype))

    def with_values(self, val: np.ndarray) -> "CSR":
        assert val.shape == self.col.shape
        return CSR(self.nrows, self.ncols, self.rowptr, self.col, val)

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.nrows, self.ncols), dtype=np.float64)
        rows = np.repeat(np.arange(self.nrows), self.row_lengths())
        np.add.at(out, (rows, self.col.astype(np.int64)), self.val.astype(np.float64))
        return out

    def sha256(self) -> str:
        h = hashlib.sha256()
        for a in (self.rowptr.astype(np.int64), self.col.astype(np.int32), self.val):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


def from_coo(nrows: int, ncols: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Build a canonical CSR from coordinates that are already duplicate-free."""
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    vals = vals[order]
    counts = np.bincount(rows, minlength=nrows)
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(nrows, ncols, rowptr, cols, vals)


def from_dense(dense: np.ndarray, dtype=np.float64) -> CSR:
    rows, cols = np.nonzero(dense)
    return from_coo(dense.shape[0], dense.shape[1], rows, cols, dense[rows, cols].astype(dtype))


def _distinct_columns(rng: np.random.Generator, nrows: int, ncols: int, d: int) -> np.ndarray:
    """``nrows x d`` array, each row ``d`` distinct columns in [0, ncols), sorted.

    Draws ``d`` uniform columns per row and redraws every repeated entry until
    each row is duplicate-free (rejection of repeats, which leaves every
    d-subset equally likely)."""
    if d > ncols:
        raise ValueError(f"d={d} > ncols={ncols}")
    if d == 0 or nrows == 0:
        return np.zeros((nrows, d), dtype=np.int32)
    if 2 * d > ncols:
        # dense regime: a random permutation prefix per row
        keys = rng.random((nrows, ncols))
        cols = np.argpartition(keys, d - 1, axis=1)[:, :d]
        cols.sort(axis=1)
        return cols.astype(np.int32)
    cols = rng.integers(0, ncols, size=(nrows, d), dtype=np.int64)
    while True:
        cols.sort(axis=1)
        dup = np.zeros(cols.shape, dtype=bool)
        dup[:, 1:] = cols[:, 1:] == cols[:, :-1]
        nd = int(dup.sum())
        if nd == 0:
            return cols.astype(np.int32)
        cols[dup] = rng.integers(0, ncols, size=nd, dtype=np.int64)


def _values(rng: np.random.Generator, size: int, dtype, values: str) -> np.ndarray:
    if values == "uniform":
        return rng.uniform(-1.0, 1.0, size=size).astype(dtype)
    if values == "normal":
        return rng.standard_normal(size=size).astype(dtype)
    if values == "int":
        # small integers: every product and every sum of a few thousand of
        # them is exact in float32 and float64
        return rng.integers(-3, 4, size=size).astype(dtype)
    if values == "ones":
        return np.ones(size, dtype=dtype)
    raise ValueError(values)


def er(nrows: int, ncols: int, d: int, seed: int, dtype=np.float64, values: str = "uniform") -> CSR:
    """Erdos-Renyi CSR: exactly ``d`` distinct uniform-random columns per row."""
    rng = np.random.default_rng(seed)
    cols = _distinct_columns(rng, nrows, ncols, d).reshape(-1)
    vrng = np.random.default_rng([seed, 0x5EED])
    val = _values(vrng, cols.size, dtype, values)
    rowptr = np.arange(nrows + 1, dtype=np.int64) * d
    return CSR(nrows, ncols, rowptr, cols, val)


def er_variable(nrows: int, ncols: int, dmax: int, seed: int, dtype=np.float64,
                values: str = "uniform", p_empty: float = 0.0) -> CSR:
    """ER-like CSR with a row length drawn uniformly from [0, dmax] per row
    (plus a fraction ``p_empty`` of forced-empty rows): ragged test input."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, dmax + 1, size=nrows)
    if p_empty > 0:
        lens[rng.random(nrows) < p_empty] = 0
    lens = np.minimum(lens, ncols)
    cols = []
    for L in np.unique(lens):
        idx = np.nonzero(lens == L)[0]
        cols.append((idx, _distinct_columns(rng, idx.size, ncols, int(L))))
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(lens, out=rowptr[1:])
    col = np.zeros(int(rowptr[-1]), dtype=np.int32)
    for idx, c in cols:
        if c.shape[1] == 0:
            continue
        pos = rowptr[idx][:, None] + np.arange(c.shape[1])[None, :]
        col[pos.reshape(-1)] = c.reshape(-1)
    vrng = np.random.default_rng([seed, 0x5EED])
    val = _values(vrng, col.size, dtype, values)
    return CSR(nrows, ncols, rowptr, col, val)


def er_batch_shapes(count: int = 256, seed: int = 999, log2_lo: float = 10.0, log2_hi: float = 16.0,
                    d_lo: int = 4, d_hi: int = 64):
    """(n, d) per independent product: n = round(2**U(lo, hi)), d ~ U{d_lo..d_hi}."""
    rng = np.random.default_rng(seed)
    n = np.rint(2.0 ** rng.uniform(log2_lo, log2_hi, size=count)).astype(np.int64)
    d = rng.integers(d_lo, d_hi + 1, size=count)
    return [(int(a), int(b)) for a, b in zip(n, d)]


def er_batch(count: int = 256, seed: int = 999, dtype=np.float64, values: str = "uniform",
             log2_lo: float = 10.0, log2_hi: float = 16.0):
    """``count`` independent square ER products A_t, B_t (seeds 1000+2t, 1000+2t+1)."""
    out = []
    for t, (n, d) in enumerate(er_batch_shapes(count, seed, log2_lo, log2_hi)):
        A = er(n, n, d, 1000 + 2 * t, dtype, values)
        B = er(n, n, d, 1000 + 2 * t + 1, dtype, values)
        out.append((A, B))
    return out


def rmat_edges(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int):
    """Directed R-MAT edge list: each edge picks one quadrant per level with
    probabilities (a, b, c, d=1-a-b-c); no noise."""
    rng = np.random.default_rng(seed)
    m = edge_factor << scale
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    for _ in range(scale):
        u = rng.random(m)
        down = u >= a + b            # quadrants c, d: row bit 1
        right = ((u >= a) & (u < a + b)) | (u >= a + b + c)  # quadrants b, d: col bit 1
        src = (src << 1) | down
        dst = (dst << 1) | right
    return src, dst


def rmat_stochastic(scale: int = 20, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
                    c: float = 0.19, seed: int = 3, dtype=np.float32) -> CSR:
    """Column-stochastic R-MAT matrix stored TRANSPOSED (row r of the CSR is
    column r of the Markov matrix M): random vertex permutation, symmetrise,
    add self-loops, drop duplicates, unit weights, normalise each column."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, a, b, c, seed)
    perm = np.random.default_rng([seed, 0xBEEF]).permutation(n)
    src, dst = perm[src], perm[dst]
    loops = np.arange(n, dtype=np.int64)
    r = np.concatenate([src, dst, loops])
    q = np.concatenate([dst, src, loops])
    key = np.unique(r * n + q)
    rows = key // n
    cols = key % n
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    # symmetric pattern: column sums of M equal row sums of M^T
    val = (1.0 / np.repeat(counts, counts)).astype(dtype)
    return CSR(n, n, rowptr, cols.astype(np.int32), val)


def random_dense_weights(csr: CSR, seed: int, dtype=np.float32) -> np.ndarray:
    """N(0,1) weights on a given pattern (the loss weights W of the autograd check)."""
    return np.random.default_rng([seed, 0x3E16]).standard_normal(csr.nnz).astype(dtype)


def identity(n: int, dtype=np.float64) -> CSR:
    return CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n, dtype=dtype))


def permutation_matrix(perm: np.ndarray, dtype=np.float64) -> CSR:
    """P with P[i, perm[i]] = 1, so (P @ X)[i] = X[perm[i]]."""
    n = perm.size
    return CSR(n, n, np.arange(n + 1, dtype=np.int64), perm.astype(np.int32), np.ones(n, dtype=dtype))


def aggregation(n: int, ratio: int, seed: int, dtype=np.float64) -> CSR:
    """Unsmoothed-aggregation restriction operator R (n x ceil(n / ratio)) of
    an algebraic-multigrid setup: a seeded permutation assigns node i to
    aggregate perm[i] // ratio, so every aggregate holds ``ratio`` nodes (the
    last one the remainder), and R[i, aggregate(i)] = 1: one entry per row.
    C = A R then adds, per row of A, the entries whose columns share an
    aggregate."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    ncols = -(-n // ratio)
    cols = (perm // ratio).astype(np.int32)
    return CSR(n, ncols, np.arange(n + 1, dtype=np.int64), cols, np.ones(n, dtype=dtype))


def banded(n: int, offsets, half_width: int, seed: int, dtype=np.float64, values: str = "uniform") -> CSR:
    """A structured matrix of diagonal bands: row i holds the columns
    i + o + w for every offset o in ``offsets`` and w in [-half_width,
    half_width] that fall inside [0, n), deduplicated (the kind of
    multi-band pattern whose 2D tiles are very uneven).  Values from a seeded
    stream."""
    offs = np.unique(np.asarray(offsets, dtype=np.int64))
    w = np.arange(-half_width, half_width + 1, dtype=np.int64)
    rel = np.unique((offs[:, None] + w[None, :]).reshape(-1))
    rows = np.repeat(np.arange(n, dtype=np.int64), rel.size)
    cols = (np.arange(n, dtype=np.int64)[:, None] + rel[None, :]).reshape(-1)
    keep = (cols >= 0) & (cols < n)
    rows, cols = rows[keep], cols[keep]
    rng = np.random.default_rng([seed, 0xBA7D])
    vals = _values(rng, cols.size, dtype, values)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    np.cumsum(rowptr, out=rowptr)
    return CSR(n, n, rowptr, cols.astype(np.int32), vals)


def random_permutation(n: int, seed: int) -> np.ndarray:
    """A seeded uniform permutation of 0..n-1 (int32)."""
    return np.random.default_rng([seed, 0x9E37]).permutation(n).astype(np.int32)
