"""CPU oracle for the trident SpGEMM hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The CUDA library never
imports, links or runs anything here, and this package imports nothing from
the CUDA library; the two share only the seeded input generators in ``gen``.

Contents (each function names the passage of the paper it follows):

* ``spgemm``       C = A B in CSR, plain row-wise definition (Sec. 2), plus the
                   per-entry scale S_ij = sum_k |a_ik||b_kj|.  C code in
                   ``spgemm_oracle.c``.
* ``csr_sum``      ordered sum of partial products (Sec. 4.4; Alg. 1, the
                   accumulation C_ijk += partial).
* ``trident_bounds`` / ``trident_partition``  the hybrid 2D+1D split
                   (Sec. 3.2): q x q coarse tiles, each cut into lambda
                   contiguous row slices.
* ``static_cannon_schedule``  round order of Alg. 1 with the i+j stagger of
                   Eq. 2, read as r' = (r + i + j) mod q.
* ``trident_product``  every output block C_ijk = sum_r A_{i r' k} B_{r' j}
                   (Alg. 1 + Alg. 2 with the allgathered B_{r'j} used whole).
* ``backward``     gradients of L(C) on fixed patterns (chain rule on Sec. 2's
                   definition): dA = (G B^T) on pat(A), dB = (A^T G) on pat(B).
* ``mcl_step``     one Markov-clustering iteration (Sec. 5.6) on the transposed
                   column-stochastic matrix: expansion, inflation, pruning,
                   top-k selection, renormalisation.
* ``permute``      Y = P X Q^T by its definition (the random relabelling of
                   the permuted HV15R runs, Sec. 5).
* ``trident_loads`` nnz of every process's part of the trident partition
                   (Sec. 3.2); max / mean is Table 2's imbalance.

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from gen import CSR

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "spgemm_oracle.c")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp] + _SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_get_threads.restype = ctypes.c_int
        lib.oracle_row_products.argtypes = [I64, P, P, P, P]
        lib.oracle_spgemm_counts.argtypes = [I64, P, P, P, P, P]
        lib.oracle_spgemm_counts.restype = ctypes.c_int
        for name in ("oracle_spgemm_fill_f64", "oracle_spgemm_fill_f32"):
            f = getattr(lib, name)
            f.argtypes = [I64, P, P, P, P, P, P, P, P, P, P]
            f.restype = ctypes.c_int
        lib.oracle_csr_sum_counts.argtypes = [ctypes.c_int32, I64, P, P, P]
        lib.oracle_csr_sum_counts.restype = ctypes.c_int
        for name in ("oracle_csr_sum_fill_f64", "oracle_csr_sum_fill_f32"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_int32, I64, P, P, P, P, P, P]
            f.restype = ctypes.c_int
        lib.oracle_spgemm_backward_f64.argtypes = [I64, I64] + [P] * 11
        lib.oracle_spgemm_backward_f64.restype = ctypes.c_int
        lib.oracle_spgemm_fill_f32p64.argtypes = [I64] + [P] * 9
        lib.oracle_spgemm_fill_f32p64.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _canon(A: CSR):
    return (np.ascontiguousarray(A.rowptr, dtype=np.int64), np.ascontiguousarray(A.col, dtype=np.int32))


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def row_products(A: CSR, B: CSR) -> np.ndarray:
    """u_i = number of intermediate products of row i (sum of |B_k| over k in A_i)."""
    lib = _load()
    arp, acol = _canon(A)
    brp, _ = _canon(B)
    u = np.zeros(A.nrows, dtype=np.int64)
    if A.nrows:
        lib.oracle_row_products(A.nrows, _p(arp), _p(acol), _p(brp), _p(u))
    return u


def spgemm(A: CSR, B: CSR, precision: str | None = None, with_scale: bool = True):
    """C = A B (paper Sec. 2).  Returns (C, S) with S_ij = sum_k |a_ik||b_kj|.

    ``precision``: "f64" (double products and sums) or "f32" (float products
    and sums); default follows A's value dtype."""
    if A.ncols != B.nrows:
        raise ValueError("shape mismatch")
    lib = _load()
    if precision is None:
        precision = "f32" if A.val.dtype == np.float32 else "f64"
    T = np.float32 if precision == "f32" else np.float64
    arp, acol = _canon(A)
    brp, bcol = _canon(B)
    aval = np.ascontiguousarray(A.val, dtype=T)
    bval = np.ascontiguousarray(B.val, dtype=T)
    m = A.nrows
    counts = np.zeros(m, dtype=np.int64)
    if m and lib.oracle_spgemm_counts(m, _p(arp), _p(acol), _p(brp), _p(bcol), _p(counts)):
        raise MemoryError("oracle scratch allocation failed")
    crp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=crp[1:])
    nnz = int(crp[-1])
    ccol = np.zeros(nnz, dtype=np.int32)
    cval = np.zeros(nnz, dtype=T)
    cabs = np.zeros(nnz, dtype=np.float64) if with_scale else None
    fill = lib.oracle_spgemm_fill_f32 if precision == "f32" else lib.oracle_spgemm_fill_f64
    if m:
        rc = fill(m, _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol), _p(bval), _p(crp), _p(ccol),
                  _p(cval), _p(cabs) if cabs is not None else None)
        if rc:
            raise RuntimeError(f"oracle fill failed ({rc})")
    return CSR(m, B.ncols, crp, ccol, cval), cabs


def csr_sum(parts: list[CSR], precision: str | None = None) -> CSR:
    """Ordered sum of CSR matrices of one shape: row by row, the union of the
    patterns; equal columns are added in part order (Sec. 4.4, the spgeam
    accumulation of round partials with unit coefficients)."""
    if not parts:
        raise ValueError("no parts")
    m, n = parts[0].nrows, parts[0].ncols
    for P in parts:
        if P.nrows != m or P.ncols != n:
            raise ValueError("shape mismatch")
    lib = _load()
    if precision is None:
        precision = "f32" if parts[0].val.dtype == np.float32 else "f64"
    T = np.float32 if precision == "f32" else np.float64
    rps = [np.ascontiguousarray(P.rowptr, dtype=np.int64) for P in parts]
    cols = [np.ascontiguousarray(P.col, dtype=np.int32) for P in parts]
    vals = [np.ascontiguousarray(P.val, dtype=T) for P in parts]
    arr = lambda xs: (ctypes.c_void_p * len(xs))(*[x.ctypes.data for x in xs])
    rp_a, col_a, val_a = arr(rps), arr(cols), arr(vals)
    counts = np.zeros(m, dtype=np.int64)
    if m and lib.oracle_csr_sum_counts(len(parts), m, rp_a, col_a, _p(counts)):
        raise MemoryError("oracle scratch allocation failed")
    crp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=crp[1:])
    ccol = np.zeros(int(crp[-1]), dtype=np.int32)
    cval = np.zeros(int(crp[-1]), dtype=T)
    fill = lib.oracle_csr_sum_fill_f32 if precision == "f32" else lib.oracle_csr_sum_fill_f64
    if m and fill(len(parts), m, rp_a, col_a, val_a, _p(crp), _p(ccol), _p(cval)):
        raise RuntimeError("oracle sum failed")
    return CSR(m, n, crp, ccol, cval)


# ------------------------------------------------------------------ trident

def trident_bounds(n: int, q: int, lam: int = 1):
    """Boundaries of the hybrid 2D+1D split of an index range of length n
    (Sec. 3.2).  Coarse tile t covers [floor(t n / q), floor((t+1) n / q));
    slice s of coarse tile t covers its rows
    [lo + floor(s L / lam), lo + floor((s+1) L / lam)) with L the tile length.
    Returns (coarse bounds, length q+1; slice bounds, length q*lam+1)."""
    coarse = [(t * n) // q for t in range(q + 1)]
    fine = []
    for t in range(q):
        lo, hi = coarse[t], coarse[t + 1]
        L = hi - lo
        for s in range(lam):
            fine.append(lo + (s * L) // lam)
    fine.append(n)
    return coarse, fine


def submatrix(A: CSR, r0: int, r1: int, c0: int, c1: int) -> CSR:
    """Rows [r0, r1) and columns [c0, c1) of A, column indices shifted to be
    local to the block (column j of A becomes j - c0)."""
    rp = A.rowptr
    lo, hi = int(rp[r0]), int(rp[r1])
    col = A.col[lo:hi]
    val = A.val[lo:hi]
    rows = np.repeat(np.arange(r1 - r0), np.diff(rp[r0:r1 + 1]))
    keep = (col >= c0) & (col < c1)
    counts = np.bincount(rows[keep], minlength=r1 - r0)
    out_rp = np.zeros(r1 - r0 + 1, dtype=np.int64)
    np.cumsum(counts, out=out_rp[1:])
    return CSR(r1 - r0, c1 - c0, out_rp, (col[keep] - c0).astype(np.int32), val[keep].copy())


def trident_partition(A: CSR, B: CSR, q: int, lam: int):
    """Trident partitioning (Sec. 3.2) of A (m x kk) and B (kk x n).

    A is cut into q x q coarse tiles A_ir, each split into lam row slices
    A_irk.  B is cut into q x q coarse tiles; on one device the allgather of
    Alg. 2 (B_rj = AllGather(B_rjk)) yields the whole tile B_rj, which is
    what is returned.  Returns (A_slices[i][r][k], B_tiles[r][j])."""
    _, rows_fine = trident_bounds(A.nrows, q, lam)
    kcoarse, _ = trident_bounds(A.ncols, q, 1)
    ncoarse, _ = trident_bounds(B.ncols, q, 1)
    A_s = [[[submatrix(A, rows_fine[i * lam + k], rows_fine[i * lam + k + 1], kcoarse[r], kcoarse[r + 1])
             for k in range(lam)] for r in range(q)] for i in range(q)]
    B_t = [[submatrix(B, kcoarse[r], kcoarse[r + 1], ncoarse[j], ncoarse[j + 1]) for j in range(q)]
           for r in range(q)]
    return A_s, B_t


def permute(X: CSR, row_perm=None, col_perm=None) -> CSR:
    """Y = P X Q^T written out: entry (i, j, v) of X becomes (row_perm[i],
    col_perm[j], v) of Y (None: the identity); Y's rows sorted by column
    (Sec. 5, random permutation of rows and columns)."""
    rows = np.repeat(np.arange(X.nrows, dtype=np.int64), np.diff(X.rowptr))
    r = rows if row_perm is None else np.asarray(row_perm, dtype=np.int64)[rows]
    c = X.col.astype(np.int64) if col_perm is None else np.asarray(col_perm, dtype=np.int64)[X.col]
    order = np.lexsort((c, r))
    counts = np.bincount(r, minlength=X.nrows)
    rp = np.zeros(X.nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return CSR(X.nrows, X.ncols, rp, c[order].astype(np.int32), X.val[order].copy())


def trident_loads(X: CSR, q: int, lam: int):
    """nnz of the part X_{ijk} held by process (i, j, k) when X is cut by the
    trident partition (Sec. 3.2): q x q coarse tiles, each split into lam row
    slices.  Returns a (q*lam) x q integer array (row: slice i*lam+k, column:
    coarse column tile j); max / mean over it is the imbalance of Table 2."""
    _, fine = trident_bounds(X.nrows, q, lam)
    coarse, _ = trident_bounds(X.ncols, q, 1)
    out = np.zeros((q * lam, q), dtype=np.int64)
    for a in range(q * lam):
        for b in range(q):
            out[a, b] = submatrix(X, fine[a], fine[a + 1], coarse[b], coarse[b + 1]).nnz
    return out


def static_cannon_schedule(q: int, i: int, j: int):
    """Rounds of Alg. 1 for output tile (i, j): round r uses inner tile
    r' = (r + i + j) mod q (Eq. 2 with the stagger taken modulo q; the loop
    runs r = 0..q-1, q rounds)."""
    return [(r + i + j) % q for r in range(q)]


def trident_product(A: CSR, B: CSR, q: int, lam: int, precision: str | None = None):
    """All output blocks C_ijk = sum_r A_{i r' k} B_{r' j} (Alg. 1 with Alg. 2
    as its partial product), each partial formed by ``spgemm`` and summed in
    round order r = 0..q-1 by ``csr_sum``.  Returns C[i][j][k] (block-local
    columns) and the partials P[i][j][k] (list over r)."""
    A_s, B_t = trident_partition(A, B, q, lam)
    C = [[[None] * lam for _ in range(q)] for _ in range(q)]
    partials = [[[None] * lam for _ in range(q)] for _ in range(q)]
    for i in range(q):
        for j in range(q):
            sched = static_cannon_schedule(q, i, j)
            for k in range(lam):
                parts = [spgemm(A_s[i][rr][k], B_t[rr][j], precision, with_scale=False)[0] for rr in sched]
                partials[i][j][k] = parts
                C[i][j][k] = csr_sum(parts, precision)
    return C, partials


def assemble_blocks(blocks, row_bounds, col_bounds, nrows: int, ncols: int) -> CSR:
    """Inverse of the partition for a grid blocks[a][b] (row part a, col part b)."""
    rows_all, cols_all, vals_all = [], [], []
    for a, row in enumerate(blocks):
        for b, X in enumerate(row):
            r = np.repeat(np.arange(X.nrows), X.row_lengths()) + row_bounds[a]
            rows_all.append(r)
            cols_all.append(X.col.astype(np.int64) + col_bounds[b])
            vals_all.append(X.val)
    rows = np.concatenate(rows_all)
    cols = np.concatenate(cols_all)
    vals = np.concatenate(vals_all)
    order = np.lexsort((cols, rows))
    counts = np.bincount(rows, minlength=nrows)
    rp = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return CSR(nrows, ncols, rp, cols[order].astype(np.int32), vals[order])


# ----------------------------------------------------------------- backward

def backward(A: CSR, B: CSR, C: CSR, G: np.ndarray):
    """(dA, dB) for upstream gradient G on C's pattern, in double:
    dA_ik = sum_{j in B_k} G_ij b_kj on pat(A); dB_kj = sum_i a_ik G_ij on pat(B)."""
    lib = _load()
    arp, acol = _canon(A)
    brp, bcol = _canon(B)
    crp, ccol = _canon(C)
    aval = np.ascontiguousarray(A.val, dtype=np.float64)
    bval = np.ascontiguousarray(B.val, dtype=np.float64)
    g = np.ascontiguousarray(G, dtype=np.float64)
    da = np.zeros(A.nnz, dtype=np.float64)
    db = np.zeros(B.nnz, dtype=np.float64)
    rc = lib.oracle_spgemm_backward_f64(A.nrows, B.nrows, _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol),
                                        _p(bval), _p(crp), _p(ccol), _p(g), _p(da), _p(db))
    if rc:
        raise RuntimeError("backward: C pattern does not contain a product position")
    return da, db


# ------------------------------------------------------------------ helpers

def dense_product(A: CSR, B: CSR) -> np.ndarray:
    return A.to_dense() @ B.to_dense()


def boolean_pattern(A: CSR, B: CSR) -> np.ndarray:
    """Structural product: True where some a_ik b_kj exists (counts of
    products > 0 with all-ones values; nothing can cancel)."""
    Ad = _pattern_dense(A)
    Bd = _pattern_dense(B)
    return (Ad.astype(np.int64) @ Bd.astype(np.int64)) > 0


def _pattern_dense(A: CSR) -> np.ndarray:
    out = np.zeros((A.nrows, A.ncols), dtype=bool)
    rows = np.repeat(np.arange(A.nrows), A.row_lengths())
    out[rows, A.col.astype(np.int64)] = True
    return out


def transpose(A: CSR) -> CSR:
    rows = np.repeat(np.arange(A.nrows, dtype=np.int64), A.row_lengths())
    cols = A.col.astype(np.int64)
    order = np.lexsort((rows, cols))
    counts = np.bincount(cols, minlength=A.ncols)
    rp = np.zeros(A.ncols + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return CSR(A.ncols, A.nrows, rp, rows[order].astype(np.int32), A.val[order])


# ---------------------------------------------------------- Markov clustering

def spgemm_f32p64(A: CSR, B: CSR) -> CSR:
    """C = A B for float inputs: each product rounded to float, the products
    of an entry added in double in list order (values returned as float64)."""
    lib = _load()
    arp, acol = _canon(A)
    brp, bcol = _canon(B)
    aval = np.ascontiguousarray(A.val, dtype=np.float32)
    bval = np.ascontiguousarray(B.val, dtype=np.float32)
    m = A.nrows
    counts = np.zeros(m, dtype=np.int64)
    if m and lib.oracle_spgemm_counts(m, _p(arp), _p(acol), _p(brp), _p(bcol), _p(counts)):
        raise MemoryError("oracle scratch allocation failed")
    crp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=crp[1:])
    ccol = np.zeros(int(crp[-1]), dtype=np.int32)
    cval = np.zeros(int(crp[-1]), dtype=np.float64)
    if m and lib.oracle_spgemm_fill_f32p64(m, _p(arp), _p(acol), _p(aval), _p(brp), _p(bcol), _p(bval), _p(crp),
                                           _p(ccol), _p(cval)):
        raise RuntimeError("oracle fill failed")
    return CSR(m, B.ncols, crp, ccol, cval)


def mcl_select(cols: np.ndarray, e: np.ndarray, inflation: float = 2.0, prune: float = 1e-4, topk: int = 1000):
    """Inflation, pruning, top-k and renormalisation of one expanded row
    (Sec. 5.6; the row is a column of the Markov matrix).  All decisions in
    double:
      w_j = e_j ** r (r = 2: e_j * e_j), v_j = w_j / sum_j w_j
      keep v_j >= prune; if nothing is kept, keep the largest v_j
      if more than topk are kept, keep the topk largest
      ties (equal v) go to the smaller column index
      out_j = float(v_j / sum of kept v)
    Returns (kept columns ascending, float32 values, dict of the cuts)."""
    if cols.size == 0:
        return cols, np.zeros(0, dtype=np.float32), {}
    w = e * e if inflation == 2.0 else np.power(e, inflation)
    v = w / w.sum()
    keep = v >= prune
    cuts = {"prune": prune}
    if not keep.any():
        order = np.lexsort((cols, -v))
        keep = np.zeros_like(keep)
        keep[order[0]] = True
        cuts["largest"] = float(v[order[0]])
    elif keep.sum() > topk:
        idx = np.nonzero(keep)[0]
        order = idx[np.lexsort((cols[idx], -v[idx]))]
        keep = np.zeros_like(keep)
        keep[order[:topk]] = True
        cuts["topk_value"] = float(v[order[topk - 1]])
    t = v[keep].sum()
    return cols[keep], (v[keep] / t).astype(np.float32), dict(cuts, v=v, cols=cols)


def mcl_step(Mt: CSR, inflation: float = 2.0, prune: float = 1e-4, topk: int = 1000,
             rows: np.ndarray | None = None):
    """One MCL iteration on the transposed stochastic matrix Mt (row r of Mt
    is column r of M): the expansion (M M)^T = Mt Mt, then ``mcl_select`` per
    row.  With ``rows``, only those rows are formed (returned as a dict
    row -> (cols, vals, cuts)); otherwise the whole next iterate as CSR."""
    sel = np.arange(Mt.nrows) if rows is None else np.asarray(rows)
    lens = Mt.row_lengths()[sel]
    rp = np.zeros(sel.size + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(Mt.rowptr[r], Mt.rowptr[r + 1]) for r in sel]) if sel.size else \
        np.zeros(0, dtype=np.int64)
    sub = CSR(sel.size, Mt.ncols, rp, Mt.col[idx], Mt.val[idx])
    E = spgemm_f32p64(sub, Mt)
    out = {}
    for t, r in enumerate(sel):
        a, b = E.rowptr[t], E.rowptr[t + 1]
        out[int(r)] = mcl_select(E.col[a:b], E.val[a:b], inflation, prune, topk)
    if rows is not None:
        return out
    counts = np.array([out[r][0].size for r in range(Mt.nrows)], dtype=np.int64)
    nrp = np.zeros(Mt.nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=nrp[1:])
    col = np.concatenate([out[r][0] for r in range(Mt.nrows)]).astype(np.int32)
    val = np.concatenate([out[r][1] for r in range(Mt.nrows)]).astype(np.float32)
    return CSR(Mt.nrows, Mt.ncols, nrp, col, val)
