"""Pins for the oracle's trident pieces: the hybrid 2D+1D partition (Sec. 3.2),
the static-Cannon round order (Alg. 1, Eq. 2), the ordered sum of partials
(Sec. 4.4) and the backward pass (chain rule on Sec. 2's definition)."""
import itertools

import numpy as np
import pytest

import gen
import oracle


@pytest.mark.parametrize("n,q,lam", [(64, 2, 2), (97, 3, 2), (2 ** 10, 4, 4), (10, 4, 3), (5, 1, 1)])
def test_bounds_cover_range(n, q, lam):
    coarse, fine = oracle.trident_bounds(n, q, lam)
    assert coarse[0] == 0 and coarse[-1] == n and len(coarse) == q + 1
    assert fine[0] == 0 and fine[-1] == n and len(fine) == q * lam + 1
    assert all(a <= b for a, b in zip(fine, fine[1:]))
    # every coarse boundary is a slice boundary: slices nest in tiles
    assert set(coarse) <= set(fine)
    # equal-count split for a power of two
    if n % (q * lam) == 0:
        assert np.all(np.diff(fine) == n // (q * lam))


def test_partition_reassembles_exactly():
    A = gen.er_variable(203, 157, 12, 3, np.float64, "uniform", p_empty=0.1)
    B = gen.er_variable(157, 181, 12, 4, np.float64, "uniform", p_empty=0.1)
    q, lam = 3, 2
    A_s, B_t = oracle.trident_partition(A, B, q, lam)
    _, rows_fine = oracle.trident_bounds(A.nrows, q, lam)
    kc, _ = oracle.trident_bounds(A.ncols, q, 1)
    nc, _ = oracle.trident_bounds(B.ncols, q, 1)
    grid = [[A_s[s // lam][r][s % lam] for r in range(q)] for s in range(q * lam)]
    A2 = oracle.assemble_blocks(grid, rows_fine, kc, A.nrows, A.ncols)
    assert np.array_equal(A2.rowptr, A.rowptr) and np.array_equal(A2.col, A.col)
    assert np.array_equal(A2.val, A.val)
    B2 = oracle.assemble_blocks(B_t, kc, nc, B.nrows, B.ncols)
    assert np.array_equal(B2.rowptr, B.rowptr) and np.array_equal(B2.col, B.col)
    # nnz is conserved and block-local columns are in range
    assert sum(X.nnz for row in grid for X in row) == A.nnz
    for row in grid:
        for X in row:
            assert X.nnz == 0 or (X.col.min() >= 0 and X.col.max() < X.ncols)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_static_cannon_schedule(q):
    for i, j in itertools.product(range(q), repeat=2):
        s = oracle.static_cannon_schedule(q, i, j)
        # every inner tile exactly once (q rounds, r = 0..q-1)
        assert sorted(s) == list(range(q))
        # Eq. 2: round r uses r + i + j (mod q)
        assert s[0] == (i + j) % q
    # Cannon's alignment: in a round, the tiles of one block row use distinct
    # inner tiles, and so do the tiles of one block column
    for r in range(q):
        for i in range(q):
            assert len({oracle.static_cannon_schedule(q, i, j)[r] for j in range(q)}) == q
        for j in range(q):
            assert len({oracle.static_cannon_schedule(q, i, j)[r] for i in range(q)}) == q


def test_csr_sum_union_and_order():
    # union of patterns, values added in part order: (1e16 + 1) + (-1e16) = 0
    P0 = gen.from_dense(np.array([[1e16, 0.0, 2.0]]))
    P1 = gen.from_dense(np.array([[1.0, 3.0, 0.0]]))
    P2 = gen.from_dense(np.array([[-1e16, 0.0, 0.0]]))
    C = oracle.csr_sum([P0, P1, P2])
    assert C.col.tolist() == [0, 1, 2]
    assert C.val.tolist() == [0.0, 3.0, 2.0]
    C2 = oracle.csr_sum([P0, P2, P1])
    assert C2.val.tolist() == [1.0, 3.0, 2.0]


def test_csr_sum_dense_reference():
    parts = [gen.er_variable(50, 70, 9, 60 + t, np.float64, "int", p_empty=0.2) for t in range(4)]
    C = oracle.csr_sum(parts)
    dense = sum(P.to_dense() for P in parts)
    pat = np.zeros_like(dense, dtype=bool)
    for P in parts:
        pat |= oracle._pattern_dense(P)
    assert np.array_equal(oracle._pattern_dense(C), pat)
    assert np.array_equal(C.to_dense(), dense)


@pytest.mark.parametrize("q,lam,values", [(2, 2, "int"), (3, 2, "int"), (4, 4, "uniform"), (2, 3, "uniform")])
def test_trident_blocks_equal_unpartitioned_product(q, lam, values):
    n = 96
    A = gen.er(n, n, 10, 40 + q, np.float64, values)
    B = gen.er(n, n, 10, 41 + q, np.float64, values)
    C, S = oracle.spgemm(A, B)
    blocks, _ = oracle.trident_product(A, B, q, lam)
    _, rows_fine = oracle.trident_bounds(n, q, lam)
    nc, _ = oracle.trident_bounds(n, q, 1)
    grid = [[blocks[s // lam][j][s % lam] for j in range(q)] for s in range(q * lam)]
    C2 = oracle.assemble_blocks(grid, rows_fine, nc, n, n)
    assert np.array_equal(C2.rowptr, C.rowptr)
    assert np.array_equal(C2.col, C.col)
    if values == "int":
        assert np.array_equal(C2.val, C.val)
    else:
        assert np.all(np.abs(C2.val - C.val) <= 1e-12 * S)


def test_stagger_versus_natural_order():
    # rounds in stagger order (Eq. 2) or natural order (Eq. 1) give the same
    # pattern; integer values agree exactly
    n, q, lam = 64, 4, 2
    A = gen.er(n, n, 8, 70, np.float64, "int")
    B = gen.er(n, n, 8, 71, np.float64, "int")
    A_s, B_t = oracle.trident_partition(A, B, q, lam)
    for i, j, k in itertools.product(range(q), range(q), range(lam)):
        stag = [oracle.spgemm(A_s[i][r][k], B_t[r][j], with_scale=False)[0]
                for r in oracle.static_cannon_schedule(q, i, j)]
        nat = [oracle.spgemm(A_s[i][r][k], B_t[r][j], with_scale=False)[0] for r in range(q)]
        X, Y = oracle.csr_sum(stag), oracle.csr_sum(nat)
        assert np.array_equal(X.rowptr, Y.rowptr) and np.array_equal(X.col, Y.col)
        assert np.array_equal(X.val, Y.val)


# ----------------------------------------------------------------- backward

def _dense_grads(A, B, C, G):
    Gd = np.zeros((C.nrows, C.ncols))
    rows = np.repeat(np.arange(C.nrows), C.row_lengths())
    Gd[rows, C.col] = G
    dA = Gd @ B.to_dense().T
    dB = A.to_dense().T @ Gd
    ra = np.repeat(np.arange(A.nrows), A.row_lengths())
    rb = np.repeat(np.arange(B.nrows), B.row_lengths())
    return dA[ra, A.col], dB[rb, B.col]


@pytest.mark.parametrize("seed", range(3))
def test_backward_dense_reference(seed):
    A = gen.er_variable(40, 30, 8, 80 + seed, np.float64, "int", p_empty=0.1)
    B = gen.er_variable(30, 50, 8, 90 + seed, np.float64, "int", p_empty=0.1)
    C, _ = oracle.spgemm(A, B)
    G = np.random.default_rng(seed).integers(-3, 4, size=C.nnz).astype(np.float64)
    dA, dB = oracle.backward(A, B, C, G)
    rA, rB = _dense_grads(A, B, C, G)
    assert np.array_equal(dA, rA) and np.array_equal(dB, rB)


def test_backward_central_differences():
    # L = sum(C * W) is bilinear in (A, B): central differences with a dyadic
    # step have no truncation error.  Only the rows touched by an entry are
    # re-evaluated, so the difference is not lost in a large sum.
    A = gen.er(60, 60, 6, 5, np.float64, "normal")
    B = gen.er(60, 45, 6, 6, np.float64, "normal")
    C, _ = oracle.spgemm(A, B)
    W = np.random.default_rng(7).standard_normal(C.nnz)
    dA, dB = oracle.backward(A, B, C, W)
    h = 2.0 ** -8
    rng = np.random.default_rng(8)

    def loss(Ax, Bx):
        Cx, _ = oracle.spgemm(Ax, Bx, with_scale=False)
        assert np.array_equal(Cx.col, C.col)
        return float(np.dot(Cx.val, W))

    for e in rng.choice(A.nnz, 20, replace=False):
        vp, vm = A.val.copy(), A.val.copy()
        vp[e] += h
        vm[e] -= h
        fd = (loss(A.with_values(vp), B) - loss(A.with_values(vm), B)) / (2 * h)
        assert abs(fd - dA[e]) <= 1e-6 * max(abs(fd), abs(dA[e]), 1e-300)
    for e in rng.choice(B.nnz, 20, replace=False):
        vp, vm = B.val.copy(), B.val.copy()
        vp[e] += h
        vm[e] -= h
        fd = (loss(A, B.with_values(vp)) - loss(A, B.with_values(vm))) / (2 * h)
        assert abs(fd - dB[e]) <= 1e-6 * max(abs(fd), abs(dB[e]), 1e-300)
