"""Pins for the oracle's Markov-clustering iteration (Sec. 5.6 with the
configured inflation 2, pruning 1e-4, top-1000, renormalisation), on the
transposed column-stochastic matrix."""
import numpy as np
import pytest

import gen
import oracle


def csr(rows_cols_vals, n):
    rp = [0]
    cols, vals = [], []
    for cs, vs in rows_cols_vals:
        cols += cs
        vals += vs
        rp.append(len(cols))
    return gen.CSR(len(rows_cols_vals), n, np.array(rp, dtype=np.int64), np.array(cols, dtype=np.int32),
                   np.array(vals, dtype=np.float32))


def test_hand_derived_two_nodes():
    # columns of M: node 0 -> {0: 1}, node 1 -> {0: 1/2, 1: 1/2}
    # expansion row 1: 0.5 * (1, 0) + 0.5 * (0.5, 0.5) = (0.75, 0.25)
    # squares (0.5625, 0.0625), sum 0.625 -> (0.9, 0.1)
    Mt = csr([([0], [1.0]), ([0, 1], [0.5, 0.5])], 2)
    R = oracle.mcl_step(Mt)
    assert R.rowptr.tolist() == [0, 1, 3]
    assert R.col.tolist() == [0, 0, 1]
    assert np.allclose(R.val, [1.0, 0.9, 0.1], rtol=1e-7)


def test_uniform_blocks_are_fixed_points():
    # block-diagonal, each block uniform 1/b: M^2 = M, inflation keeps 1/b
    rows = []
    n = 0
    for b in (1, 3, 7, 50):
        for _ in range(b):
            rows.append((list(range(n, n + b)), [1.0 / b] * b))
        n += b
    Mt = csr(rows, n)
    R = oracle.mcl_step(Mt)
    assert np.array_equal(R.rowptr, Mt.rowptr) and np.array_equal(R.col, Mt.col)
    assert np.allclose(R.val, Mt.val, rtol=1e-6)


def test_topk_ties_go_to_smaller_columns():
    cols = np.arange(10, dtype=np.int32)[::-1].copy()
    e = np.ones(10)
    kc, kv, _ = oracle.mcl_select(np.sort(cols), e, topk=3)
    assert kc.tolist() == [0, 1, 2]
    assert np.allclose(kv, 1.0 / 3)


def test_prune_everything_keeps_largest():
    cols = np.arange(20000, dtype=np.int32)
    e = np.ones(20000)       # each v = 5e-5 < 1e-4
    e[777] = 1.0             # ties: the smallest column wins
    kc, kv, _ = oracle.mcl_select(cols, e)
    assert kc.tolist() == [0] and kv.tolist() == [1.0]


def test_prune_threshold_is_inclusive_of_cut():
    # v = (0.5, 0.5) after inflation of (1, 1); prune 0.5 keeps both (v >= cut)
    kc, kv, _ = oracle.mcl_select(np.array([3, 4], dtype=np.int32), np.array([1.0, 1.0]), prune=0.5)
    assert kc.tolist() == [3, 4]


@pytest.mark.parametrize("scale", [9, 10])
def test_rmat_iteration_invariants(scale):
    Mt = gen.rmat_stochastic(scale=scale, edge_factor=16, seed=3)
    # column-stochastic input: rows of Mt sum to 1
    assert np.allclose(np.add.reduceat(Mt.val.astype(np.float64), Mt.rowptr[:-1]), 1.0, atol=1e-6)
    R = oracle.mcl_step(Mt, topk=40)
    sums = np.add.reduceat(R.val.astype(np.float64), R.rowptr[:-1])
    assert np.allclose(sums, 1.0, atol=1e-5)
    assert R.row_lengths().max() <= 40 and R.row_lengths().min() >= 1
    assert R.val.min() >= 1e-4 * (1 - 1e-6)
    for i in range(R.nrows):
        assert np.all(np.diff(R.col[R.rowptr[i]:R.rowptr[i + 1]]) > 0)
    # a sampled-row call gives the same rows
    rows = np.array([0, 5, R.nrows - 1])
    part = oracle.mcl_step(Mt, topk=40, rows=rows)
    for r in rows:
        a, b = R.rowptr[r], R.rowptr[r + 1]
        assert np.array_equal(part[int(r)][0], R.col[a:b]) and np.array_equal(part[int(r)][1], R.val[a:b])


def test_mixed_precision_product_matches_definition():
    # float products rounded once, double sums: compare with a double recompute
    A = gen.er_variable(200, 150, 12, 3, np.float32, "uniform")
    B = gen.er_variable(150, 180, 12, 4, np.float32, "uniform")
    C = oracle.spgemm_f32p64(A, B)
    Ad = A.to_dense().astype(np.float32)
    Bd = B.to_dense().astype(np.float32)
    ref, S = oracle.spgemm(A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(C.col, ref.col)
    # each float product is within 2^-24 of the exact one
    assert np.all(np.abs(C.val - ref.val) <= 2.0 ** -23 * S)
    del Ad, Bd
