"""Property-based pins of the oracle on many tiny random inputs (hypothesis):
integer-valued matrices, so every product and sum is exact and the oracle
must equal dense numpy arithmetic to the bit, for any shape including empty
rows, columns and matrices."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402


@st.composite
def int_matrix(draw, rows=None, cols=None, max_dim=9):
    m = draw(st.integers(0, max_dim)) if rows is None else rows
    n = draw(st.integers(0, max_dim)) if cols is None else cols
    density = draw(st.sampled_from([0.0, 0.15, 0.4, 0.8, 1.0]))
    seed = draw(st.integers(0, 2**31 - 1))
    rng = np.random.default_rng(seed)
    D = rng.integers(-3, 4, size=(m, n)).astype(np.float64)
    D[rng.random((m, n)) >= density] = 0.0
    return D


@st.composite
def product_pair(draw):
    m, k, n = (draw(st.integers(0, 9)) for _ in range(3))
    return draw(int_matrix(m, k)), draw(int_matrix(k, n))


def canonical(X):
    for i in range(X.nrows):
        c = X.col[X.rowptr[i]:X.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
        assert np.all((c >= 0) & (c < X.ncols))


@settings(max_examples=300, deadline=None)
@given(product_pair())
def test_product_equals_dense_and_boolean_pattern(pair):
    Da, Db = pair
    A, B = gen.from_dense(Da), gen.from_dense(Db)
    C, S = oracle.spgemm(A, B)
    canonical(C)
    assert (C.nrows, C.ncols) == (Da.shape[0], Db.shape[1])
    assert np.array_equal(C.to_dense(), Da @ Db)
    # the pattern is the structural product: cancellations stay as explicit zeros
    pat = (Da != 0).astype(np.int64) @ (Db != 0).astype(np.int64) > 0
    Pc = np.zeros(pat.shape, dtype=bool)
    rows = np.repeat(np.arange(C.nrows), np.diff(C.rowptr))
    Pc[rows, C.col] = True
    assert np.array_equal(Pc, pat)
    # S = |A| |B| on the pattern
    Sd = np.abs(Da) @ np.abs(Db)
    assert np.array_equal(S, Sd[rows, C.col])


@settings(max_examples=200, deadline=None)
@given(st.integers(1, 5).flatmap(lambda p: st.tuples(st.just(p), st.integers(0, 8), st.integers(0, 8))),
       st.data())
def test_ordered_sum_equals_dense(shape, data):
    nparts, m, n = shape
    Ds = [data.draw(int_matrix(m, n)) for _ in range(nparts)]
    S = oracle.csr_sum([gen.from_dense(D) for D in Ds])
    canonical(S)
    assert np.array_equal(S.to_dense(), sum(Ds))
    union = np.zeros((m, n), dtype=bool)
    for D in Ds:
        union |= D != 0
    Ps = np.zeros((m, n), dtype=bool)
    Ps[np.repeat(np.arange(m), np.diff(S.rowptr)), S.col] = True
    assert np.array_equal(Ps, union)


@settings(max_examples=200, deadline=None)
@given(int_matrix(), st.integers(0, 2**31 - 1))
def test_transpose_and_permute_against_dense(D, seed):
    X = gen.from_dense(D)
    T = oracle.transpose(X)
    canonical(T)
    assert np.array_equal(T.to_dense(), D.T)
    rng = np.random.default_rng(seed)
    rp, cp = rng.permutation(D.shape[0]), rng.permutation(D.shape[1])
    Y = oracle.permute(X, rp, cp)
    canonical(Y)
    E = np.zeros_like(D)
    E[np.ix_(rp, cp)] = D
    assert np.array_equal(Y.to_dense(), E)


@settings(max_examples=150, deadline=None)
@given(product_pair(), st.integers(1, 3), st.integers(1, 3))
def test_trident_blocks_reassemble_the_product(pair, q, lam):
    Da, Db = pair
    A, B = gen.from_dense(Da), gen.from_dense(Db)
    blocks, _ = oracle.trident_product(A, B, q, lam)
    _, fine = oracle.trident_bounds(A.nrows, q, lam)
    coarse, _ = oracle.trident_bounds(B.ncols, q, 1)
    grid = [[blocks[a // lam][b][a % lam] for b in range(q)] for a in range(q * lam)]
    C = oracle.assemble_blocks(grid, fine, coarse, A.nrows, B.ncols)
    assert np.array_equal(C.to_dense(), Da @ Db)
