"""Pins for the CPU oracle's product (paper Sec. 2: C = A B in CSR).

Each check compares the oracle with something other than itself: dense
brute force, the boolean product, algebraic identities, scipy, closed forms
and hand-derived values.  All run on the CPU in seconds."""
import numpy as np
import pytest

import gen
import oracle

scipy_sparse = pytest.importorskip("scipy.sparse")


def small_cases():
    """Rectangular shapes, ragged rows, empty rows and columns."""
    out = []
    for seed, (m, k, n, dA, dB) in enumerate([(1, 1, 1, 1, 1), (7, 5, 3, 3, 2), (64, 64, 64, 8, 8),
                                               (40, 17, 63, 6, 9), (33, 64, 1, 12, 1), (17, 1, 29, 1, 20),
                                               (50, 60, 40, 0, 5), (64, 50, 64, 30, 40)]):
        A = gen.er_variable(m, k, dA, 100 + seed, np.float64, "int", p_empty=0.2)
        B = gen.er_variable(k, n, dB, 200 + seed, np.float64, "int", p_empty=0.2)
        out.append((A, B))
    return out


def test_hand_derived_3x3():
    # A = [[1,2,0],[0,0,3],[4,0,5]], B = [[0,1,0],[2,0,0],[0,0,6]]
    # C row 0: 1*(0,1,0) + 2*(2,0,0) = (4,1,0); row 1: 3*(0,0,6) = (0,0,18)
    # row 2: 4*(0,1,0) + 5*(0,0,6) = (0,4,30)
    A = gen.from_dense(np.array([[1, 2, 0], [0, 0, 3], [4, 0, 5]], dtype=float))
    B = gen.from_dense(np.array([[0, 1, 0], [2, 0, 0], [0, 0, 6]], dtype=float))
    C, S = oracle.spgemm(A, B)
    assert C.rowptr.tolist() == [0, 2, 3, 5]
    assert C.col.tolist() == [0, 1, 2, 1, 2]
    assert C.val.tolist() == [4.0, 1.0, 18.0, 4.0, 30.0]
    assert S.tolist() == [4.0, 1.0, 18.0, 4.0, 30.0]


@pytest.mark.parametrize("case", range(8))
def test_dense_brute_force_integer_exact(case):
    A, B = small_cases()[case]
    C, S = oracle.spgemm(A, B)
    dense = A.to_dense() @ B.to_dense()
    got = C.to_dense()
    pat = oracle.boolean_pattern(A, B)
    # pattern == boolean product, values exact (small integers)
    assert np.array_equal(oracle._pattern_dense(C), pat)
    assert np.array_equal(got, dense)
    # scale S = |A| |B| on the pattern
    Sd = np.abs(A.to_dense()) @ np.abs(B.to_dense())
    rows = np.repeat(np.arange(C.nrows), C.row_lengths())
    assert np.array_equal(S, Sd[rows, C.col])
    # rows sorted and duplicate-free
    for i in range(C.nrows):
        r = C.col[C.rowptr[i]:C.rowptr[i + 1]]
        assert np.all(np.diff(r) > 0)


@pytest.mark.parametrize("seed", range(5))
def test_dense_brute_force_random_values(seed):
    A = gen.er_variable(48, 40, 10, seed, np.float64, "uniform", p_empty=0.1)
    B = gen.er_variable(40, 56, 10, seed + 50, np.float64, "uniform", p_empty=0.1)
    C, S = oracle.spgemm(A, B)
    dense = A.to_dense() @ B.to_dense()
    rows = np.repeat(np.arange(C.nrows), C.row_lengths())
    err = np.abs(C.val - dense[rows, C.col])
    assert np.all(err <= 1e-12 * S)
    assert np.array_equal(oracle._pattern_dense(C), oracle.boolean_pattern(A, B))


def test_float32_working_precision_matches_rounded_sequence():
    # f32 mode: products and sums each round to float32, in list order
    A = gen.from_dense(np.array([[1.0, 3.0, 7.0]], dtype=np.float32), dtype=np.float32)
    B = gen.from_dense(np.array([[0.1], [0.2], [0.3]], dtype=np.float32), dtype=np.float32)
    C, _ = oracle.spgemm(A, B, "f32")
    a = np.float32
    want = (a(1.0) * a(0.1) + a(3.0) * a(0.2)) + a(7.0) * a(0.3)
    assert C.val.dtype == np.float32 and C.val[0] == want


def test_duplicate_sum_order_is_ascending_k():
    # three products land on column 0: 1e16, 1, -1e16 (k = 0, 1, 2).
    # Left to right: (1e16 + 1) rounds to 1e16, minus 1e16 gives 0.
    # Any other association gives 1.  This pins the summation order.
    A = gen.from_dense(np.array([[1e16, 1.0, -1e16]]))
    B = gen.from_dense(np.array([[1.0], [1.0], [1.0]]))
    C, S = oracle.spgemm(A, B)
    assert C.val.tolist() == [0.0]
    assert S.tolist() == [2e16]


def test_identity_and_permutation_exact():
    A = gen.er_variable(300, 200, 12, 7, np.float64, "uniform", p_empty=0.1)
    I_m = gen.identity(300)
    I_k = gen.identity(200)
    C1, _ = oracle.spgemm(I_m, A)
    C2, _ = oracle.spgemm(A, I_k)
    for C in (C1, C2):
        assert np.array_equal(C.rowptr, A.rowptr)
        assert np.array_equal(C.col, A.col)
        assert np.array_equal(C.val, A.val)
    perm = np.random.default_rng(3).permutation(300)
    C3, _ = oracle.spgemm(gen.permutation_matrix(perm), A)
    assert np.array_equal(C3.to_dense(), A.to_dense()[perm])


def test_power_of_two_row_scaling_exact():
    A = gen.er_variable(100, 80, 9, 8, np.float64, "uniform")
    B = gen.er_variable(80, 90, 9, 9, np.float64, "uniform")
    e = np.random.default_rng(1).integers(-4, 5, size=100)
    D = gen.CSR(100, 100, np.arange(101, dtype=np.int64), np.arange(100, dtype=np.int32), 2.0 ** e)
    C, _ = oracle.spgemm(A, B)
    DA, _ = oracle.spgemm(D, A)
    DC, _ = oracle.spgemm(DA, B)
    rows = np.repeat(np.arange(100), C.row_lengths())
    assert np.array_equal(DC.col, C.col)
    assert np.array_equal(DC.val, C.val * 2.0 ** e[rows])


def test_product_with_ones_vector():
    # C 1 = A (B 1) within the error bound of the two sums
    A = gen.er_variable(500, 400, 16, 11, np.float64, "uniform", p_empty=0.05)
    B = gen.er_variable(400, 300, 16, 12, np.float64, "uniform", p_empty=0.05)
    C, S = oracle.spgemm(A, B)
    lhs = C.to_dense().sum(axis=1)
    rhs = A.to_dense() @ B.to_dense().sum(axis=1)
    bound = (np.abs(A.to_dense()) @ np.abs(B.to_dense())).sum(axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * np.maximum(bound, 1e-300))


def test_transpose_identity():
    # (A B)^T = B^T A^T: identical pattern; integer values exact
    A = gen.er_variable(120, 90, 10, 13, np.float64, "int", p_empty=0.1)
    B = gen.er_variable(90, 110, 10, 14, np.float64, "int", p_empty=0.1)
    C, _ = oracle.spgemm(A, B)
    Ct, _ = oracle.spgemm(oracle.transpose(B), oracle.transpose(A))
    T = oracle.transpose(C)
    assert np.array_equal(T.rowptr, Ct.rowptr)
    assert np.array_equal(T.col, Ct.col)
    assert np.array_equal(T.val, Ct.val)


@pytest.mark.parametrize("shape", [(1, 1), (7, 3), (50, 80), (0, 4)])
def test_transpose_matches_dense(shape):
    m, n = shape
    X = gen.er_variable(m, n, min(n, 6), 15, np.float64, "normal", p_empty=0.2)
    T = oracle.transpose(X)
    assert (T.nrows, T.ncols) == (n, m)
    assert np.array_equal(T.to_dense(), X.to_dense().T)
    for i in range(n):
        assert np.all(np.diff(T.col[T.rowptr[i]:T.rowptr[i + 1]]) > 0)


def test_row_products_brute_force():
    A = gen.er_variable(60, 40, 7, 16, np.float64, "uniform", p_empty=0.2)
    B = gen.er_variable(40, 30, 9, 17, np.float64, "uniform", p_empty=0.2)
    u = oracle.row_products(A, B)
    blen = np.diff(B.rowptr)
    assert u.tolist() == [int(sum(blen[k] for k in A.col[A.rowptr[i]:A.rowptr[i + 1]])) for i in range(A.nrows)]


@pytest.mark.parametrize("seed", range(3))
def test_scipy_cross_check(seed):
    # positive values: nothing cancels, so scipy keeps every structural entry
    A = gen.er_variable(700, 600, 20, 20 + seed, np.float64, "uniform", p_empty=0.05)
    B = gen.er_variable(600, 800, 20, 30 + seed, np.float64, "uniform", p_empty=0.05)
    A = A.with_values(np.abs(A.val) + 0.5)
    B = B.with_values(np.abs(B.val) + 0.5)
    sa = scipy_sparse.csr_matrix((A.val, A.col, A.rowptr), shape=(A.nrows, A.ncols))
    sb = scipy_sparse.csr_matrix((B.val, B.col, B.rowptr), shape=(B.nrows, B.ncols))
    sc = (sa @ sb).tocsr()
    sc.sort_indices()
    C, S = oracle.spgemm(A, B)
    assert np.array_equal(C.rowptr, sc.indptr)
    assert np.array_equal(C.col, sc.indices)
    assert np.all(np.abs(C.val - sc.data) <= 1e-12 * S)


def test_boolean_pattern_with_cancellation_kept():
    # structural pattern: a cancelling entry stays as an explicit zero
    A = gen.from_dense(np.array([[1.0, 1.0]]))
    B = gen.from_dense(np.array([[2.0], [-2.0]]))
    C, S = oracle.spgemm(A, B)
    assert C.nnz == 1 and C.val[0] == 0.0 and S[0] == 4.0


def test_empty_operands():
    A = gen.CSR(5, 4, np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = gen.er(4, 7, 3, 0)
    C, _ = oracle.spgemm(A, B)
    assert C.nnz == 0 and C.rowptr.tolist() == [0] * 6
    A0 = gen.CSR(0, 4, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    C0, _ = oracle.spgemm(A0, B)
    assert C0.nrows == 0 and C0.nnz == 0


def er_expected_nnz_per_row(d, n):
    # entries of one B row never collide; a pair of products from different
    # B rows collides with probability 1/n: E[distinct] ~ d^2 - C(d,2) d^2 / n
    return d * d - d ** 3 * (d - 1) / (2.0 * n)


@pytest.mark.parametrize("n,d", [(4096, 8), (1 << 14, 16)])
def test_er_output_size_closed_form(n, d):
    A = gen.er(n, n, d, 0)
    B = gen.er(n, n, d, 1)
    C, _ = oracle.spgemm(A, B)
    per_row = C.row_lengths()
    mean = per_row.mean()
    expect = er_expected_nnz_per_row(d, n)
    lam = d * d - expect  # collisions ~ Poisson(lam)
    sigma = np.sqrt(lam / n)
    assert abs(mean - expect) <= 5 * sigma + 1e-3
    assert per_row.max() <= d * d


def test_config1_square_of_er():
    # C = A A for the 4096 x 4096, 8-per-row matrix: 262144 products
    A = gen.er(4096, 4096, 8, 0)
    u = oracle.row_products(A, A)
    assert int(u.sum()) == 4096 * 64
    C, S = oracle.spgemm(A, A)
    assert abs(C.row_lengths().mean() - er_expected_nnz_per_row(8, 4096)) < 0.1
    assert np.all(S > 0)


def test_thread_count_does_not_change_results():
    A = gen.er_variable(2000, 1500, 20, 5, np.float64, "uniform")
    B = gen.er_variable(1500, 1700, 20, 6, np.float64, "uniform")
    oracle.set_threads(1)
    C1, S1 = oracle.spgemm(A, B)
    oracle.set_threads(4)
    C4, S4 = oracle.spgemm(A, B)
    assert np.array_equal(C1.col, C4.col) and np.array_equal(C1.val, C4.val) and np.array_equal(S1, S4)
