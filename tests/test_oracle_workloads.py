"""Pins of the oracle's permutation and trident-load functions and of the
restriction-operator workload (C = A R with an aggregation R), each against
something other than the function itself: dense brute force, products with
permutation matrices through the oracle's own SpGEMM, closed forms."""
import numpy as np
import pytest

import gen
import oracle


def _inverse(p):
    inv = np.empty_like(p)
    inv[p] = np.arange(p.size, dtype=p.dtype)
    return inv


@pytest.mark.parametrize("shape", [(7, 5), (40, 40), (33, 90)])
def test_permute_matches_dense_relabelling(shape):
    m, n = shape
    X = gen.er_variable(m, n, min(n, 9), 3, np.float64, "int", p_empty=0.2)
    rp, cp = gen.random_permutation(m, 1), gen.random_permutation(n, 2)
    Y = oracle.permute(X, rp, cp)
    D = X.to_dense()
    E = np.zeros_like(D)
    E[np.ix_(rp, cp)] = D  # E[rp[i], cp[j]] = D[i, j]
    assert np.array_equal(Y.to_dense(), E)
    for i in range(m):  # rows sorted, no repeats
        c = Y.col[Y.rowptr[i]:Y.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_permute_equals_permutation_matrix_products():
    # Y = P X Q with P[i, inv_r[i]] = 1 and Q[j, cp[j]] = 1, through oracle.spgemm
    X = gen.er_variable(300, 200, 12, 5, np.float64, "int")
    rp, cp = gen.random_permutation(300, 6), gen.random_permutation(200, 7)
    P = gen.permutation_matrix(_inverse(rp))
    Q = gen.permutation_matrix(cp)
    PX, _ = oracle.spgemm(P, X)
    ref, _ = oracle.spgemm(PX, Q)
    Y = oracle.permute(X, rp, cp)
    assert np.array_equal(Y.rowptr, ref.rowptr) and np.array_equal(Y.col, ref.col)
    assert np.array_equal(Y.val, ref.val)


def test_permute_identity_and_inverse():
    X = gen.er_variable(120, 80, 10, 8, np.float64, "normal")
    Y = oracle.permute(X, None, None)
    assert np.array_equal(Y.rowptr, X.rowptr) and np.array_equal(Y.col, X.col) and np.array_equal(Y.val, X.val)
    rp, cp = gen.random_permutation(120, 9), gen.random_permutation(80, 10)
    Z = oracle.permute(oracle.permute(X, rp, cp), _inverse(rp), _inverse(cp))
    assert np.array_equal(Z.rowptr, X.rowptr) and np.array_equal(Z.col, X.col) and np.array_equal(Z.val, X.val)


def test_trident_loads_closed_forms():
    # all-ones n x n, q | n and lam | n / q: every part holds (n / (q lam)) (n / q)
    n, q, lam = 48, 4, 3
    X = gen.from_dense(np.ones((n, n)))
    L = oracle.trident_loads(X, q, lam)
    assert L.shape == (q * lam, q) and np.all(L == (n // (q * lam)) * (n // q))
    # a diagonal matrix: only the parts on the coarse diagonal hold entries,
    # each slice its own rows
    D = gen.identity(n)
    L = oracle.trident_loads(D, q, lam)
    for a in range(q * lam):
        for b in range(q):
            assert L[a, b] == (n // (q * lam) if a // lam == b else 0)
    # any matrix: the loads add up to nnz
    R = gen.er_variable(100, 70, 9, 4)
    assert oracle.trident_loads(R, 3, 2).sum() == R.nnz


def test_banded_generator_and_its_imbalance():
    n = 64
    B = gen.banded(n, [-16, 0, 16], 2, 1)
    D = B.to_dense() != 0
    i, j = np.nonzero(D)
    d = j - i
    assert set(np.unique(d)) <= set(range(-18, -13)) | set(range(-2, 3)) | set(range(14, 19))
    # interior rows hold all 15 columns
    assert np.all(D[20:44].sum(axis=1) == 15)
    # narrow bands pile up on the coarse diagonal: about q times the mean
    # there, while a random relabelling spreads them evenly
    n = 4096
    B = gen.banded(n, [0, 7], 3, 2)
    L = oracle.trident_loads(B, 4, 4)
    P = oracle.permute(B, gen.random_permutation(n, 3), gen.random_permutation(n, 4))
    Lp = oracle.trident_loads(P, 4, 4)
    assert L.sum() == Lp.sum() == B.nnz
    assert L.max() / L.mean() > 3.5
    assert Lp.max() / Lp.mean() < 1.3


def test_aggregation_restriction_product():
    # C = A R for an unsmoothed aggregation R: C[i, a] = sum of A[i, k] over
    # the nodes k of aggregate a (dense matmul, exact for integers)
    n, ratio = 203, 4
    R = gen.aggregation(n, ratio, 11)
    assert R.ncols == -(-n // ratio) and np.all(np.diff(R.rowptr) == 1)
    sizes = np.bincount(R.col, minlength=R.ncols)
    assert np.all(sizes[:-1] == ratio) and 1 <= sizes[-1] <= ratio
    A = gen.er_variable(150, n, 20, 12, np.float64, "int", p_empty=0.1)
    C, _ = oracle.spgemm(A, R)
    assert np.array_equal(C.to_dense(), A.to_dense() @ R.to_dense())
    # row sums survive the restriction (R 1 = 1)
    assert np.array_equal(C.to_dense().sum(axis=1), A.to_dense().sum(axis=1))
