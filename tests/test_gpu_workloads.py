"""GPU parity of the permutation kernel (Y = P X Q^T), the device trident
loads, and the restriction-operator product C = A R, all through the C ABI,
against the oracle."""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tsg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2603_21444_gb300 as m
    return m


@pytest.fixture()
def handle(tsg):
    h = tsg.Handle()
    yield h
    assert h.device_status() == 0
    h.close()


def _maps(m, n, s1, s2, rows=True, cols=True):
    rp = gen.random_permutation(m, s1) if rows else None
    cp = gen.random_permutation(n, s2) if cols else None
    dev = lambda p: torch.from_numpy(p).cuda() if p is not None else None
    return rp, cp, dev(rp), dev(cp)


def _same(Y, ref):
    rp, col, val = Y.to_host()
    assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
    if val is not None:
        assert np.array_equal(val, ref.val)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("rows,cols", [(True, True), (True, False), (False, True), (False, False)])
def test_permute_matches_oracle(tsg, handle, dtype, rows, cols):
    X = gen.er_variable(3000, 2500, 40, 21, dtype, "normal", p_empty=0.1)
    rp, cp, drp, dcp = _maps(3000, 2500, 5, 6, rows, cols)
    Y = tsg.permute(tsg.DeviceCSR.from_host(X), drp, dcp, handle)
    torch.cuda.synchronize()
    _same(Y, oracle.permute(X, rp, cp))


def test_permute_banded_and_long_rows(tsg, handle):
    # a banded matrix plus rows longer than one warp's on-chip sort (1024):
    # dense rows of 1025, 3000 and 5000 entries take the block path
    n = 6000
    B = gen.banded(n, [-1500, 0, 1500], 4, 3)
    D = gen.er_variable(n, n, 2, 4)
    dense_rows = {17: 1025, 2000: 3000, 5999: 5000}
    rows, cols, vals = [], [], []
    for i in range(n):
        if i in dense_rows:
            c = np.sort(np.random.default_rng(i).choice(n, dense_rows[i], replace=False))
        else:
            c = B.col[B.rowptr[i]:B.rowptr[i + 1]]
        rows.append(np.full(c.size, i))
        cols.append(c)
        vals.append(np.random.default_rng(n + i).standard_normal(c.size))
    X = gen.from_coo(n, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    del D
    rp, cp, drp, dcp = _maps(n, n, 7, 8)
    Y = tsg.permute(tsg.DeviceCSR.from_host(X), drp, dcp, handle)
    torch.cuda.synchronize()
    _same(Y, oracle.permute(X, rp, cp))


def test_permute_pattern_only_and_empty(tsg, handle):
    X = gen.er_variable(500, 400, 9, 9)
    rp, cp, drp, dcp = _maps(500, 400, 1, 2)
    dX = tsg.DeviceCSR.from_host(X)
    Xp = tsg.DeviceCSR(dX.nrows, dX.ncols, dX.row_ptr, dX.col, None)
    Y = tsg.permute(Xp, drp, dcp, handle)
    torch.cuda.synchronize()
    ref = oracle.permute(X, rp, cp)
    assert np.array_equal(Y.row_ptr.cpu().numpy(), ref.rowptr) and np.array_equal(Y.col.cpu().numpy(), ref.col)
    E = gen.CSR(300, 200, np.zeros(301, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    _, _, drp, dcp = _maps(300, 200, 3, 4)
    Y = tsg.permute(tsg.DeviceCSR.from_host(E), drp, dcp, handle)
    torch.cuda.synchronize()
    assert np.all(Y.row_ptr.cpu().numpy() == 0)


def test_permute_rejects_non_permutations(tsg, handle):
    from paper_2603_21444_gb300._abi import SpgemmError
    X = gen.er_variable(400, 300, 8, 12)
    dX = tsg.DeviceCSR.from_host(X)
    bad = gen.random_permutation(400, 1).copy()
    bad[5] = bad[6]  # two rows sent to one target (in range)
    with pytest.raises(SpgemmError) as e:
        tsg.permute(dX, torch.from_numpy(bad).cuda(), None, handle)
    assert e.value.code == 1
    out = gen.random_permutation(300, 2).copy()
    out[0] = 300  # out of range: checked before any use
    with pytest.raises(SpgemmError):
        tsg.permute(dX, None, torch.from_numpy(out).cuda(), handle)
    # the handle recovers
    rp, cp, drp, dcp = _maps(400, 300, 3, 4)
    Y = tsg.permute(dX, drp, dcp, handle)
    torch.cuda.synchronize()
    _same(Y, oracle.permute(X, rp, cp))


@pytest.mark.parametrize("q,lam", [(4, 4), (8, 4), (3, 2)])
def test_trident_loads_match_oracle(tsg, handle, q, lam):
    X = gen.banded(5000, [0, 1200], 5, 6)
    loads = np.array(tsg.trident_loads(tsg.DeviceCSR.from_host(X), q, lam, handle))
    assert np.array_equal(loads, oracle.trident_loads(X, q, lam))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_restriction_product(tsg, handle, dtype):
    # C = A R, R an aggregation restriction (n x n/4, one entry per row)
    A = gen.er(6000, 6000, 16, 31, dtype, "normal")
    R = gen.aggregation(6000, 4, 32, dtype)
    C = tsg.spgemm(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(R), handle)
    torch.cuda.synchronize()
    ref, _ = oracle.spgemm(A, R, "f32" if dtype == np.float32 else "f64")
    _same(C, ref)


def test_restriction_full_size_sampled_rows(tsg, handle):
    # the restriction workload: A ER n = 2^20, 16 per row, float64; R n x n/4
    n = 1 << 20
    A = gen.er(n, n, 16, 0)
    R = gen.aggregation(n, 4, 7)
    C = tsg.spgemm(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(R), handle)
    torch.cuda.synchronize()
    rp = C.row_ptr.cpu().numpy().astype(np.int64)
    rows = np.sort(np.random.default_rng(1).choice(n, 4096, replace=False))
    lens = np.diff(A.rowptr)[rows]
    srp = np.zeros(rows.size + 1, dtype=np.int64)
    srp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows])
    ref, _ = oracle.spgemm(gen.CSR(rows.size, n, srp, A.col[idx], A.val[idx]), R)
    col, val = C.col.cpu().numpy(), C.val.cpu().numpy()
    for t, r in enumerate(rows):
        assert np.array_equal(col[rp[r]:rp[r + 1]], ref.col[ref.rowptr[t]:ref.rowptr[t + 1]])
        assert np.array_equal(val[rp[r]:rp[r + 1]], ref.val[ref.rowptr[t]:ref.rowptr[t + 1]])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("offsets,hw", [([0], 4), ([-700, 0, 700], 4), ([0, 5], 2), ([-1100, 0, 900], 7)])
def test_banded_products(tsg, handle, dtype, offsets, hw):
    # clustered, heavily repeated columns: rows deferred to the grouped
    # accumulation (u >= 4 nnz(C_i), few columns) and rows that stay on the
    # buckets, all bit-identical to the oracle
    A = gen.banded(3000, offsets, hw, 11, dtype, "normal")
    B = gen.banded(3000, offsets, hw, 12, dtype, "normal")
    C = tsg.spgemm(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), handle)
    torch.cuda.synchronize()
    ref, _ = oracle.spgemm(A, B, "f32" if dtype == np.float32 else "f64")
    _same(C, ref)


def test_banded_trident_grid(tsg, handle):
    # the grouped accumulation with several instances per output row (the
    # fused trident grid) and with partials (merge mode of the unfused path)
    n, q, lam = 2048, 4, 2
    A = gen.banded(n, [-300, 0, 300], 4, 13, np.float64, "normal")
    B = gen.banded(n, [-300, 0, 300], 4, 14, np.float64, "normal")
    ref, _ = oracle.trident_product(A, B, q, lam)
    plan = tsg.TridentPlan(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), q, lam, handle)
    fused = plan.run_fused(use_graph=False)
    unfused = plan.run_unfused()
    torch.cuda.synchronize()
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                g = plan.block_index(i, j, k)
                _same(fused[g], ref[i][j][k])
                _same(unfused[g], ref[i][j][k])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tiny_rows_thread_variant(tsg, handle, dtype):
    # rows of at most 16 products run one thread per row; ragged rows mix
    # the thread variant with the warp variants
    for A, B in ((gen.er(5000, 5000, 4, 41, dtype, "normal"), gen.er(5000, 5000, 4, 42, dtype, "normal")),
                 (gen.er_variable(4000, 300, 5, 43, dtype, "normal", p_empty=0.1),
                  gen.er_variable(300, 200, 5, 44, dtype, "normal", p_empty=0.1)),
                 (gen.er_variable(3000, 2000, 4, 45, dtype, "int"), gen.er(2000, 40, 4, 46, dtype, "int"))):
        C = tsg.spgemm(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), handle)
        torch.cuda.synchronize()
        ref, _ = oracle.spgemm(A, B, "f32" if dtype == np.float32 else "f64")
        _same(C, ref)


def test_tiny_rows_trident_grid(tsg, handle):
    # several instances (fused) and partials (unfused merge) on tiny rows
    n, q, lam = 2048, 4, 2
    A = gen.er(n, n, 4, 47, np.float64, "normal")
    B = gen.er(n, n, 4, 48, np.float64, "normal")
    ref, _ = oracle.trident_product(A, B, q, lam)
    plan = tsg.TridentPlan(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), q, lam, handle)
    fused = plan.run_fused(use_graph=False)
    unfused = plan.run_unfused()
    torch.cuda.synchronize()
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                g = plan.block_index(i, j, k)
                _same(fused[g], ref[i][j][k])
                _same(unfused[g], ref[i][j][k])


def test_split_then_deferred_product_same_handle(tsg, handle):
    # the tile split sizes the handle's per-unit workspace for rows x column
    # tiles units; a later product on the same handle, with rows deferred to
    # the grouped kernel, keeps its deferred-row list inside that workspace
    X = gen.banded(6000, [-1500, 0, 1500], 4, 3, np.float64, "normal")
    dX = tsg.DeviceCSR.from_host(X)
    loads = tsg.trident_loads(dX, 8, 4, handle)
    assert sum(map(sum, loads)) == X.nnz
    C = tsg.spgemm(dX, dX, handle)
    torch.cuda.synchronize()
    ref, _ = oracle.spgemm(X, X)
    _same(C, ref)


def test_permute_row_too_long_to_resort(tsg, handle):
    from paper_2603_21444_gb300._abi import SpgemmError
    n = 70000
    rows = np.concatenate([np.zeros(n, dtype=np.int64), np.arange(1, 50)])
    cols = np.concatenate([np.arange(n), np.arange(1, 50)])
    X = gen.from_coo(50, n, rows, cols, np.ones(rows.size))
    dX = tsg.DeviceCSR.from_host(X)
    rp, cp, drp, dcp = _maps(50, n, 1, 2)
    with pytest.raises(SpgemmError) as e:
        tsg.permute(dX, drp, dcp, handle)
    assert e.value.code == 11
    # a row map alone needs no re-sort
    Y = tsg.permute(dX, drp, None, handle)
    torch.cuda.synchronize()
    _same(Y, oracle.permute(X, rp, None))
