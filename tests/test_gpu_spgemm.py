"""GPU parity of the product C = A B (paper Sec. 2) against the CPU oracle.

Pattern (row_ptr, col) must match bit for bit.  Values must satisfy
|dC_ij| <= tol * S_ij with S_ij = sum_k |a_ik||b_kj| (tol 1e-12 for float64,
1e-5 for float32); for rows on the deterministic sort accumulator the values
are also required to equal the oracle's bit for bit (same products, same
summation order, no fused multiply-add on either side)."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu

TOL = {np.float64: 1e-12, np.float32: 1e-5}


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


def run_product(tsg, A, B, handle, dtype=np.float64):
    dA = tsg.DeviceCSR.from_host(A.astype(dtype))
    dB = tsg.DeviceCSR.from_host(B.astype(dtype))
    C = tsg.spgemm(dA, dB, handle)
    torch.cuda.synchronize()
    return C.to_host()


def assert_matches(got, A, B, dtype=np.float64, exact=True):
    rp, col, val = got
    prec = "f32" if dtype == np.float32 else "f64"
    ref, S = oracle.spgemm(A.astype(dtype), B.astype(dtype), prec)
    assert np.array_equal(rp, ref.rowptr), "row_ptr"
    assert np.array_equal(col, ref.col), "col"
    err = np.abs(val.astype(np.float64) - ref.val.astype(np.float64))
    assert np.all(err <= TOL[dtype] * S), float((err / np.maximum(S, 1e-300)).max())
    if exact:
        assert np.array_equal(val, ref.val), "values not bit-identical to the oracle"


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_er_square_4096(tsg, handle, dtype):
    # 4096 x 4096, 8 per row, C = A A (the small ER workload)
    A = gen.er(4096, 4096, 8, 0, dtype)
    assert_matches(run_product(tsg, A, A, handle, dtype), A, A, dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape", [(300, 200, 500, 12, 9), (1000, 37, 2000, 30, 40), (129, 4000, 3, 60, 2),
                                   (2048, 2048, 2048, 1, 1), (777, 888, 999, 0, 10)])
def test_ragged_rectangular(tsg, handle, dtype, shape):
    m, k, n, dA, dB = shape
    A = gen.er_variable(m, k, dA, m + 1, dtype, "uniform", p_empty=0.1)
    B = gen.er_variable(k, n, dB, n + 2, dtype, "uniform", p_empty=0.1)
    assert_matches(run_product(tsg, A, B, handle, dtype), A, B, dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_every_bin_and_heavy_rows(tsg, handle, dtype):
    # u_i = |A_i| * 8 spans 0 .. ~9600 products: every bin boundary, the
    # heavy path, and rows straddling each threshold
    lens = np.concatenate([np.arange(0, 1200), [4, 8, 16, 32, 64, 128, 256, 512, 1024, 1025]])
    k = 3000
    rng = np.random.default_rng(5)
    rows = [np.sort(rng.choice(k, size=int(L), replace=False)) for L in lens]
    rp = np.zeros(len(lens) + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    A = gen.CSR(len(lens), k, rp, np.concatenate(rows).astype(np.int32),
                rng.uniform(-1, 1, int(rp[-1])).astype(dtype))
    B = gen.er(k, 5000, 8, 6, dtype)
    assert_matches(run_product(tsg, A, B, handle, dtype), A, B, dtype, exact=False)
    # rows on the on-chip bins (u <= 8192, |A_i| <= 4096) are bit-exact
    got = run_product(tsg, A, B, handle, dtype)
    ref, _ = oracle.spgemm(A.astype(dtype), B.astype(dtype), "f32" if dtype == np.float32 else "f64")
    u = oracle.row_products(A, B)
    for i in np.nonzero(u <= 8192)[0][::7]:
        s, e = ref.rowptr[i], ref.rowptr[i + 1]
        assert np.array_equal(got[2][s:e], ref.val[s:e])


def test_dense_row_many_column_chunks(tsg, handle):
    # one A row touching every B row, B wider than one 2^20-column pass:
    # the heavy path runs several chunks
    k, n = 3000, (1 << 21) + 77
    B = gen.er(k, n, 6, 11)
    A = gen.CSR(2, k, np.array([0, k, k + 3], dtype=np.int64),
                np.concatenate([np.arange(k), [5, 17, 2999]]).astype(np.int32),
                np.random.default_rng(1).uniform(-1, 1, k + 3))
    assert_matches(run_product(tsg, A, B, handle), A, B, exact=False)


def test_integer_values_exact(tsg, handle):
    A = gen.er_variable(3000, 2500, 40, 21, np.float64, "int", p_empty=0.05)
    B = gen.er_variable(2500, 3500, 40, 22, np.float64, "int", p_empty=0.05)
    assert_matches(run_product(tsg, A, B, handle), A, B)


def test_cancellation_keeps_explicit_zero(tsg, handle):
    A = gen.from_dense(np.array([[1.0, 1.0], [0.0, 2.0]]))
    B = gen.from_dense(np.array([[2.0, 1.0], [-2.0, 0.0]]))
    rp, col, val = run_product(tsg, A, B, handle)
    assert rp.tolist() == [0, 2, 3] and col.tolist() == [0, 1, 0] and val.tolist() == [0.0, 1.0, -4.0]


def test_empty_inputs(tsg, handle):
    A = gen.CSR(50, 40, np.zeros(51, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    B = gen.er(40, 30, 3, 0)
    rp, col, val = run_product(tsg, A, B, handle)
    assert rp.tolist() == [0] * 51 and col.size == 0
    A0 = gen.CSR(0, 40, np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    rp, col, val = run_product(tsg, A0, B, handle)
    assert rp.tolist() == [0] and col.size == 0
    # B with no entries: every product row is empty
    Bz = gen.CSR(40, 30, np.zeros(41, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    A2 = gen.er(50, 40, 5, 1)
    rp, col, val = run_product(tsg, A2, Bz, handle)
    assert rp.tolist() == [0] * 51


def test_deterministic_across_tunes_and_runs(tsg, handle):
    A = gen.er_variable(5000, 4000, 48, 31, np.float64, "normal")
    B = gen.er_variable(4000, 4500, 48, 32, np.float64, "normal")
    base = run_product(tsg, A, B, handle)
    again = run_product(tsg, A, B, handle)
    assert all(np.array_equal(x, y) for x, y in zip(base, again))
    # every row on the largest on-chip variant, fewer warps per block
    t = tsg.default_tune()
    t.num_bins = 1
    t.bin_upper[0] = 8192
    t.bin_kernel[0] = 8
    t.warps_per_block = 3
    handle.set_tune(t)
    other = run_product(tsg, A, B, handle)
    assert all(np.array_equal(x, y) for x, y in zip(base, other))
    # every row with more than one product on the heavy path
    t.bin_upper[0] = 1
    t.bin_kernel[0] = 0
    handle.set_tune(t)
    heavy = run_product(tsg, A, B, handle)
    assert np.array_equal(heavy[0], base[0]) and np.array_equal(heavy[1], base[1])
    ref, S = oracle.spgemm(A, B)
    assert np.all(np.abs(heavy[2] - ref.val) <= 1e-12 * S)
    handle.set_tune(None)


def test_validation_rejects_bad_input(tsg, handle):
    from paper_2603_21444_gb300._abi import SpgemmError
    t = tsg.default_tune()
    t.validate = 1
    handle.set_tune(t)
    A = gen.er(100, 50, 4, 0)
    B = gen.er(50, 60, 4, 1)
    bad = A.col.copy()
    bad[17] = 50  # column == ncols
    Abad = gen.CSR(A.nrows, A.ncols, A.rowptr, bad, A.val)
    with pytest.raises(SpgemmError) as e:
        run_product(tsg, Abad, B, handle)
    assert e.value.code == 9
    rp = A.rowptr.copy()
    rp[10], rp[11] = rp[11], rp[10]  # decreasing row pointer
    with pytest.raises(SpgemmError):
        run_product(tsg, gen.CSR(A.nrows, A.ncols, rp, A.col, A.val), B, handle)
    assert_matches(run_product(tsg, A, B, handle), A, B)
    handle.set_tune(None)


def test_shape_and_dtype_errors(tsg, handle):
    from paper_2603_21444_gb300._abi import SpgemmError
    A = tsg.DeviceCSR.from_host(gen.er(10, 20, 3, 0))
    B = tsg.DeviceCSR.from_host(gen.er(21, 5, 3, 1))
    with pytest.raises(SpgemmError) as e:
        tsg.spgemm(A, B, handle)
    assert e.value.code == 2


def test_index_overflow_reported(tsg, handle):
    # nnz(C) ~ 2^20 rows * ~4090 distinct > INT32_MAX: the symbolic call must
    # refuse with SPGEMM_ERR_INDEX_OVERFLOW (no numeric call can follow)
    from paper_2603_21444_gb300._abi import SpgemmError
    m = 1 << 20
    dev = "cuda"
    d = 64
    rp = torch.arange(0, (m + 1) * d, d, dtype=torch.int32, device=dev)
    g = torch.Generator(device=dev).manual_seed(0)
    acol = torch.randint(0, m, (m * d,), dtype=torch.int32, device=dev, generator=g)
    bcol = torch.randint(0, 1 << 24, (m * d,), dtype=torch.int32, device=dev, generator=g)
    acol = acol.view(m, d).sort(dim=1).values.reshape(-1)
    bcol = bcol.view(m, d).sort(dim=1).values.reshape(-1)
    A = tsg.DeviceCSR(m, m, rp, acol, None)
    B = tsg.DeviceCSR(m, 1 << 24, rp, bcol, None)
    with pytest.raises(SpgemmError) as e:
        tsg.symbolic(A, B, handle)
    assert e.value.code == 4


def test_full_size_er_sampled_rows(tsg, handle):
    # the benchmark workload: A, B ER n = 2^20, 16 per row, float64; compare
    # 4096 sampled rows with the oracle and check global properties
    n, d = 1 << 20, 16
    A = gen.er(n, n, d, 0)
    B = gen.er(n, n, d, 1)
    dA, dB = tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B)
    C = tsg.spgemm(dA, dB, handle)
    torch.cuda.synchronize()
    rp = C.row_ptr.cpu().numpy().astype(np.int64)
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and np.all(np.diff(rp) <= d * d)
    mean = C.nnz / n
    expect = d * d - d ** 3 * (d - 1) / (2.0 * n)
    assert abs(mean - expect) < 5 * np.sqrt((d * d - expect) / n) + 1e-3
    rows = np.sort(np.random.default_rng(0).choice(n, 4096, replace=False))
    lens = np.diff(A.rowptr)[rows]
    srp = np.zeros(rows.size + 1, dtype=np.int64)
    srp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows])
    As = gen.CSR(rows.size, n, srp, A.col[idx], A.val[idx])
    ref, S = oracle.spgemm(As, B)
    col = C.col.cpu().numpy()
    val = C.val.cpu().numpy()
    for t, r in enumerate(rows):
        s0, s1 = rp[r], rp[r + 1]
        o0, o1 = ref.rowptr[t], ref.rowptr[t + 1]
        assert np.array_equal(col[s0:s1], ref.col[o0:o1])
        assert np.array_equal(val[s0:s1], ref.val[o0:o1])


def _fused(tsg, A, B, handle, dtype=np.float64, cap=None):
    dA = tsg.DeviceCSR.from_host(A.astype(dtype))
    dB = tsg.DeviceCSR.from_host(B.astype(dtype))
    cap = tsg.products(dA, dB, handle) if cap is None else cap
    C = tsg.DeviceCSR(A.nrows, B.ncols, torch.empty(A.nrows + 1, dtype=torch.int32, device="cuda"),
                      torch.empty(cap, dtype=torch.int32, device="cuda"),
                      torch.empty(cap, dtype=torch.from_numpy(np.zeros(0, dtype)).dtype, device="cuda"))
    nnz = tsg.fused_into(dA, dB, C, handle)
    torch.cuda.synchronize()
    rp, col, val = C.to_host()
    return rp, col[:nnz], val[:nnz]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_single_pass_er(tsg, handle, dtype):
    A = gen.er(4096, 4096, 8, 0, dtype)
    assert_matches(_fused(tsg, A, A, handle, dtype), A, A, dtype)


@pytest.mark.parametrize("dmax", [12, 30, 90])
def test_single_pass_ragged_and_repeats(tsg, handle, dmax):
    # ragged rows spread over several warp bins (and, for dmax = 90, block
    # bins: the two-pass route); integer values make repeated columns exact
    A = gen.er_variable(3000, 500, dmax, 41, np.float64, "int", p_empty=0.1)
    B = gen.er_variable(500, 700, dmax, 42, np.float64, "int", p_empty=0.1)
    assert_matches(_fused(tsg, A, B, handle), A, B)


def test_single_pass_capacity_error(tsg, handle):
    from paper_2603_21444_gb300._abi import SpgemmError
    A = gen.er(2000, 2000, 8, 3)
    ref, _ = oracle.spgemm(A, A)
    with pytest.raises(SpgemmError) as e:
        _fused(tsg, A, A, handle, cap=ref.nnz - 1)
    assert e.value.code == 12
    # the handle recovers: the next call succeeds
    assert_matches(_fused(tsg, A, A, handle), A, A)


@pytest.mark.parametrize("spin_limit", [1, 1000])
def test_single_pass_bounded_wait_reports_timeout(tsg, handle, spin_limit):
    # injected on the host: tile 0 of the single pass never publishes its
    # look-back entry, so tile 1's wait runs out after spin_limit polls; the
    # call reports SPGEMM_ERR_DEVICE_TIMEOUT and the device stays usable
    from paper_2603_21444_gb300._abi import SpgemmError
    A = gen.er(4096, 4096, 8, 0)
    handle.set_wait_test(spin_limit, 0)
    with pytest.raises(SpgemmError) as e:
        _fused(tsg, A, A, handle)
    assert e.value.code == 7
    # a held tile beyond the last one changes nothing (default cap: with a
    # cap of a few polls an ordinary wait on a tile still being computed
    # could run out too)
    handle.set_wait_test(0, 1 << 30)
    assert_matches(_fused(tsg, A, A, handle), A, A)
    handle.set_wait_test()
    assert_matches(_fused(tsg, A, A, handle), A, A)
    with pytest.raises(SpgemmError) as e:
        handle.set_wait_test(0, -2)
    assert e.value.code == 1


def test_workspace_limit_reports_oom_and_recovers(tsg, handle):
    # allocation failure injected on the host: a call whose workspace would
    # grow past the handle's cap reports SPGEMM_ERR_OOM before allocating,
    # keeps the buffers it holds, and the handle stays usable and exact
    from paper_2603_21444_gb300._abi import SpgemmError
    A = gen.er(4096, 4096, 8, 0)
    handle.set_workspace_limit(0)
    with pytest.raises(SpgemmError) as e:
        run_product(tsg, A, A, handle)
    assert e.value.code == 5
    handle.set_workspace_limit(None)
    assert_matches(run_product(tsg, A, A, handle), A, A)
    held = handle.workspace_bytes()
    assert held > 0
    handle.set_workspace_limit(held)
    assert_matches(run_product(tsg, A, A, handle), A, A)  # fits in what is held
    A2 = gen.er(1 << 15, 1 << 15, 8, 1)
    with pytest.raises(SpgemmError) as e:
        run_product(tsg, A2, A2, handle)
    assert e.value.code == 5
    assert handle.workspace_bytes() == held
    assert_matches(run_product(tsg, A, A, handle), A, A)
    handle.set_workspace_limit(None)
    assert_matches(run_product(tsg, A2, A2, handle), A2, A2)


def test_single_pass_full_size_matches_two_pass(tsg, handle):
    n, d = 1 << 20, 16
    A = gen.er(n, n, d, 0)
    B = gen.er(n, n, d, 1)
    dA, dB = tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B)
    C2 = tsg.spgemm(dA, dB, handle)
    C1 = tsg.spgemm_single_pass(dA, dB, handle)
    torch.cuda.synchronize()
    assert torch.equal(C1.row_ptr, C2.row_ptr)
    assert torch.equal(C1.col, C2.col)
    assert torch.equal(C1.val, C2.val)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("da,db", [(32, 10), (40, 8), (12, 30), (20, 3), (31, 12), (6, 50)])
def test_gather_orders_and_384_variant(tsg, handle, dtype, da, db):
    # the strided gather (at most 32 A entries, mean B row below 16), the
    # chunked gather (more A entries or long B rows) and the 384-product warp
    # variant (u in (256, 384]) against the oracle, bit for bit; repeated
    # columns come from a narrow B
    A = gen.er(3000, 1500, da, 71 + da, dtype, "normal")
    B = gen.er(1500, 600, db, 72 + db, dtype, "normal")
    assert_matches(run_product(tsg, A, B, handle, dtype), A, B, dtype)


def test_gather_orders_ragged_b_rows(tsg, handle):
    # B rows of every length 0..24 at every alignment; A rows of 0..16
    # entries, so that u <= 384 and every row fits either forced variant
    A = gen.er_variable(4000, 3000, 16, 81, np.float64, "normal", p_empty=0.05)
    B = gen.er_variable(3000, 900, 24, 82, np.float64, "normal", p_empty=0.1)
    assert_matches(run_product(tsg, A, B, handle), A, B)
    # the same rows forced onto the 384 variant and onto the 512 variant
    for kernel, upper in ((9, 384), (4, 512)):
        t = tsg.default_tune()
        t.num_bins = 1
        t.bin_upper[0] = upper
        t.bin_kernel[0] = kernel
        handle.set_tune(t)
        assert_matches(run_product(tsg, A, B, handle), A, B)
    handle.set_tune(None)
