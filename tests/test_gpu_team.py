"""GPU parity of the block-team counting-sort variants (11-14: 128, 256, 512
and 1024 threads holding 1024, 2048, 4096 and 8192 products of a row; 16-19:
the same with the row's B segments staged in shared memory by TMA) against
the CPU oracle (Sec. 2's row-wise product): patterns and values bit for bit,
in product, multi-instance (trident) and merge mode, with and without
repeated columns, with one bucket per column (narrow outputs), and against
the rank-in-bucket block variants 5-8, which add in the same order."""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu

TEAM = {11: 1024, 12: 2048, 13: 4096, 14: 8192, 16: 1024, 17: 2048, 18: 4096, 19: 8192}
RANK = {11: 5, 12: 6, 13: 7, 14: 8, 16: 5, 17: 6, 18: 7, 19: 8}
STAGED = (16, 17, 18, 19)  # B rows staged in shared memory by TMA bulk copies


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


def one_bin(tsg, upper, kernel):
    t = tsg.default_tune()
    t.num_bins = 1
    t.bin_upper[0] = upper
    t.bin_kernel[0] = kernel
    return t


def product(tsg, A, B, handle, dtype=np.float64):
    dA = tsg.DeviceCSR.from_host(A.astype(dtype))
    dB = tsg.DeviceCSR.from_host(B.astype(dtype))
    C = tsg.spgemm(dA, dB, handle)
    torch.cuda.synchronize()
    return C.to_host()


def exact(got, ref):
    rp, col, val = got
    assert np.array_equal(rp, ref.rowptr), "row_ptr"
    assert np.array_equal(col, ref.col), "col"
    assert np.array_equal(val, ref.val), "values not bit-identical to the oracle"


def rows_of_lengths(lens, k, seed, dtype):
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(k, size=int(L), replace=False)) for L in lens]
    rp = np.zeros(len(lens) + 1, dtype=np.int64)
    rp[1:] = np.cumsum(lens)
    return gen.CSR(len(lens), k, rp, np.concatenate(rows).astype(np.int32),
                   rng.uniform(-1, 1, int(rp[-1])).astype(dtype))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_default_bins_rows_513_to_8192(tsg, handle, dtype):
    # u_i = 8 |A_i| from 8 to 8192 products: every team bin, their edges
    lens = np.concatenate([np.arange(64, 1025, 3), [64, 65, 128, 129, 256, 257, 512, 513, 1023, 1024]])
    A = rows_of_lengths(lens, 3000, 7, dtype)
    B = gen.er(3000, 6000, 8, 8, dtype)
    prec = "f32" if dtype == np.float32 else "f64"
    exact(product(tsg, A, B, handle, dtype), oracle.spgemm(A, B, prec)[0])


@pytest.mark.parametrize("variant", sorted(TEAM))
def test_each_team_variant_alone_equals_rank_variant(tsg, handle, variant):
    # every row (from 1 product up to the variant's capacity) on one variant:
    # small rows leave most bucket slices and warps empty
    cap = TEAM[variant]
    lens = np.concatenate([np.arange(0, cap // 8 + 1, max(1, cap // 512)), [1, 2, cap // 16, cap // 8]])
    A = rows_of_lengths(lens, 2500, variant, np.float64)
    B = gen.er(2500, 40000, 8, variant + 1)
    ref = oracle.spgemm(A, B)[0]
    handle.set_tune(one_bin(tsg, cap, variant))
    team = product(tsg, A, B, handle)
    handle.set_tune(one_bin(tsg, cap, RANK[variant]))
    rank = product(tsg, A, B, handle)
    handle.set_tune(None)
    exact(team, ref)
    assert all(np.array_equal(x, y) for x, y in zip(team, rank))


@pytest.mark.parametrize("ncols", [7, 300, 1000, 5000])
def test_narrow_output_one_bucket_per_column(tsg, handle, ncols):
    # rows of 600..4000 products onto few columns: many repeats per column,
    # buckets are single columns (a dense accumulator), sums in p order
    lens = np.arange(60, 400, 13)
    A = rows_of_lengths(lens, 1500, ncols, np.float64)
    B = gen.er_variable(1500, ncols, min(ncols, 14), ncols + 3, np.float64, "normal", p_empty=0.05)
    exact(product(tsg, A, B, handle), oracle.spgemm(A, B)[0])


def test_integer_values_and_cancellation(tsg, handle):
    A = gen.er_variable(2000, 1800, 120, 41, np.float64, "int", p_empty=0.05)
    B = gen.er_variable(1800, 2200, 60, 42, np.float64, "int", p_empty=0.05)
    exact(product(tsg, A, B, handle), oracle.spgemm(A, B)[0])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_merge_mode_long_rows(tsg, handle, dtype):
    # 5 partials with rows of ~150..400 entries: merged rows of 800..2000
    parts = [gen.er_variable(1500, 40000, 300 + 40 * t, 60 + t, dtype, "normal", p_empty=0.05) for t in range(5)]
    C = tsg.merge([tsg.DeviceCSR.from_host(P) for P in parts], handle)
    torch.cuda.synchronize()
    exact(C.to_host(), oracle.csr_sum(parts))


def test_trident_grid_with_long_rows(tsg, handle):
    # 3 x 3 x 2 grid over ER n = 3000, 48 per row: rows of ~4 x 16 x 16
    # products over 3 instances land on the team variants
    A = gen.er(3000, 3000, 48, 71)
    B = gen.er(3000, 3000, 48, 72)
    plan = tsg.TridentPlan(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), 3, 2, handle)
    blocks = plan.run_fused()
    torch.cuda.synchronize()
    ref, _ = oracle.trident_product(A, B, 3, 2)
    for i in range(3):
        for j in range(3):
            for k in range(2):
                exact(blocks[plan.block_index(i, j, k)].to_host(), ref[i][j][k])


def test_batch_of_uneven_products(tsg, handle):
    # the many-products shapes at small n: rows of d^2 products up to 4096
    shapes = [(1200, 64), (900, 40), (3000, 23), (1024, 64), (2000, 33), (700, 5)]
    pairs = [(gen.er(n, n, d, 1000 + 2 * t), gen.er(n, n, d, 1001 + 2 * t)) for t, (n, d) in enumerate(shapes)]
    Cs = tsg.batched([tsg.DeviceCSR.from_host(a) for a, _ in pairs], [tsg.DeviceCSR.from_host(b) for _, b in pairs],
                     handle=handle)
    torch.cuda.synchronize()
    for (a, b), C in zip(pairs, Cs):
        exact(C.to_host(), oracle.spgemm(a, b)[0])


def test_concurrent_and_sequential_bins_agree(tsg, handle):
    # the per-bin launches forked onto the handle's streams (default) and
    # issued one after another give the same bits, direct and from a graph
    shapes = [(1500, 60), (800, 30), (3000, 12), (1024, 64), (2500, 20), (600, 3)]
    pairs = [(gen.er(n, n, d, 3000 + 2 * t), gen.er(n, n, d, 3001 + 2 * t)) for t, (n, d) in enumerate(shapes)]
    As = [tsg.DeviceCSR.from_host(a) for a, _ in pairs]
    Bs = [tsg.DeviceCSR.from_host(b) for _, b in pairs]
    plan = tsg.Plan(As, Bs)
    outs = []
    for conc in (True, False, True):
        plan.set_concurrent_bins(conc)
        for C in plan.C:
            C.val.zero_()
            C.col.zero_()
        plan.execute(False)
        plan.execute(True)
        Cs = plan.execute(True)
        torch.cuda.synchronize()
        outs.append([C.to_host() for C in Cs])
    plan.close()
    for (a, b), got in zip(pairs, outs[0]):
        exact(got, oracle.spgemm(a, b)[0])
    for other in outs[1:]:
        for x, y in zip(outs[0], other):
            assert all(np.array_equal(p, q) for p, q in zip(x, y))
    # a handle's direct calls, both ways
    handle.set_concurrent_bins(False)
    seq = [product(tsg, a, b, handle) for a, b in pairs[:3]]
    handle.set_concurrent_bins(True)
    con = [product(tsg, a, b, handle) for a, b in pairs[:3]]
    for x, y in zip(seq, con):
        assert all(np.array_equal(p, q) for p, q in zip(x, y))


@pytest.mark.parametrize("variant", STAGED)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_staged_variants_ragged_b_rows(tsg, handle, variant, dtype):
    # B rows of every length 0..40 (so every start and end alignment, empty
    # rows, and the arrays' last row), A rows of up to 128 entries (staged)
    # and some longer (gathered from global memory)
    cap = TEAM[variant]
    B = gen.er_variable(3000, 5000, 40, variant, dtype, "normal", p_empty=0.05)
    lens = np.concatenate([np.arange(1, 129, 3), [129, 200, 300], [2999, 2998]])
    A = rows_of_lengths(lens, 3000, variant + 50, dtype)
    # rows beyond the variant's capacity are emptied
    u = oracle.row_products(A, B)
    lens_kept = np.where(u <= cap, np.diff(A.rowptr), 0)
    mask = np.repeat(u <= cap, np.diff(A.rowptr))
    rp = np.zeros(A.nrows + 1, dtype=np.int64)
    np.cumsum(lens_kept, out=rp[1:])
    A = gen.CSR(A.nrows, A.ncols, rp, A.col[mask], A.val[mask])
    prec = "f32" if dtype == np.float32 else "f64"
    handle.set_tune(one_bin(tsg, cap, variant))
    got = product(tsg, A, B, handle, dtype)
    handle.set_tune(None)
    exact(got, oracle.spgemm(A, B, prec)[0])


def test_staged_variant_merge_and_trident(tsg, handle):
    # merge mode (partials as B rows) and multi-instance rows on a staged variant
    parts = [gen.er_variable(1200, 40000, 300 + 40 * t, 80 + t, np.float64, "normal", p_empty=0.05) for t in range(4)]
    handle.set_tune(one_bin(tsg, 2048, 17))
    C = tsg.merge([tsg.DeviceCSR.from_host(P) for P in parts], handle)
    torch.cuda.synchronize()
    exact(C.to_host(), oracle.csr_sum(parts))
    A = gen.er(3000, 3000, 48, 73)
    B = gen.er(3000, 3000, 48, 74)
    plan = tsg.TridentPlan(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), 3, 2, handle)
    t = one_bin(tsg, 2048, 17)
    blocks = tsg.Plan(plan.As, plan.Bs, plan.group_ptr, tune=t).execute(True)
    torch.cuda.synchronize()
    handle.set_tune(None)
    ref, _ = oracle.trident_product(A, B, 3, 2)
    for i in range(3):
        for j in range(3):
            for k in range(2):
                exact(blocks[plan.block_index(i, j, k)].to_host(), ref[i][j][k])
