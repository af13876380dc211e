"""GPU parity of the ordered sum of partials (Sec. 4.4) and of the batched
trident grid (Alg. 1 + Alg. 2 on one device) against the CPU oracle."""
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


def host(C):
    rp, col, val = C.to_host()
    return rp, col, val


def same(C, ref):
    rp, col, val = host(C)
    assert np.array_equal(rp, ref.rowptr)
    assert np.array_equal(col, ref.col)
    assert np.array_equal(val, ref.val)


@pytest.mark.parametrize("nparts", [1, 2, 4, 7])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_merge_matches_ordered_sum(tsg, handle, nparts, dtype):
    parts = [gen.er_variable(3000, 2500, 30 + 7 * t, 40 + t, dtype, "normal", p_empty=0.1) for t in range(nparts)]
    dparts = [tsg.DeviceCSR.from_host(P) for P in parts]
    C = tsg.merge(dparts, handle)
    torch.cuda.synchronize()
    same(C, oracle.csr_sum(parts))


def test_merge_order_matters(tsg, handle):
    P0 = gen.from_dense(np.array([[1e16, 0.0, 2.0]]))
    P1 = gen.from_dense(np.array([[1.0, 3.0, 0.0]]))
    P2 = gen.from_dense(np.array([[-1e16, 0.0, 0.0]]))
    d = [tsg.DeviceCSR.from_host(P) for P in (P0, P1, P2)]
    assert host(tsg.merge(d, handle))[2].tolist() == [0.0, 3.0, 2.0]
    assert host(tsg.merge([d[0], d[2], d[1]], handle))[2].tolist() == [1.0, 3.0, 2.0]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batched_independent_products(tsg, handle, dtype):
    shapes = gen.er_batch_shapes(24, seed=999, log2_lo=6, log2_hi=11)
    pairs = [(gen.er(n, n, min(d, n), 1000 + 2 * t, dtype), gen.er(n, n, min(d, n), 1001 + 2 * t, dtype))
             for t, (n, d) in enumerate(shapes)]
    As = [tsg.DeviceCSR.from_host(a) for a, _ in pairs]
    Bs = [tsg.DeviceCSR.from_host(b) for _, b in pairs]
    Cs = tsg.batched(As, Bs, handle=handle)
    torch.cuda.synchronize()
    prec = "f32" if dtype == np.float32 else "f64"
    for (a, b), C in zip(pairs, Cs):
        same(C, oracle.spgemm(a, b, prec)[0])


@pytest.mark.parametrize("q,lam,values", [(4, 4, "uniform"), (3, 2, "int"), (2, 4, "normal")])
def test_batched_trident_grid_matches_oracle(tsg, handle, q, lam, values):
    n, d = 1 << 12, 32
    A = gen.er(n, n, d, 4, np.float64, values)
    B = gen.er(n, n, d, 5, np.float64, values)
    A_s, B_t = oracle.trident_partition(A, B, q, lam)
    ref, _ = oracle.trident_product(A, B, q, lam)
    dA = {(i, r, k): tsg.DeviceCSR.from_host(A_s[i][r][k]) for i in range(q) for r in range(q) for k in range(lam)}
    dB = {(r, j): tsg.DeviceCSR.from_host(B_t[r][j]) for r in range(q) for j in range(q)}
    As, Bs, gp, keys = [], [], [0], []
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                for r in oracle.static_cannon_schedule(q, i, j):
                    As.append(dA[(i, r, k)])
                    Bs.append(dB[(r, j)])
                gp.append(len(As))
                keys.append((i, j, k))
    Cs = tsg.batched(As, Bs, gp, handle=handle)
    torch.cuda.synchronize()
    for (i, j, k), C in zip(keys, Cs):
        same(C, ref[i][j][k])


def test_batched_with_empty_group_rows(tsg, handle):
    a0 = gen.er(0, 10, 0, 0)
    b0 = gen.er(10, 7, 2, 1)
    a1 = gen.er(33, 10, 3, 2)
    a2 = gen.CSR(5, 10, np.zeros(6, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0))
    As = [tsg.DeviceCSR.from_host(x) for x in (a0, a1, a2)]
    Bs = [tsg.DeviceCSR.from_host(b0)] * 3
    Cs = tsg.batched(As, Bs, handle=handle)
    torch.cuda.synchronize()
    assert host(Cs[0])[0].tolist() == [0]
    same(Cs[1], oracle.spgemm(a1, b0)[0])
    assert host(Cs[2])[0].tolist() == [0] * 6


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tile_split_matches_oracle_submatrix(tsg, handle, dtype):
    X = gen.er_variable(1000, 900, 40, 77, dtype, "normal", p_empty=0.1)
    dX = tsg.DeviceCSR.from_host(X)
    _, rb = oracle.trident_bounds(X.nrows, 3, 2)
    cb, _ = oracle.trident_bounds(X.ncols, 5, 1)
    tiles = tsg.tile_split(dX, rb, cb, handle)
    torch.cuda.synchronize()
    for r in range(len(rb) - 1):
        for c in range(len(cb) - 1):
            same(tiles[r][c], oracle.submatrix(X, rb[r], rb[r + 1], cb[c], cb[c + 1]))


@pytest.mark.parametrize("q,lam", [(4, 4), (3, 2), (1, 1)])
def test_trident_plan_fused_and_unfused(tsg, handle, q, lam):
    n, d = 1 << 12, 32
    A = gen.er(n, n, d, 4, np.float64, "uniform")
    B = gen.er(n, n, d, 5, np.float64, "uniform")
    ref, _ = oracle.trident_product(A, B, q, lam)
    plan = tsg.TridentPlan(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), q, lam, handle)
    fused = plan.run_fused(use_graph=False)
    for C in fused:
        C.val.zero_()
    fused = plan.run_fused(use_graph=True)       # direct run + capture
    for C in fused:
        C.val.zero_()
    fused = plan.run_fused(use_graph=True)       # graph replay
    unfused = plan.run_unfused()
    plain = plan.run_plain()
    torch.cuda.synchronize()
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                g = plan.block_index(i, j, k)
                same(fused[g], ref[i][j][k])
                same(unfused[g], ref[i][j][k])
                same(plain[g], ref[i][j][k])


def test_plan_autotune_keeps_bits(tsg, handle):
    shapes = gen.er_batch_shapes(16, seed=999, log2_lo=8, log2_hi=12)
    pairs = [(gen.er(n, n, min(d, n), 2000 + 2 * t), gen.er(n, n, min(d, n), 2001 + 2 * t))
             for t, (n, d) in enumerate(shapes)]
    As = [tsg.DeviceCSR.from_host(a) for a, _ in pairs]
    Bs = [tsg.DeviceCSR.from_host(b) for _, b in pairs]
    plan = tsg.Plan(As, Bs)
    t = plan.autotune()
    assert 1 <= t.num_bins <= 12 and 1 <= t.warps_per_block <= 32
    Cs = plan.execute()
    Cs = plan.execute()
    torch.cuda.synchronize()
    for (a, b), C in zip(pairs, Cs):
        same(C, oracle.spgemm(a, b)[0])
    n0 = plan.launch_count()
    plan.execute()
    n1 = plan.launch_count()
    plan.execute()
    torch.cuda.synchronize()
    # every replay launches the same captured kernels
    assert n1 > n0 and plan.launch_count() - n1 == n1 - n0
    plan.close()


def test_autotune_choice_persists_in_cache_file(tsg, tmp_path):
    # the layout autotune chooses is appended to the cache file; a later
    # process (here: the same one with its cache emptied) reads it back and
    # reuses it without timing any candidate
    shapes = gen.er_batch_shapes(8, seed=77, log2_lo=8, log2_hi=11)
    pairs = [(gen.er(n, n, min(d, n), 3000 + 2 * t), gen.er(n, n, min(d, n), 3001 + 2 * t))
             for t, (n, d) in enumerate(shapes)]
    As = [tsg.DeviceCSR.from_host(a) for a, _ in pairs]
    Bs = [tsg.DeviceCSR.from_host(b) for _, b in pairs]
    f = tmp_path / "tune.txt"

    def fields(t):
        nb = t.num_bins
        return nb, list(t.bin_upper)[:nb], list(t.bin_kernel)[:nb], t.warps_per_block, t.sym_warps_per_block

    tsg.tune_cache_clear()
    try:
        assert tsg.tune_cache_open(str(f)) == 0
        p1 = tsg.Plan(As, Bs)
        before = p1.launch_count()
        t1 = p1.autotune()
        tuned = p1.launch_count() - before
        lines = f.read_text().splitlines()
        assert len(lines) == 1 and lines[0].startswith("tsg-tune-1 ")
        p1.close()
        tsg.tune_cache_clear()
        assert tsg.tune_cache_open(str(f)) == 1
        p2 = tsg.Plan(As, Bs)
        before = p2.launch_count()
        t2 = p2.autotune()
        hit = p2.launch_count() - before
        assert fields(t2) == fields(t1)
        assert 0 < hit and 4 * hit < tuned
        assert len(f.read_text().splitlines()) == 1  # a hit appends nothing
        Cs = p2.execute()
        torch.cuda.synchronize()
        for (a, b), C in zip(pairs, Cs):
            same(C, oracle.spgemm(a, b)[0])
        p2.close()
    finally:
        tsg.tune_cache_clear()
