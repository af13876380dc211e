"""GPU parity of the backward pass (chain rule on Sec. 2's definition) and of
the CSR transpose, plus central finite differences through the autograd
Function."""
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


def _grads(tsg, handle, A, B, W, deterministic):
    from paper_2603_21444_gb300 import autograd as ag
    dA = tsg.DeviceCSR.from_host(A)
    dB = tsg.DeviceCSR.from_host(B)
    C = tsg.spgemm(dA, dB, handle)
    g = torch.from_numpy(W).to("cuda")
    ga, gb = ag.backward(dA, dB, C, g, deterministic=deterministic, handle=handle)
    torch.cuda.synchronize()
    return C, ga.cpu().numpy(), gb.cpu().numpy()


@pytest.mark.parametrize("values", ["normal", "int"])
def test_backward_matches_oracle(tsg, handle, values):
    A = gen.er_variable(700, 500, 20, 3, np.float64, values, p_empty=0.1)
    B = gen.er_variable(500, 600, 20, 4, np.float64, values, p_empty=0.1)
    Cref, _ = oracle.spgemm(A, B)
    W = np.random.default_rng(5).standard_normal(Cref.nnz) if values == "normal" else \
        np.random.default_rng(5).integers(-3, 4, Cref.nnz).astype(np.float64)
    ra, rb = oracle.backward(A, B, Cref, W)
    _, ga, gb = _grads(tsg, handle, A, B, W, deterministic=True)
    assert np.array_equal(ga, ra)       # same order of the same rounded products
    assert np.array_equal(gb, rb)       # deterministic path: i ascending, like the oracle
    _, ga2, gb2 = _grads(tsg, handle, A, B, W, deterministic=False)
    assert np.array_equal(ga2, ra)
    # atomic scatter: the scale of each entry bounds the reordering error
    At = oracle.transpose(A)
    scale = np.zeros(B.nnz)
    Bd_rows = np.repeat(np.arange(B.nrows), B.row_lengths())
    Wd = np.zeros((Cref.nrows, Cref.ncols))
    Wd[np.repeat(np.arange(Cref.nrows), Cref.row_lengths()), Cref.col] = np.abs(W)
    S = (np.abs(A.to_dense()).T @ Wd)[Bd_rows, B.col]
    assert np.all(np.abs(gb2 - rb) <= 1e-12 * S + 1e-300)
    del At, scale


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_transpose_matches_oracle(tsg, handle, dtype):
    from paper_2603_21444_gb300 import autograd as ag
    X = gen.er_variable(3000, 2000, 30, 9, dtype, "normal", p_empty=0.1)
    T = ag.transpose(tsg.DeviceCSR.from_host(X), handle)
    torch.cuda.synchronize()
    ref = oracle.transpose(X)
    rp, col, val = T.to_host()
    assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col) and np.array_equal(val, ref.val)


def long_column_matrix(nrows, ncols, lens, seed, dtype):
    """X with 2 random entries per row in columns >= 100 plus columns
    j < 100 holding exactly lens[j] entries at distinct random rows: rows of
    X^T far longer than one warp's share."""
    rng = np.random.default_rng(seed)
    r = [np.repeat(np.arange(nrows), 2)]
    c = [rng.integers(100, ncols, 2 * nrows)]
    for j, L in lens.items():
        r.append(rng.choice(nrows, size=L, replace=False))
        c.append(np.full(L, j))
    rows, cols = np.concatenate(r), np.concatenate(c)
    key = np.unique(rows.astype(np.int64) * ncols + cols)
    return gen.from_coo(nrows, ncols, key // ncols, key % ncols, rng.normal(size=key.size).astype(dtype))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_transpose_long_columns(tsg, handle, dtype):
    # columns of 1024 (the warp path's limit), 1025, 20000 and 300000
    # entries; 700000 rows of X: two bitmap windows of row indices
    from paper_2603_21444_gb300 import autograd as ag
    X = long_column_matrix(700000, 5000, {3: 20000, 7: 1025, 11: 1024, 40: 300000}, 5, dtype)
    T = ag.transpose(tsg.DeviceCSR.from_host(X), handle)
    torch.cuda.synchronize()
    ref = oracle.transpose(X)
    rp, col, val = T.to_host()
    assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col) and np.array_equal(val, ref.val)


def test_autograd_gradcheck_tiny(tsg, handle):
    from paper_2603_21444_gb300 import autograd as ag
    A = gen.er_variable(12, 9, 4, 1, np.float64, "normal")
    B = gen.er_variable(9, 11, 4, 2, np.float64, "normal")
    pat = ag.Pattern(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), handle)
    a = torch.from_numpy(A.val.copy()).cuda().requires_grad_(True)
    b = torch.from_numpy(B.val.copy()).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x, y: ag.spgemm_values(x, y, pat), (a, b), eps=1e-6, atol=1e-8)


def _fd_check(tsg, handle, A, B, nsamp, seed):
    """Central differences of L = sum(C * W) with h = 2^-8 on sampled entries;
    only the rows of C an entry touches are summed (bilinear loss: no
    truncation error, no cancellation in a large sum)."""
    from paper_2603_21444_gb300 import autograd as ag
    dA = tsg.DeviceCSR.from_host(A)
    dB = tsg.DeviceCSR.from_host(B)
    pat = ag.Pattern(dA, dB, handle)
    a = dA.val.clone().requires_grad_(True)
    b = dB.val.clone().requires_grad_(True)
    c = ag.spgemm_values(a, b, pat)
    W = torch.from_numpy(np.random.default_rng(seed).standard_normal(c.numel())).cuda()
    (c * W).sum().backward()
    ga, gb = a.grad.cpu().numpy(), b.grad.cpu().numpy()
    crp = pat.C.row_ptr.cpu().numpy().astype(np.int64)
    Wh = W.cpu().numpy()
    At = oracle.transpose(gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, np.arange(A.nnz, dtype=np.float64)))
    rng = np.random.default_rng(seed + 1)
    h = 2.0 ** -8
    C = tsg.DeviceCSR(pat.C.nrows, pat.C.ncols, pat.C.row_ptr, pat.C.col, torch.empty_like(c))

    def local_loss(av, bv, rows):
        numeric = tsg.numeric_into(tsg.DeviceCSR(A.nrows, A.ncols, dA.row_ptr, dA.col, av),
                                   tsg.DeviceCSR(B.nrows, B.ncols, dB.row_ptr, dB.col, bv), C, handle)
        vals = numeric.val.cpu().numpy()
        tot = 0.0
        for i in rows:
            tot += float(np.dot(vals[crp[i]:crp[i + 1]], Wh[crp[i]:crp[i + 1]]))
        return tot

    worst = 0.0
    base_a, base_b = dA.val.clone(), dB.val.clone()
    for e in rng.choice(A.nnz, nsamp // 2, replace=False):
        i = int(np.searchsorted(A.rowptr, e, side="right") - 1)
        ap, am = base_a.clone(), base_a.clone()
        ap[e] += h
        am[e] -= h
        fd = (local_loss(ap, base_b, [i]) - local_loss(am, base_b, [i])) / (2 * h)
        worst = max(worst, abs(fd - ga[e]) / max(abs(fd), abs(ga[e]), 1e-300))
    for f in rng.choice(B.nnz, nsamp - nsamp // 2, replace=False):
        k = int(np.searchsorted(B.rowptr, f, side="right") - 1)
        rows = At.col[At.rowptr[k]:At.rowptr[k + 1]]
        bp, bm = base_b.clone(), base_b.clone()
        bp[f] += h
        bm[f] -= h
        fd = (local_loss(base_a, bp, rows) - local_loss(base_a, bm, rows)) / (2 * h)
        worst = max(worst, abs(fd - gb[f]) / max(abs(fd), abs(gb[f]), 1e-300))
    return worst


def test_finite_differences_small(tsg, handle):
    A = gen.er(2000, 2000, 16, 5, np.float64, "normal")
    B = gen.er(2000, 500, 16, 6, np.float64, "normal")
    assert _fd_check(tsg, handle, A, B, 100, 11) <= 1e-6


def test_finite_differences_full_size(tsg, handle):
    # A 2^18 x 2^18, B 2^18 x 2^16, 16 per row, float64; 1000 sampled entries
    A = gen.er(1 << 18, 1 << 18, 16, 5, np.float64, "normal")
    B = gen.er(1 << 18, 1 << 16, 16, 6, np.float64, "normal")
    assert _fd_check(tsg, handle, A, B, 1000, 12) <= 1e-6
