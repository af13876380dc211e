"""Full-size parity of the batched workloads, in the launch configuration the
benchmark times (a plan sized once, replayed from its CUDA graph):

* the trident grid 4 x 4 x lambda=4 over ER A, B with n = 2^21 and 32 per
  row (Sec. 3.2 partition, Alg. 1 rounds in Eq. 2 order, fused ordered sum):
  blocks (0,0,0) and (3,3,3) whole, 4096 seeded rows of every other block,
  each against the oracle run on that block only (its four rounds, summed in
  round order), plus the total nnz against the ER collision estimate.  The
  total product count is exactly 2^31, so any 32-bit total or offset that
  overflows shows here and nowhere smaller;
* the 256 independent ER products (n log-uniform in [2^10, 2^16], 4..64 per
  row): 512 seeded rows of every product against the oracle.

Patterns and values are compared bit for bit (every row here sits on an
on-chip variant, which adds in the oracle's order)."""
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


def take_rows(X, rows):
    """The CSR of X's rows `rows` (sorted), columns unchanged."""
    lens = X.rowptr[rows + 1] - X.rowptr[rows]
    rp = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.repeat(X.rowptr[rows] - rp[:-1], lens) + np.arange(rp[-1])
    return gen.CSR(len(rows), X.ncols, rp, X.col[idx], X.val[idx])


def device_rows(C, rows):
    """(row_ptr, col, val) of rows `rows` of a device CSR, gathered on the device."""
    rp = C.row_ptr.cpu().numpy().astype(np.int64)
    assert rp[0] == 0 and rp[-1] == C.nnz and np.all(np.diff(rp) >= 0)
    lens = rp[rows + 1] - rp[rows]
    out = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=out[1:])
    idx = torch.from_numpy(np.repeat(rp[rows] - out[:-1], lens) + np.arange(out[-1])).to(C.col.device)
    return out, C.col[idx].cpu().numpy(), C.val[idx].cpu().numpy()


def same(got, ref):
    rp, col, val = got
    assert np.array_equal(rp, ref.rowptr), "row_ptr"
    assert np.array_equal(col, ref.col), "col"
    assert np.array_equal(val, ref.val), "values"


def test_trident_grid_full_size(tsg):
    n, d, q, lam = 1 << 21, 32, 4, 4
    A = gen.er(n, n, d, 4)
    B = gen.er(n, n, d, 5)
    h = tsg.Handle()
    plan = tsg.TridentPlan(tsg.DeviceCSR.from_host(A), tsg.DeviceCSR.from_host(B), q, lam, h)
    fp = plan.fused_plan()
    fp.execute(True)
    blocks = fp.execute(True)  # replayed from the graph
    torch.cuda.synchronize()
    assert h.device_status() == 0
    # every row has 32 x 32 products from 32 distinct B rows, which never
    # collide with themselves: E[collisions] = (1024^2 - 32 * 32^2) / 2 / n
    # per row, Poisson; the total must sit within 5 sigma of the estimate
    total = sum(fp.nnz)
    mean_coll = n * (1024 ** 2 - 32 * 32 ** 2) / 2 / n
    assert abs((n * 1024 - total) - mean_coll) <= 5 * np.sqrt(mean_coll), total
    coarse, fine = oracle.trident_bounds(n, q, lam)
    b_tiles = {}

    def b_tile(r, j):
        if (r, j) not in b_tiles:
            b_tiles[(r, j)] = oracle.submatrix(B, coarse[r], coarse[r + 1], coarse[j], coarse[j + 1])
        return b_tiles[(r, j)]

    def oracle_block(i, j, k, rows=None):
        r0, r1 = fine[i * lam + k], fine[i * lam + k + 1]
        parts = []
        for r in oracle.static_cannon_schedule(q, i, j):
            As = oracle.submatrix(A, r0, r1, coarse[r], coarse[r + 1])
            if rows is not None:
                As = take_rows(As, rows)
            parts.append(oracle.spgemm(As, b_tile(r, j), with_scale=False)[0])
        return oracle.csr_sum(parts)

    rng = np.random.default_rng(2024)
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                C = blocks[plan.block_index(i, j, k)]
                if (i, j, k) in ((0, 0, 0), (3, 3, 3)):
                    same(C.to_host(), oracle_block(i, j, k))
                else:
                    rows = np.sort(rng.choice(C.nrows, 4096, replace=False))
                    same(device_rows(C, rows), oracle_block(i, j, k, rows))
    h.close()


def test_many_products_full_size(tsg):
    pairs = gen.er_batch(256)
    As = [tsg.DeviceCSR.from_host(a) for a, _ in pairs]
    Bs = [tsg.DeviceCSR.from_host(b) for _, b in pairs]
    plan = tsg.Plan(As, Bs)
    plan.execute(True)
    Cs = plan.execute(True)  # replayed from the graph
    torch.cuda.synchronize()
    rng = np.random.default_rng(77)
    for (a, b), C in zip(pairs, Cs):
        rows = np.sort(rng.choice(a.nrows, min(512, a.nrows), replace=False))
        same(device_rows(C, rows), oracle.spgemm(take_rows(a, rows), b, with_scale=False)[0])
    plan.close()
