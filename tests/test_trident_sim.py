"""Host simulation of Alg. 1's message flow: q^2 lambda gloo ranks on the CPU
exchange their slices round by round; every rank's merged block must equal
the oracle's trident block bit for bit, its rounds must follow Eq. 2, and
the nonzeros it received must equal the Alg. 1 round walk of the volume
model, which Prop. 1's closed form pins on uniform inputs."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs(case):
    import gen
    m, kk, n, d, seed = case
    A = gen.er_variable(m, kk, d, seed, np.float64, "uniform", p_empty=0.1)
    B = gen.er_variable(kk, n, d, seed + 1, np.float64, "uniform", p_empty=0.1)
    return A, B


def _own_parts(A, B, q, lam, i, j, k):
    import oracle
    a_fine = oracle.trident_bounds(A.nrows, q, lam)[1]
    a_cols = oracle.trident_bounds(A.ncols, q, 1)[0]
    b_fine = oracle.trident_bounds(B.nrows, q, lam)[1]
    b_cols = oracle.trident_bounds(B.ncols, q, 1)[0]
    s = i * lam + k
    A_own = oracle.submatrix(A, a_fine[s], a_fine[s + 1], a_cols[j], a_cols[j + 1])
    B_own = oracle.submatrix(B, b_fine[s], b_fine[s + 1], b_cols[j], b_cols[j + 1])
    return A_own, B_own


def _worker(rank, world, port, q, lam, case, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime

    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=90))
    try:
        import gen
        import oracle
        from paper_2603_21444_gb300 import trident_sim
        oracle.set_threads(1)
        A, B = _inputs(case)
        i, j, k = trident_sim.coords(rank, q, lam)
        A_own, B_own = _own_parts(A, B, q, lam, i, j, k)
        C, stats = trident_sim.run_alg1(
            A_own, B_own, q, lam,
            local_product=lambda X, Y: oracle.spgemm(X, Y, with_scale=False)[0],
            local_sum=oracle.csr_sum, make=gen.CSR)
        out.put((rank, (C.nrows, C.ncols, C.rowptr, C.col, C.val), stats))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run_grid(q, lam, case):
    import multiprocessing as mp
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    world = q * q * lam
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, lam, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict()
    try:
        for _ in procs:
            rank, C, stats = out.get(timeout=150)
            got[rank] = (C, stats)
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    finally:
        # a rank that failed leaves the others waiting in a collective: end them
        for p in procs:
            if p.is_alive():
                p.kill()
                p.join(timeout=10)
    return got


@pytest.mark.timeout(240)
@pytest.mark.parametrize("q,lam,case", [
    (1, 2, (90, 70, 80, 9, 11)),      # two ranks: only the local allgather
    (2, 1, (101, 77, 93, 8, 21)),     # ragged tiles, point to point only
    (2, 2, (130, 96, 110, 10, 31)),   # eight ranks: both interconnects
    (3, 1, (150, 121, 133, 9, 41)),   # nine ranks: sends and receives go round 3-cycles
])
def test_alg1_message_flow_matches_oracle_and_volume_model(q, lam, case):
    import oracle
    from paper_2603_21444_gb300 import trident_sim, volume
    got = _run_grid(q, lam, case)
    A, B = _inputs(case)
    C_ref, _ = oracle.trident_product(A, B, q, lam)
    vol = volume.trident_volumes(oracle.trident_loads(A, q, lam).tolist(),
                                 oracle.trident_loads(B, q, lam).tolist(), q, lam)
    for rank, ((m, ncols, rp, col, val), stats) in got.items():
        i, j, k = trident_sim.coords(rank, q, lam)
        ref = C_ref[i][j][k]
        assert (m, ncols) == (ref.nrows, ref.ncols)
        assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col)
        assert np.array_equal(val, ref.val), "merged block not bit-identical to the oracle's"
        assert [r for r, _, _ in stats["rounds"]] == oracle.static_cannon_schedule(q, i, j)
        assert stats["rounds"] == [tuple(x) for x in vol["rounds"][i][j][k]]
        assert stats["gi"] == vol["gi"][i][j][k] and stats["li"] == vol["li"][i][j][k]


def test_rank_coordinates_round_trip():
    from paper_2603_21444_gb300 import trident_sim
    for q, lam in [(1, 1), (2, 3), (4, 4)]:
        seen = set()
        for r in range(q * q * lam):
            i, j, k = trident_sim.coords(r, q, lam)
            assert 0 <= i < q and 0 <= j < q and 0 <= k < lam
            assert trident_sim.rank_of(i, j, k, q, lam) == r
            seen.add((i, j, k))
        assert len(seen) == q * q * lam
