"""The communication-volume model (Prop. 1 and the Alg. 1 round order) on
the host: pinned by Prop. 1's closed form for uniform loads, by hand-counted
small grids and by the skip rule for tiles a node already holds."""
import math

import numpy as np
import pytest

import gen
import oracle
from paper_2603_21444_gb300 import volume


@pytest.mark.parametrize("q,lam", [(4, 4), (8, 4), (2, 1), (3, 2)])
def test_uniform_loads_match_prop1(q, lam):
    P = q * q * lam
    nnz = 7 * P  # every slice holds nnz / P = 7
    loads = [[nnz // P] * q for _ in range(q * lam)]
    model = volume.prop1_volumes(nnz, P, lam)
    assert model["q"] == q
    assert math.isclose(model["total_gi"], model["total_gi_closed_form"])
    v = volume.trident_volumes(loads, loads, q, lam, skip_local=False)
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                assert v["gi"][i][j][k] == model["total_gi"]
                assert v["li"][i][j][k] == model["total_li"]
                assert [rp for rp, _, _ in v["rounds"][i][j][k]] == [(r + i + j) % q for r in range(q)]
    # with local copies skipped each process fetches A once and B once less
    # over the q rounds (r' = j once, r' = i once)
    s = volume.trident_volumes(loads, loads, q, lam, skip_local=True)
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                assert s["gi"][i][j][k] == model["total_gi"] - 2 * (nnz // P)
    # the global volume is a factor sqrt(lam) below Sparse SUMMA's 2 nnz / sqrt(P)
    assert math.isclose(model["total_gi"] * math.sqrt(lam), 2 * nnz / math.sqrt(P))


def test_hand_counted_grid():
    # q = 2, lam = 1: process (0, 1) runs r' = 1 then 0; it holds A_01 and
    # B_01 (r' = 1 = j: A local; r' = 0 = i: B local)
    a = [[1, 2], [3, 4]]   # a[i][r] = nnz(A_ir)
    b = [[5, 6], [7, 8]]   # b[r][j] = nnz(B_rj)
    v = volume.trident_volumes(a, b, 2, 1)
    # round 0: r' = 1 -> A_01 local (skip), B_11 = 8 remote; round 1: r' = 0
    # -> A_00 = 1 remote, B_01 local (skip)
    assert v["rounds"][0][1][0] == [(1, 8, 0), (0, 1, 0)]
    assert v["gi"][0][1][0] == 9 and v["li"][0][1][0] == 0


def test_local_allgather_counts_other_slices():
    q, lam = 2, 3
    a = [[1] * q for _ in range(q * lam)]
    b = [[10 * (s + 1)] * q for s in range(q * lam)]  # slice s of B rows
    v = volume.trident_volumes(a, b, q, lam)
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                for rp, _, loc in v["rounds"][i][j][k]:
                    assert loc == sum(b[rp * lam + h][j] for h in range(lam) if h != k)


def test_er_volumes_near_prop1():
    # an ER matrix is close to uniform: counted global volumes (no skipping)
    # within a few percent of Prop. 1 for every process
    n, q, lam = 4096, 4, 4
    A = gen.er(n, n, 16, 3)
    L = oracle.trident_loads(A, q, lam).tolist()
    v = volume.trident_volumes(L, L, q, lam, skip_local=False)
    model = volume.prop1_volumes(A.nnz, q * q * lam, lam)
    g = np.array(v["gi"], dtype=float).reshape(-1)
    assert np.all(np.abs(g / model["total_gi"] - 1) < 0.05)
    s = volume.summarize(v, q, lam)
    assert s["gi"]["imbalance"] < 1.05
