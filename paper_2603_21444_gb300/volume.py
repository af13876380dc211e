"""Communication volumes of the trident algorithm (Prop. 1, Alg. 1, Alg. 2).

Host-side model of what every process of the q x q x lambda grid would move
when the grid runs on P = q^2 lambda GPUs, computed from the nonzero count of
every process's part of A and of B (``trident_loads``, counted on the
device).  Nothing here moves data: on one GPU every tile is already in HBM.

Per process (i, j, k) and round r = 0 .. q-1 of Alg. 1, with the inner tile
r' = (r + i + j) mod q (Eq. 2):

* global interconnect: the slice A_{i r' k} from process (i, r', k) and the
  slice B_{r' j k} from process (r', j, k) -- each skipped when it lives on
  the same node already (r' = j for A, r' = i for B; the paper's "skip
  intranode" reads as this local copy);
* local interconnect: the allgather of Alg. 2 brings the other lambda - 1
  slices B_{r' j h}, h != k.

Prop. 1 gives the same quantities for a uniform matrix with nnz / P
nonzeros per slice: 2 nnz / P over the global and (lambda - 1) nnz / P over
the local interconnect per process and round; over the q rounds the global
volume per process is 2 nnz q / P = 2 nnz / (sqrt(P) sqrt(lambda)).
"""
from __future__ import annotations

import math


def trident_volumes(a_loads, b_loads, q: int, lam: int, skip_local: bool = True):
    """Per-process volumes (in nonzeros) over all q rounds.

    a_loads[i * lam + k][r]: nnz of A_{i r k} (slice k of coarse tile (i, r));
    b_loads[r * lam + k][j]: nnz of B_{r j k}.  Returns a dict with
    ``gi`` and ``li``, each a q x q x lam nested list, and ``rounds``: for
    every process the list of (r', gi, li) per round."""
    if len(a_loads) != q * lam or len(b_loads) != q * lam:
        raise ValueError("loads must have q * lam rows")
    gi = [[[0] * lam for _ in range(q)] for _ in range(q)]
    li = [[[0] * lam for _ in range(q)] for _ in range(q)]
    rounds = [[[[] for _ in range(lam)] for _ in range(q)] for _ in range(q)]
    for i in range(q):
        for j in range(q):
            for k in range(lam):
                for r in range(q):
                    rp = (r + i + j) % q
                    g = 0
                    if not (skip_local and rp == j):
                        g += a_loads[i * lam + k][rp]
                    if not (skip_local and rp == i):
                        g += b_loads[rp * lam + k][j]
                    loc = sum(b_loads[rp * lam + h][j] for h in range(lam) if h != k)
                    gi[i][j][k] += g
                    li[i][j][k] += loc
                    rounds[i][j][k].append((rp, g, loc))
    return {"gi": gi, "li": li, "rounds": rounds}


def prop1_volumes(nnz: float, P: int, lam: int):
    """Prop. 1 for a uniform matrix (nnz per operand): per process and
    round, global 2 nnz / P and local (lam - 1) nnz / P; over the
    sqrt(P / lam) rounds, global 2 nnz / (sqrt(P) sqrt(lam))."""
    q = math.isqrt(P // lam)
    if q * q * lam != P:
        raise ValueError("P must be q^2 lambda")
    per_round_gi = 2.0 * nnz / P
    per_round_li = (lam - 1) * nnz / P
    return {"q": q, "per_round_gi": per_round_gi, "per_round_li": per_round_li,
            "total_gi": per_round_gi * q, "total_li": per_round_li * q,
            "total_gi_closed_form": 2.0 * nnz / (math.sqrt(P) * math.sqrt(lam))}


def summarize(vol, q: int, lam: int):
    """Max, mean and max / mean of the per-process global and local volumes."""
    out = {}
    for key in ("gi", "li"):
        flat = [vol[key][i][j][k] for i in range(q) for j in range(q) for k in range(lam)]
        mean = sum(flat) / len(flat)
        out[key] = {"max": max(flat), "mean": mean, "imbalance": (max(flat) / mean) if mean else 0.0}
    return out
