"""Host simulation of the trident message flow (Alg. 1 with Alg. 2 as its
partial product) over torch.distributed ranks on the CPU (gloo).

This is not a GPU path: on one GPU every tile is already in HBM and the
batched plan runs all of Alg. 1's instances at once.  The simulation checks
the ORDER of the distributed algorithm -- which process fetches which slice
in which round, and what the allgather assembles -- with real messages, and
counts what each process receives, for any grid (P = q^2 lambda processes).

Process (i, j, k) (rank (i q + j) lambda + k) owns, before round 0:
  A_{ijk}: row slice k of A's coarse tile (i, j), block-local columns;
  B_{ijk}: row slice k of B's coarse tile (i, j), block-local columns.
Round r = 0 .. q-1 uses the inner tile r' = (r + i + j) mod q (Eq. 2):
  * global interconnect: A_{i r' k} arrives from process (i, r', k) and
    B_{r' j k} from process (r', j, k) (point to point), unless r' names the
    process itself (r' = j for A, r' = i for B: a local copy);
  * local interconnect: the lambda processes (i, j, *) allgather their
    slices B_{r' j h}, which stacked by rows form the whole tile B_{r' j}
    (Alg. 2);
  * the partial C_{ijk}^{(r)} = A_{i r' k} B_{r' j} is formed by the caller's
    local product.
After the last round C_{ijk} is the caller's ordered sum of the q partials
(round order).  Volumes are counted in nonzeros, as in Prop. 1.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch
import torch.distributed as dist


@dataclass
class Block:
    """Host CSR block (int64 row pointers, int32 columns, float values)."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def rank_of(i: int, j: int, k: int, q: int, lam: int) -> int:
    return (i * q + j) * lam + k


def coords(rank: int, q: int, lam: int):
    """(i, j, k) of a rank."""
    k = rank % lam
    ij = rank // lam
    return ij // q, ij % q, k


def _pack(X):
    meta = torch.tensor([X.nrows, X.ncols, int(X.rowptr[-1])], dtype=torch.int64)
    idx = torch.from_numpy(np.concatenate([np.asarray(X.rowptr, dtype=np.int64),
                                           np.asarray(X.col, dtype=np.int64)]))
    val = torch.from_numpy(np.ascontiguousarray(X.val, dtype=np.float64))
    return meta, idx, val


def _unpack(meta, idx, val, make):
    m, ncols, nnz = (int(x) for x in meta.tolist())
    rp = idx[: m + 1].numpy().astype(np.int64)
    col = idx[m + 1: m + 1 + nnz].numpy().astype(np.int32)
    return make(m, ncols, rp, col, val[:nnz].numpy().copy())


def _stack_rows(blocks, make):
    """Row concatenation of blocks of equal width (the slices of one tile)."""
    ncols = blocks[0].ncols
    rps, cols, vals, base = [np.zeros(1, dtype=np.int64)], [], [], 0
    for X in blocks:
        rp = np.asarray(X.rowptr, dtype=np.int64)
        rps.append(rp[1:] + base)
        base += int(rp[-1])
        cols.append(np.asarray(X.col, dtype=np.int32))
        vals.append(np.asarray(X.val))
    return make(sum(X.nrows for X in blocks), ncols, np.concatenate(rps), np.concatenate(cols),
                np.concatenate(vals))


def _exchange(mine, dst: int, src: int, tag: int, make):
    """Send `mine` to rank dst and receive a block from rank src."""
    meta, idx, val = _pack(mine)
    reqs = [dist.isend(meta, dst, tag=tag), dist.isend(idx, dst, tag=tag + 1), dist.isend(val, dst, tag=tag + 2)]
    rmeta = torch.empty(3, dtype=torch.int64)
    dist.recv(rmeta, src, tag=tag)
    m, _, nnz = (int(x) for x in rmeta.tolist())
    ridx = torch.empty(m + 1 + nnz, dtype=torch.int64)
    rval = torch.empty(nnz, dtype=torch.float64)
    dist.recv(ridx, src, tag=tag + 1)
    dist.recv(rval, src, tag=tag + 2)
    for r in reqs:
        r.wait()
    return _unpack(rmeta, ridx, rval, make)


def _allgather(mine, group, lam: int, make):
    """Blocks of the lambda ranks of a group, in slice order."""
    meta, idx, val = _pack(mine)
    metas = [torch.empty(3, dtype=torch.int64) for _ in range(lam)]
    dist.all_gather(metas, meta, group=group)
    li = max(int(m[0]) + 1 + int(m[2]) for m in metas)
    lv = max(int(m[2]) for m in metas)
    pidx = torch.zeros(li, dtype=torch.int64)
    pidx[: idx.numel()] = idx
    pval = torch.zeros(lv, dtype=torch.float64)
    pval[: val.numel()] = val
    idxs = [torch.empty(li, dtype=torch.int64) for _ in range(lam)]
    vals = [torch.empty(lv, dtype=torch.float64) for _ in range(lam)]
    dist.all_gather(idxs, pidx, group=group)
    dist.all_gather(vals, pval, group=group)
    return [_unpack(metas[h], idxs[h], vals[h], make) for h in range(lam)]


def slice_groups(q: int, lam: int):
    """One process group per output tile (i, j): its lambda slice ranks.
    Every rank must create all of them, in this order."""
    return [[dist.new_group([rank_of(i, j, k, q, lam) for k in range(lam)]) for j in range(q)] for i in range(q)]


def run_alg1(A_own, B_own, q: int, lam: int, local_product, local_sum, groups=None, make=Block):
    """Alg. 1 on this rank of a P = q^2 lambda gloo world.

    A_own, B_own: this process's A_{ijk} and B_{ijk} (objects with nrows,
    ncols, rowptr, col, val).  local_product(A_blk, B_blk) -> partial block;
    local_sum(list of partials in round order) -> C_{ijk}.  groups: the
    result of slice_groups (created here when None).  make(nrows, ncols,
    rowptr, col, val) builds received blocks.

    Returns (C_ijk, stats): stats["rounds"] lists (r', gi, li) per round,
    stats["gi"] / stats["li"] the nonzeros received over the global and the
    local interconnect."""
    world = dist.get_world_size()
    if world != q * q * lam:
        raise ValueError(f"world size {world} != q^2 lambda = {q * q * lam}")
    if groups is None:
        groups = slice_groups(q, lam)
    i, j, k = coords(dist.get_rank(), q, lam)
    parts, rounds = [], []
    for r in range(q):
        rp = (r + i + j) % q
        gi = 0
        # A_{i r' k}: from (i, r', k); mine goes to the process whose r' is j
        if rp == j:
            a_blk = A_own
        else:
            a_dst = rank_of(i, (j - r - i) % q, k, q, lam)
            a_blk = _exchange(A_own, a_dst, rank_of(i, rp, k, q, lam), 8 * r, make)
            gi += a_blk.nnz
        # B_{r' j k}: from (r', j, k); mine goes to the process whose r' is i
        if rp == i:
            b_slice = B_own
        else:
            b_dst = rank_of((i - r - j) % q, j, k, q, lam)
            b_slice = _exchange(B_own, b_dst, rank_of(rp, j, k, q, lam), 8 * r + 4, make)
            gi += b_slice.nnz
        # Alg. 2: the lambda slices of B_{r' j}, stacked by rows
        slices = _allgather(b_slice, groups[i][j], lam, make) if lam > 1 else [b_slice]
        li = sum(slices[h].nnz for h in range(lam) if h != k)
        parts.append(local_product(a_blk, _stack_rows(slices, make)))
        rounds.append((rp, gi, li))
    C = local_sum(parts)
    return C, {"rounds": rounds, "gi": sum(g for _, g, _ in rounds), "li": sum(x for _, _, x in rounds)}
