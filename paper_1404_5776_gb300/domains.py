"""Domain decomposition of one system over several ranks (host side).

The truncated products of the step, C = cut_{P_C}(A B), are row-local: output
block row i needs block row i of A and the block rows k of B with (i,k) in P_A
(Sec. II.A cut-off; the atoms do not move, so every pattern and every exchange
list is fixed once, Sec. V.A).  A rank that owns a set of output rows therefore
needs, besides its own rows of B, a halo: the rows of B that belong to other
ranks and lie within r_A of its atoms.

This module plans that decomposition and moves the halo rows:

* the atoms are ordered along a Morton (Z-order) curve of their positions, so
  a contiguous range of that order is a compact spatial domain and its halo
  is a thin shell;
* each rank owns one contiguous range, balanced by a per-row weight (blocks or
  block triples per row);
* for a block-row pattern P_A, each rank lists the rows of B it needs from
  every other rank; exchange_rows() sends and receives those rows (block
  values, row by row) with point-to-point torch.distributed calls;
* the observables are sums over rows: each rank adds its own rows' partial
  traces and an all-reduce of the 8 doubles completes them.

In the permuted (Morton) numbering the owned rows of a rank are one range
[r0, r1), which is what a row-range product needs.  Nothing here runs on a
GPU; a multi-GPU run would call the same plan with NCCL in place of gloo and
copy the received rows into the local device buffers before each product.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Sequence, Tuple

import numpy as np


def _spread_bits(v: np.ndarray) -> np.ndarray:
    """Interleave the low 21 bits of v with two zero bits between them."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(pos: np.ndarray, cell=None, bits: int = 10) -> np.ndarray:
    """Permutation of the atoms along a Morton curve: order[new] = old index.

    Positions are quantised to 2^bits cells per axis over the periodic cell
    (or the bounding box of an open system); ties keep the input order."""
    pos = np.asarray(pos, dtype=np.float64)
    if cell is not None:
        lo = np.zeros(3)
        ext = np.asarray(cell, dtype=np.float64)
    else:
        lo = pos.min(0)
        ext = np.maximum(pos.max(0) - lo, 1e-12)
    q = np.clip(((pos - lo) / ext * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1)
    code = _spread_bits(q[:, 0]) | (_spread_bits(q[:, 1]) << np.uint64(1)) | (_spread_bits(q[:, 2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def permute_pattern(rowptr: np.ndarray, col: np.ndarray, order: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Block-CSR pattern in the new numbering (new atom a = old atom order[a]).

    Returns (rowptr, col, src): src[q_new] is the old block index of new block
    q_new, so values move as val_new[q_new] = val_old[src[q_new]]."""
    n = len(order)
    inv = np.empty(n, dtype=np.int64)
    inv[order] = np.arange(n)
    rows_new, cols_new, src = [], [], []
    for a in range(n):
        i = order[a]
        q0, q1 = rowptr[i], rowptr[i + 1]
        c = inv[col[q0:q1]]
        srt = np.argsort(c, kind="stable")
        cols_new.append(c[srt])
        src.append(np.arange(q0, q1)[srt])
        rows_new.append(q1 - q0)
    rp = np.concatenate([[0], np.cumsum(rows_new)]).astype(np.int32)
    return rp, np.concatenate(cols_new).astype(np.int32), np.concatenate(src).astype(np.int64)


def balanced_ranges(weights: Sequence[float], n_ranks: int) -> List[Tuple[int, int]]:
    """Contiguous row ranges [r0, r1), one per rank, with nearly equal total weight
    (every range non-empty when there are at least as many rows as ranks)."""
    w = np.asarray(weights, dtype=np.float64)
    n = len(w)
    if n_ranks < 1 or n < n_ranks:
        raise ValueError("need at least one row per rank")
    cum = np.concatenate([[0.0], np.cumsum(w)])
    cuts = [0]
    for p in range(1, n_ranks):
        c = int(np.searchsorted(cum, cum[-1] * p / n_ranks))
        c = min(max(c, cuts[-1] + 1), n - (n_ranks - p))
        cuts.append(c)
    cuts.append(n)
    return [(cuts[p], cuts[p + 1]) for p in range(n_ranks)]


def owner_of_rows(ranges: Sequence[Tuple[int, int]], n: int) -> np.ndarray:
    own = np.empty(n, dtype=np.int32)
    for p, (r0, r1) in enumerate(ranges):
        own[r0:r1] = p
    return own


@dataclass
class HaloPlan:
    """need[(p, q)]: rows owned by rank q that rank p needs (ascending)."""
    ranges: List[Tuple[int, int]]
    need: Dict[Tuple[int, int], np.ndarray]

    def halo(self, p: int) -> np.ndarray:
        """Every row rank p receives, ascending."""
        parts = [v for (a, _), v in self.need.items() if a == p]
        return np.sort(np.concatenate(parts)) if parts else np.zeros(0, dtype=np.int64)


def plan_halo(rowptr_a: np.ndarray, col_a: np.ndarray, ranges: Sequence[Tuple[int, int]]) -> HaloPlan:
    """Halo of the B operand of C = cut(A B) for row-owned C: rank p needs row k
    of B for every (i, k) in P_A with i owned by p and k owned elsewhere."""
    n = len(rowptr_a) - 1
    own = owner_of_rows(ranges, n)
    need = {}
    for p, (r0, r1) in enumerate(ranges):
        ks = np.unique(col_a[rowptr_a[r0]:rowptr_a[r1]].astype(np.int64))
        for q in range(len(ranges)):
            if q == p:
                continue
            sel = ks[own[ks] == q]
            if len(sel):
                need[(p, q)] = sel
    return HaloPlan(list(ranges), need)


def row_slices(rowptr: np.ndarray, voff: np.ndarray, rows: np.ndarray) -> List[slice]:
    """Value slices of whole block rows (blocks of a row are contiguous in block-CSR)."""
    return [slice(int(voff[rowptr[k]]), int(voff[rowptr[k + 1]])) for k in rows]


def exchange_rows(dist, plan: HaloPlan, rank: int, rowptr: np.ndarray, voff: np.ndarray, val: np.ndarray) -> None:
    """Fills, in val (the rank's copy of a block-CSR matrix, complex128), every
    halo row the plan lists for this rank, from the ranks that own them, and
    sends this rank's rows to the ranks that need them.  Point-to-point
    messages, one per (sender, receiver) pair, in a fixed order (lower rank
    pair first) so that every send meets its receive."""
    import torch
    n_ranks = len(plan.ranges)
    for a in range(n_ranks):
        for b in range(a + 1, n_ranks):
            if rank not in (a, b):
                continue
            other = b if rank == a else a
            # a sends first, then b (blocking send/recv in a fixed order)
            for sender, receiver in ((a, b), (b, a)):
                rows = plan.need.get((receiver, sender))
                if rows is None:
                    continue
                sl = row_slices(rowptr, voff, rows)
                if rank == sender:
                    buf = np.concatenate([val[s] for s in sl]) if sl else np.zeros(0, np.complex128)
                    dist.send(torch.from_numpy(np.ascontiguousarray(buf).view(np.float64)), dst=other)
                else:
                    total = sum(s.stop - s.start for s in sl)
                    t = torch.empty(2 * total, dtype=torch.float64)
                    dist.recv(t, src=other)
                    got = t.numpy().view(np.complex128)
                    o = 0
                    for s in sl:
                        m = s.stop - s.start
                        val[s] = got[o:o + m]
                        o += m


def allreduce_traces(dist, partial: np.ndarray) -> np.ndarray:
    """Sum of the ranks' partial traces (8 doubles: Re/Im of Tr(KS), Tr(KD_xyz))."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(partial, dtype=np.float64).copy())
    dist.all_reduce(t)
    return t.numpy()
