"""Coefficients sharded by lattice rows across ranks (the W table and the pair
sum split by rows of kappa).

The paper names distributed storage of the bispectrum values as the way past
one node's memory (Sec. 4.3, the complexity and memory paragraph).  Here a
rank holds the W table and runs the pair sum for a contiguous range of lattice
rows kk only (a plan created with ``rows=(lo, hi)``, srm3_grid.row_begin /
row_end); one all-gather of the coefficient rows then gives every rank the
whole C, from which the transform (srm3_field_from_coeffs) makes the fields.
The gather is the only exchange step of the path.

Balance: row kk carries sum_kw |Pi(kk, kw)| sum pairs (about (kk + 1) nw^2 / 4)
and, with mixed interactions, (kk + 1) (nw - 1)(nw - 2) / 2 difference pairs,
so equal row counts would load the high rows' ranks about twice the average;
the ranges are cut at equal shares of the cumulative pair count instead.
"""
from __future__ import annotations

import numpy as np


def row_pairs(nk: int, nw: int, mixed: bool = False) -> np.ndarray:
    """Pairs of each lattice row (one sheet): sum over kw of
    ceil(((kk + 1)(kw + 1) - 2) / 2) (no pair at k = 0), plus the difference
    pairs (kk + 1)(nw - 1 - kw), kw >= 1, when ``mixed``."""
    kk = np.arange(nk, dtype=np.int64)[:, None]
    kw = np.arange(nw, dtype=np.int64)[None, :]
    cnt = ((kk + 1) * (kw + 1) - 1) // 2
    cnt[0, 0] = 0
    out = cnt.sum(axis=1)
    if mixed and nw > 1:
        out = out + (kk[:, 0] + 1) * ((nw - 1) * (nw - 2) // 2)
    return out


def row_partition(nk: int, nw: int, world: int, mixed: bool = False):
    """Contiguous row ranges [lo, hi) for ranks 0..world-1, disjoint and
    covering 0..nk-1, cut where the cumulative pair count crosses r/world of
    the total (every range non-empty while nk >= world)."""
    if world < 1 or nk < world:
        raise ValueError("need 1 <= world <= n_kappa")
    cum = np.cumsum(row_pairs(nk, nw, mixed))
    total = int(cum[-1])
    cuts = [0]
    for r in range(1, world):
        c = int(np.searchsorted(cum, total * r / world, side="left")) + 1
        c = max(c, cuts[-1] + 1)            # non-empty
        c = min(c, nk - (world - r))        # leave a row for every later rank
        cuts.append(c)
    cuts.append(nk)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def gather_rows(C, ranges, rank, dist, group=None):
    """All-gather of coefficient rows.  ``C`` is a tensor [n][2][nk][nw](...)
    whose rows ranges[rank] this rank has computed; returns a tensor of the
    same shape with every rank's rows in place.  One all_gather of equal-size
    slabs (each range padded to the longest) on ``dist`` (torch.distributed:
    NCCL for device tensors, gloo for host tensors)."""
    import torch
    lo, hi = ranges[rank]
    rmax = max(h - l for l, h in ranges)
    slab = torch.zeros((C.shape[0], C.shape[1], rmax) + tuple(C.shape[3:]), dtype=C.dtype,
                       device=C.device)
    slab[:, :, :hi - lo] = C[:, :, lo:hi]
    parts = [torch.empty_like(slab) for _ in ranges]
    dist.all_gather(parts, slab, group=group)
    out = torch.empty_like(C)
    for (l, h), part in zip(ranges, parts):
        out[:, :, l:h] = part[:, :, :h - l]
    return out
