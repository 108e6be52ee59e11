"""Splitting one listing into independent shards (replicas on several GPUs).

Seed vertices are independent (each iteration of the outer loop of
Algorithms 1 and 2 lists the triangles whose B vertex it is), so ranks can
list disjoint ranges of seed ranks with ``tl_list_triangles_range`` and no
exchange; only the per-rank (count, set hash) is combined at the end, by a sum
(mod 2^64 for the hash).  These helpers hold the host side of that: the work
of each seed vertex, contiguous ranges of near-equal work, and the combine.
"""
from __future__ import annotations

import numpy as np

TL_APP, TL_APM, TL_AMM = 0, 1, 2


def seed_work(out_off: np.ndarray, out_adj: np.ndarray, in_off: np.ndarray, in_adj: np.ndarray,
              alg: int) -> np.ndarray:
    """Membership tests of each seed rank x (Property 1, per vertex):
    A++ (x = w): sum of d+_u over u in N-_w; A+- (x = u): sum of d+_v over v
    in N+_u; A-- (x = v): sum of d-_w over w in N+_v.  Inputs are the
    rank-space CSR of N+ and N- (``tl_graph_csr``)."""
    dplus = np.diff(np.asarray(out_off, dtype=np.int64))
    dminus = np.diff(np.asarray(in_off, dtype=np.int64))
    off, adj = (in_off, in_adj) if alg == TL_APP else (out_off, out_adj)
    length = dminus if alg == TL_AMM else dplus
    off = np.asarray(off, dtype=np.int64)
    vals = length[np.asarray(adj, dtype=np.int64)]
    csum = np.zeros(len(vals) + 1, dtype=np.int64)
    np.cumsum(vals, out=csum[1:])
    return csum[off[1:]] - csum[off[:-1]]


def balanced_ranges(work: np.ndarray, parts: int) -> list[tuple[int, int]]:
    """Cut [0, n) into `parts` contiguous ranges whose work sums are as equal
    as a cut at vertex boundaries allows (a range may be empty)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    w = np.asarray(work, dtype=np.float64)
    n = len(w)
    pref = np.zeros(n + 1)
    np.cumsum(w, out=pref[1:])
    total = pref[-1]
    cuts = [0]
    for k in range(1, parts):
        c = int(np.searchsorted(pref, total * k / parts, side="left"))
        cuts.append(min(max(c, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[k], cuts[k + 1]) for k in range(parts)]


def combine(results) -> tuple[int, int]:
    """Sum of per-shard (count, hash) pairs, the hash mod 2^64."""
    c = sum(int(r[0]) for r in results)
    h = sum(int(r[1]) for r in results) % (1 << 64)
    return c, h
