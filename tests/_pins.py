"""Independent definitions used to pin the oracle (pure Python, tiny inputs).

Nothing here is imported by the library.  These restate the mathematics the
paper fixes, not the paper's algorithms.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np


def simple_edge_set(edges) -> set[tuple[int, int]]:
    """The undirected simple graph of Sec. 1.3 behind a raw edge list."""
    out = set()
    for a, b in np.asarray(edges).reshape(-1, 2).tolist():
        if a != b:
            out.add((min(a, b), max(a, b)))
    return out


def brute_force_triangles(n: int, edges) -> list[tuple[int, int, int]]:
    """Every vertex set {a,b,c} whose three pairs are edges (Sec. 1.3), by
    testing all C(n,3) triples."""
    E = simple_edge_set(edges)
    adj = [[False] * n for _ in range(n)]
    for a, b in E:
        adj[a][b] = adj[b][a] = True
    tri = []
    for a, b, c in itertools.combinations(range(n), 3):
        if adj[a][b] and adj[a][c] and adj[b][c]:
            tri.append((a, b, c))
    return tri


def kn_costs(n: int) -> tuple[int, int, int]:
    """K_n under any ordering: the vertex at rank r has n-1-r successors and
    r predecessors, so C++ = sum r^2 = (n-1)n(2n-1)/6 and
    C+- = sum r(n-1-r) = n(n-1)(n-2)/6; every 3-set is a triangle."""
    return (n - 1) * n * (2 * n - 1) // 6, n * (n - 1) * (n - 2) // 6, comb(n, 3)


def ld_closed_form(d: int) -> int:
    """C_d of Appendix B: d^2 + d (d+1)^2 + sum_{i=0..d} i^2."""
    return d * d + d * (d + 1) ** 2 + sum(i * i for i in range(d + 1))


def ld_triangles(d: int) -> int:
    """Triangles of L_d: those of the (d+1)-clique, plus v_i with any two
    clique vertices (the v_i are pairwise non-adjacent and e_d touches only
    the v_i)."""
    return comb(d + 1, 3) + d * comb(d + 1, 2)
