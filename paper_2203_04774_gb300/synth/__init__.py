"""Seeded synthetic inputs: undirected edge lists and vertex orderings.

This module is shared by the CUDA path's tests and benches and by the CPU
oracle's tests.  It holds none of the listing method's arithmetic: it draws
edge lists (which may contain loops and duplicate pairs, exactly as a raw
dataset would before the cleaning of Sec. 4.1) and produces rank arrays
(0-based permutations: ``rank[v] = pi_v - 1`` with ``pi`` the 1-based index
of Sec. 1.3).  The orderings are inputs of the listing path (the "mere
listing" task of Sec. 3.2 takes the ordering as given).

Random numbers come from one counter-based generator, the splitmix64 output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the i-th draw of stream ``s`` under seed ``k`` is
``mix64(key(k, s) + (i + 1) * GAMMA)``.  Being counter-based, any slice of a
stream can be drawn independently and the result does not depend on how the
draws are chunked.

Stand-ins for the paper's datasets (Table 1 of Sec. 4.1 lists real web and
social graphs that are not available here):

* ``chung_lu``: power-law expected degrees, endpoints drawn i.i.d.
  proportional to the weights (social-network stand-in).
* ``rmat``: recursive-matrix graph (web/social stand-in).
* small exact families (complete, complete bipartite, star, random tree,
  G(n, p)) and the paper's own example graphs (Fig. 3, the L_d family of
  Appendix B, the G_phi construction of Appendix A), used as test fixtures.
"""
from __future__ import annotations

import math

import numpy as np

from .orderings import (  # noqa: F401  (re-exported)
    order_check,
    order_core,
    order_degree,
    order_degree_from_degrees,
    order_identity,
    order_neigh,
    order_random,
    order_split,
    simple_csr,
    simple_degrees,
)

GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied elementwise to a uint64 array."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    k = mix64(np.array([(seed * GAMMA + stream * 0xD1B54A32D192ED03) & _M64],
                       dtype=np.uint64))[0]
    return np.uint64(k)


def counter_u64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of stream ``stream`` under ``seed``."""
    key = _stream_key(seed, stream)
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key + i * np.uint64(GAMMA))


def counter_uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    x = counter_u64(seed, stream, count, start) >> np.uint64(11)
    return x.astype(np.float64) * (1.0 / (1 << 53))


def _draw_from_cdf(cdf: np.ndarray, seed: int, stream: int, count: int,
                   block: int = 1 << 24, threads: int = 1) -> np.ndarray:
    """Inverse-CDF draws of indices: draw i is the first index whose cdf
    exceeds uniform i of the stream.  Blocks are independent (the generator
    is counter-based), so ``threads`` > 1 draws them concurrently with the
    same result."""
    n = cdf.shape[0]
    out = np.empty(count, dtype=np.uint32)

    def one(s):
        c = min(block, count - s)
        u = counter_uniform(seed, stream, c, start=s)
        idx = np.searchsorted(cdf, u, side="right")
        np.minimum(idx, n - 1, out=idx)
        out[s:s + c] = idx

    starts = range(0, count, block)
    if threads > 1:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(one, starts))
    else:
        for s in starts:
            one(s)
    return out


# ---- arithmetic that gives the same bits on every machine -------------------
#
# Library routines for log, exp and pow may differ in their last bit between
# machines (numpy's vectorised float64 pow does on AVX-512 hosts), and a
# one-bit change of a Chung-Lu weight moves draws that fall on a bin edge,
# so the same seed would give slightly different graphs on the host that
# writes stored results and on the GPU machine.  These versions use only
# correctly rounded IEEE operations (+, -, *, /, exact frexp / ldexp / rint),
# one numpy ufunc at a time, in a fixed order; they are accurate to a few
# units in the last place and, above all, reproducible.

_LN2 = 0.6931471805599453


def det_log(x: np.ndarray) -> np.ndarray:
    """Natural logarithm of positive float64 values: x = m 2^k with m in
    [sqrt(1/2), sqrt(2)), ln m = 2 atanh(s), s = (m - 1) / (m + 1), summed as
    an odd series (|s| < 0.172, 14 terms reach double precision)."""
    x = np.asarray(x, dtype=np.float64)
    m, k = np.frexp(x)  # x = m 2^k, m in [0.5, 1)
    low = m < 0.7071067811865476
    m = np.where(low, m * 2.0, m)
    k = np.where(low, k - 1, k).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    acc = np.full_like(s, 1.0 / 29.0)
    for j in range(27, 0, -2):  # Horner over 1/29, 1/27, ..., 1/1
        acc = acc * s2
        acc = acc + 1.0 / j
    return k * _LN2 + 2.0 * s * acc


def det_exp(y: np.ndarray) -> np.ndarray:
    """exp of float64 values in a moderate range: y = q ln2 + r with q an
    integer and |r| <= ln2 / 2, exp r by its Taylor series (18 terms), then
    scaled by 2^q exactly."""
    y = np.asarray(y, dtype=np.float64)
    q = np.rint(y / _LN2)
    r = y - q * _LN2
    acc = np.full_like(r, 1.0)
    for j in range(18, 0, -1):  # Horner: 1 + r/1 (1 + r/2 (1 + ... (1 + r/18)))
        acc = acc * r
        acc = acc / j
        acc = acc + 1.0
    return np.ldexp(acc, q.astype(np.int64))


def det_pow(x: np.ndarray, e: float) -> np.ndarray:
    """x^e for positive x as exp(e ln x), reproducible bit for bit."""
    return det_exp(det_log(x) * float(e))


def chung_lu_weights(n: int, avg_deg: float, gamma: float) -> np.ndarray:
    """Expected-degree weights w_i proportional to (i+1)^(-1/(gamma-1)).

    Scaled so that sum(w) = n * avg_deg, then capped at sqrt(sum(w)) (the
    cap keeps every expected edge probability w_i w_j / sum(w) at most 1).
    The capped weights are not rescaled.  The power is det_pow and the sums
    are sequential (np.cumsum), so the weights are the same bits on every
    machine.
    """
    i = np.arange(n, dtype=np.float64)
    w = det_pow(i + 1.0, -1.0 / (gamma - 1.0))
    w *= (n * avg_deg) / np.cumsum(w)[-1]
    cap = math.sqrt(np.cumsum(w)[-1])
    np.minimum(w, cap, out=w)
    return w


def chung_lu(n: int, avg_deg: float, gamma: float, seed: int, threads: int = 1) -> np.ndarray:
    """Chung-Lu power-law multigraph as a raw edge list, uint32 [M, 2].

    M = round(n * avg_deg / 2) pairs, each endpoint drawn independently with
    probability proportional to the capped weights.  Loops and repeated pairs
    are left in; the listing path's graph loading removes them.  ``threads``
    only changes how fast the draws are made, not their values.
    """
    w = chung_lu_weights(n, avg_deg, gamma)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(round(n * avg_deg / 2.0))
    e = np.empty((m, 2), dtype=np.uint32)
    e[:, 0] = _draw_from_cdf(cdf, seed, 0, m, threads=threads)
    e[:, 1] = _draw_from_cdf(cdf, seed, 1, m, threads=threads)
    return e


def chung_lu_family(count: int, n_range: tuple[int, int], deg_range: tuple[float, float],
                    gamma_range: tuple[float, float], seed: int) -> dict:
    """Parameters of ``count`` independent Chung-Lu graphs: n log-uniform in
    n_range (rounded), average degree and exponent uniform in their ranges,
    and a distinct edge seed per graph (all from the counter generator under
    ``seed``, streams 10-12).  Graph i is ``chung_lu(n[i], deg[i], gamma[i],
    seeds[i])``."""
    lo, hi = det_log(np.array([float(n_range[0]), float(n_range[1])]))
    n = np.rint(det_exp(lo + (hi - lo) * counter_uniform(seed, 10, count))).astype(np.int64)
    n = np.clip(n, n_range[0], n_range[1])
    deg = deg_range[0] + (deg_range[1] - deg_range[0]) * counter_uniform(seed, 11, count)
    gam = gamma_range[0] + (gamma_range[1] - gamma_range[0]) * counter_uniform(seed, 12, count)
    seeds = (seed << 32) + np.arange(count, dtype=np.int64)
    pairs = np.rint(n * deg / 2.0).astype(np.int64)
    return {"n": n, "deg": deg, "gamma": gam, "seeds": seeds, "pairs": pairs}


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float,
         seed: int) -> np.ndarray:
    """R-MAT edge list (Chakrabarti, Zhan and Faloutsos, SDM 2004), uint32 [M, 2].

    M = edge_factor * 2^scale draws; at each of the ``scale`` levels one
    uniform draw picks the quadrant: [0,a) top-left, [a,a+b) top-right,
    [a+b,a+b+c) bottom-left, else bottom-right.  No noise, no id scrambling.
    """
    m = edge_factor << scale
    src = np.zeros(m, dtype=np.uint32)
    dst = np.zeros(m, dtype=np.uint32)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        u = counter_uniform(seed, level, m)
        bit = np.uint32(1 << (scale - 1 - level))
        sbit = u >= ab
        dbit = ((u >= a) & (u < ab)) | (u >= abc)
        src |= sbit.astype(np.uint32) * bit
        dst |= dbit.astype(np.uint32) * bit
    return np.stack([src, dst], axis=1)


def gnp(n: int, p: float, seed: int) -> np.ndarray:
    """Erdos-Renyi G(n, p): every pair i<j kept when its draw is < p."""
    iu, ju = np.triu_indices(n, k=1)
    keep = counter_uniform(seed, 0, iu.shape[0]) < p
    return np.stack([iu[keep], ju[keep]], axis=1).astype(np.uint32)


def complete(n: int) -> np.ndarray:
    iu, ju = np.triu_indices(n, k=1)
    return np.stack([iu, ju], axis=1).astype(np.uint32)


def complete_bipartite(a: int, b: int) -> np.ndarray:
    i, j = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return np.stack([i.ravel(), j.ravel()], axis=1).astype(np.uint32)


def star(n: int, hub: int = 0) -> np.ndarray:
    leaves = np.array([v for v in range(n) if v != hub], dtype=np.uint32)
    return np.stack([np.full_like(leaves, hub), leaves], axis=1)


def random_tree(n: int, seed: int) -> np.ndarray:
    """Random recursive tree: vertex i > 0 joins a uniform earlier vertex."""
    u = counter_uniform(seed, 0, n - 1)
    parent = np.floor(u * np.arange(1, n)).astype(np.uint32)
    return np.stack([parent, np.arange(1, n, dtype=np.uint32)], axis=1)


# --- the paper's example graphs ------------------------------------------

FIG3_NAMES = "abcdefg"
# The 7-vertex, 10-edge graph of Fig. 3 (the Neigh update example).
FIG3_EDGES = ["ad", "ab", "ae", "bc", "be", "bg", "cg", "de", "ef", "fg"]


def fig3_graph() -> np.ndarray:
    idx = {c: i for i, c in enumerate(FIG3_NAMES)}
    return np.array([[idx[s[0]], idx[s[1]]] for s in FIG3_EDGES], dtype=np.uint32)


def rank_from_sequence(seq: str, names: str = FIG3_NAMES) -> np.ndarray:
    """Rank array of an ordering written as a sequence of vertex names."""
    rank = np.empty(len(names), dtype=np.uint32)
    for pos, ch in enumerate(seq):
        rank[names.index(ch)] = pos
    return rank


def ld_gadget(d: int) -> tuple[np.ndarray, dict]:
    """The L_d graph of Appendix B: a (d+1)-clique K_0..K_d, d vertices
    v_1..v_d each joined to every K_j, and e_d joined to every v_i.

    Vertex ids: e_d = 0, v_i = i (1..d), K_j = d + 1 + j (0..d).
    """
    e = []
    ks = [d + 1 + j for j in range(d + 1)]
    for i in range(1, d + 1):
        e.append((0, i))
        for k in ks:
            e.append((i, k))
    for x in range(len(ks)):
        for y in range(x + 1, len(ks)):
            e.append((ks[x], ks[y]))
    return np.array(e, dtype=np.uint32).reshape(-1, 2), {"e": 0, "v": list(range(1, d + 1)), "K": ks}


def nae3sat_gadget(clauses: list[tuple[int, int, int]], n_vars: int) -> tuple[np.ndarray, dict]:
    """The G_phi graph of Appendix A for a positive 3-CNF formula.

    Each clause j gets three mutually joined literal vertices L_j^1..L_j^3;
    variable vertex X_i is joined to every literal vertex that names x_i.
    Vertex ids: X_i = i (0-based variables), L_j^a = n_vars + 3j + a.
    """
    e = []
    for j, cl in enumerate(clauses):
        lj = [n_vars + 3 * j + a for a in range(3)]
        e += [(lj[0], lj[1]), (lj[0], lj[2]), (lj[1], lj[2])]
        for a, var in enumerate(cl):
            e.append((var, lj[a]))
    return np.array(e, dtype=np.uint32).reshape(-1, 2), {"n": n_vars + 3 * len(clauses)}
