"""CPU oracle for triangle listing with a given vertex ordering.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may use this package; the library under
test never does.  It wraps ``oracle.cpp`` (plain C++17, compiled here with
g++) through ctypes and shares no code with the CUDA library.

Parity status of every function is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, the paper's printed Fig. 3 and Split values,
the Appendix A/B gadgets, Property 1 and cross-ordering invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

APP = 0  # Algorithm 1, A++
APM = 1  # Algorithm 2, A+-
AMM = 2  # A--, the third variant (seed edge S2), cost C--
LITERAL = 0
SETS = 1


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++ -O2, C++17)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
            lib.or_graph_new.argtypes = [U32, P, U64, ctypes.POINTER(P)]
            lib.or_graph_new.restype = I
            lib.or_graph_free.argtypes = [P]
            lib.or_graph_free.restype = None
            lib.or_num_edges.argtypes = [P]
            lib.or_num_edges.restype = U64
            lib.or_order_apply.argtypes = [P, P]
            lib.or_order_apply.restype = I
            lib.or_cost.argtypes = [P, I]
            lib.or_cost.restype = U64
            lib.or_list.argtypes = [P, I, I, U32, U32, P, U64, P, P, P]
            lib.or_list.restype = I
            lib.or_csr.argtypes = [P, I, P, P]
            lib.or_csr.restype = I
            lib.or_degrees.argtypes = [P, P]
            lib.or_degrees.restype = I
            lib.or_hash_triples.argtypes = [P, U64]
            lib.or_hash_triples.restype = U64
            lib.or_mix64.argtypes = [U64]
            lib.or_mix64.restype = U64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


class Graph:
    """Undirected simple graph + ordering, as the paper's CPU algorithms see it."""

    def __init__(self, n: int, edges: np.ndarray):
        lib = _load()
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.uint32).reshape(-1, 2))
        h = ctypes.c_void_p()
        st = lib.or_graph_new(n, _ptr(e), e.shape[0], ctypes.byref(h))
        if st != 0:
            raise OracleError(f"or_graph_new: invalid edge list (status {st})")
        self._h = h
        self.n = n

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.or_graph_free(h)
            self._h = None

    @property
    def m(self) -> int:
        return int(_lib.or_num_edges(self._h))

    def order_apply(self, rank: np.ndarray) -> None:
        r = np.ascontiguousarray(np.asarray(rank, dtype=np.uint32))
        if r.shape[0] != self.n:
            raise OracleError("rank has the wrong length")
        if _lib.or_order_apply(self._h, _ptr(r)) != 0:
            raise OracleError("rank is not a permutation of [0, n)")

    def cost(self, alg: int) -> int:
        return int(_lib.or_cost(self._h, alg))

    def list(self, alg: int, mode: int = LITERAL, seed_begin: int = 0,
             seed_end: int | None = None, store: bool = True):
        """Returns (triples uint32[T,3] or None, count, hash, probes)."""
        if seed_end is None:
            seed_end = self.n
        cnt, hsh, prb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        if store:
            # First pass counts, second pass stores (the oracle is deliberately
            # simple; running it twice is cheaper than guessing a size).
            st = _lib.or_list(self._h, alg, mode, seed_begin, seed_end, None, 0,
                              ctypes.byref(cnt), ctypes.byref(hsh), ctypes.byref(prb))
            if st != 0:
                raise OracleError(f"or_list status {st}")
            buf = np.empty((int(cnt.value), 3), dtype=np.uint32)
            st = _lib.or_list(self._h, alg, mode, seed_begin, seed_end, _ptr(buf),
                              buf.shape[0], ctypes.byref(cnt), ctypes.byref(hsh),
                              ctypes.byref(prb))
            if st != 0:
                raise OracleError(f"or_list status {st}")
            return buf, int(cnt.value), int(hsh.value), int(prb.value)
        st = _lib.or_list(self._h, alg, mode, seed_begin, seed_end, None, 0,
                          ctypes.byref(cnt), ctypes.byref(hsh), ctypes.byref(prb))
        if st != 0:
            raise OracleError(f"or_list status {st}")
        return None, int(cnt.value), int(hsh.value), int(prb.value)

    def degrees(self) -> np.ndarray:
        """Degree of every vertex of the cleaned simple graph (Sec. 1.3)."""
        deg = np.empty(self.n, dtype=np.uint32)
        _lib.or_degrees(self._h, _ptr(deg))
        return deg

    def csr(self, direction: int):
        """(off uint64[n+1], adj uint32[m]) of N+ (0) or N- (1), rank space."""
        off = np.empty(self.n + 1, dtype=np.uint64)
        adj = np.empty(self.m, dtype=np.uint32)
        _lib.or_csr(self._h, direction, _ptr(off), _ptr(adj))
        return off, adj


def hash_triples(triples: np.ndarray) -> int:
    t = np.ascontiguousarray(np.asarray(triples, dtype=np.uint32).reshape(-1, 3))
    return int(_load().or_hash_triples(_ptr(t), t.shape[0]))


def mix64(z: int) -> int:
    return int(_load().or_mix64(z))


def canonical(triples: np.ndarray) -> np.ndarray:
    """Triples as a lexicographically sorted uint32[T,3] array (each row a<b<c)."""
    t = np.asarray(triples, dtype=np.uint32).reshape(-1, 3)
    t = np.sort(t, axis=1)
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
    return t[order]


def core_numbers(n: int, edges: np.ndarray) -> np.ndarray:
    """Coreness c_v of every vertex (Sec. 1.3: the largest k such that v lies
    in a subgraph whose vertices all have degree >= k), by the plain
    peeling argument: repeatedly delete a vertex of minimum remaining
    degree; c_v is the largest minimum degree seen up to v's deletion.
    Pure Python with a lazy heap -- small graphs only."""
    import heapq
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    pairs = np.unique(lo * n + hi)
    adj = [[] for _ in range(n)]
    for key in pairs.tolist():
        a, b = divmod(key, n)
        adj[a].append(b)
        adj[b].append(a)
    deg = [len(x) for x in adj]
    heap = [(d, v) for v, d in enumerate(deg)]
    heapq.heapify(heap)
    gone = [False] * n
    core = np.zeros(n, dtype=np.int64)
    k = 0
    while heap:
        d, v = heapq.heappop(heap)
        if gone[v] or d != deg[v]:
            continue
        gone[v] = True
        k = max(k, d)
        core[v] = k
        for u in adj[v]:
            if not gone[u]:
                deg[u] -= 1
                heapq.heappush(heap, (deg[u], u))
    return core


def core_order_levels(n: int, edges: np.ndarray) -> np.ndarray:
    """Ranks of the level-synchronous core ordering (the reading of the core
    ordering of Sec. 1.3 taken by the device path), computed one vertex at a
    time: at level k, every remaining vertex of degree <= k is removed in one
    round; the vertices whose degree falls to k while that round's vertices
    are deleted form the next round; when a round is empty, k moves up to the
    smallest remaining degree (or k+1).  Vertices are ranked by (round, id).
    The outcome does not depend on the order in which a round's deletions are
    made: a vertex enters the next round when its degree reaches k, whichever
    neighbour brings it there."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    adj = [[] for _ in range(n)]
    for key in np.unique(lo * n + hi).tolist():
        a, b = divmod(key, n)
        adj[a].append(b)
        adj[b].append(a)
    deg = [len(x) for x in adj]
    removed = [False] * n
    rnd_of = [0] * n
    active = set(range(n))
    k, rnd = 0, 0
    while active:
        frontier = sorted(v for v in active if deg[v] <= k)
        if not frontier:
            k = max(k + 1, min(deg[v] for v in active))
            continue
        for v in frontier:
            removed[v] = True
        active.difference_update(frontier)
        while frontier:
            nxt = []
            for v in frontier:
                rnd_of[v] = rnd
                for u in adj[v]:
                    if not removed[u]:
                        deg[u] -= 1
                        if deg[u] == k:
                            removed[u] = True
                            nxt.append(u)
            active.difference_update(nxt)
            rnd += 1
            frontier = nxt
        k += 1
    order = sorted(range(n), key=lambda v: (rnd_of[v], v))
    rank = np.empty(n, dtype=np.uint32)
    rank[np.asarray(order, dtype=np.int64)] = np.arange(n, dtype=np.uint32)
    return rank
