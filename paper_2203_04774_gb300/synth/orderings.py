"""Vertex orderings (inputs of the listing path), as 0-based rank arrays.

``rank[v] = pi_v - 1`` where ``pi`` is the 1-based ordering of Sec. 1.3.

* identity: the "original ordering" of the dataset (Sec. 2.2).
* random: a uniformly random permutation (ranks = positions after a stable
  sort of per-vertex counter draws).
* degree: non-decreasing degree (Sec. 2.2), ties by increasing id.
* core: degeneracy (core) ordering (Sec. 1.3), Batagelj-Zaversnik peeling.
* split / check / neigh: the paper's three heuristics of Sec. 3.3.

The sequential heuristics (core, check, neigh) run in a small C helper
(``orderings.c``) compiled on first use with the system C compiler.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orderings.c")
_LIB = os.path.join(_HERE, "_orderings.so")
_lock = threading.Lock()
_lib = None


def build_helper(force: bool = False) -> str:
    """Compile the C helper in place (plain C99, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _helper():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_helper())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.tls_order_core.argtypes = [I64, P, P, P]
            lib.tls_order_core.restype = I64
            lib.tls_order_check.argtypes = [I64, P, P, P, P]
            lib.tls_order_check.restype = None
            lib.tls_order_neigh.argtypes = [I64, P, P, P, ctypes.c_double, I64, P, I64]
            lib.tls_order_neigh.restype = I64
            lib.tls_neigh_move_one.argtypes = [I64, P, P, P, I64, I64]
            lib.tls_neigh_move_one.restype = None
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def simple_csr(n: int, edges: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric CSR of the simple graph behind a raw edge list.

    Loops dropped, pairs merged regardless of direction (the cleaning of
    Sec. 4.1).  Rows sorted by id.  Used only to compute orderings.
    """
    e = np.asarray(edges, dtype=np.uint64).reshape(-1, 2)
    a, b = e[:, 0], e[:, 1]
    keep = a != b
    lo = np.minimum(a, b)[keep]
    hi = np.maximum(a, b)[keep]
    key = np.unique((lo << np.uint64(32)) | hi)
    lo = (key >> np.uint64(32)).astype(np.int64)
    hi = (key & np.uint64(0xFFFFFFFF)).astype(np.int64)
    both = np.sort(np.concatenate([lo * n + hi, hi * n + lo]))
    src, dst = both // n, both % n
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=off[1:])
    return off, dst.astype(np.uint32)


def degrees(off: np.ndarray) -> np.ndarray:
    return np.diff(off)


def simple_degrees(n: int, edges: np.ndarray) -> np.ndarray:
    """Degrees in the simple graph behind a raw edge list (no CSR built)."""
    e = np.asarray(edges, dtype=np.uint64).reshape(-1, 2)
    a, b = e[:, 0], e[:, 1]
    keep = a != b
    key = np.unique((np.minimum(a, b)[keep] << np.uint64(32)) | np.maximum(a, b)[keep])
    lo = (key >> np.uint64(32)).astype(np.int64)
    hi = (key & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return np.bincount(lo, minlength=n) + np.bincount(hi, minlength=n)


def order_degree_from_degrees(deg: np.ndarray) -> np.ndarray:
    """Non-decreasing degree, ties by increasing id."""
    return _positions_to_rank(np.argsort(deg, kind="stable"))


def _positions_to_rank(seq: np.ndarray) -> np.ndarray:
    rank = np.empty(seq.shape[0], dtype=np.uint32)
    rank[seq] = np.arange(seq.shape[0], dtype=np.uint32)
    return rank


def order_identity(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.uint32)


def order_random(n: int, seed: int) -> np.ndarray:
    from . import counter_u64
    keys = counter_u64(seed, 0x5EED, n)
    return _positions_to_rank(np.argsort(keys, kind="stable"))


def order_degree(off: np.ndarray) -> np.ndarray:
    """Non-decreasing degree, ties by increasing id."""
    deg = degrees(off)
    return _positions_to_rank(np.argsort(deg, kind="stable"))


def by_degree_desc(off: np.ndarray) -> np.ndarray:
    """Vertices by non-increasing degree, ties by increasing id."""
    deg = degrees(off)
    return np.lexsort((np.arange(deg.shape[0]), -deg)).astype(np.uint32)


def order_core(off: np.ndarray, adj: np.ndarray) -> np.ndarray:
    n = off.shape[0] - 1
    rank = np.empty(n, dtype=np.uint32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    _helper().tls_order_core(n, _p(off), _p(adj), _p(rank))
    return rank


def order_split(off: np.ndarray | None = None, delta: np.ndarray | None = None) -> np.ndarray:
    """Split heuristic (Sec. 3.3.3).

    ``delta`` lists the vertices by non-increasing degree (default: ties by
    id).  The vertex at 1-based position 2i+1 of delta gets pi = i+1; the one
    at position 2i gets pi = n+1-i.
    """
    if delta is None:
        delta = by_degree_desc(off)
    delta = np.asarray(delta, dtype=np.int64)
    n = delta.shape[0]
    pos = np.arange(n, dtype=np.int64)          # 0-based position in delta
    r = np.where(pos % 2 == 0, pos // 2, n - (pos + 1) // 2)
    rank = np.empty(n, dtype=np.uint32)
    rank[delta] = r.astype(np.uint32)
    return rank


def order_check(off: np.ndarray, adj: np.ndarray, order: np.ndarray | None = None) -> np.ndarray:
    """Check heuristic (Sec. 3.3.2); vertices taken by non-increasing degree."""
    n = off.shape[0] - 1
    if order is None:
        order = by_degree_desc(off)
    order = np.ascontiguousarray(order, dtype=np.uint32)
    rank = np.empty(n, dtype=np.uint32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    _helper().tls_order_check(n, _p(off), _p(adj), _p(order), _p(rank))
    return rank


_OBJECTIVES = {"C+-": 0, "C++": 1}


def order_neigh(off: np.ndarray, adj: np.ndarray, start: np.ndarray | None = None,
                eps: float = 1e-2, max_iter: int = 50,
                objective: str = "C+-") -> tuple[np.ndarray, list[int]]:
    """Neigh heuristic (Algorithm 3), epsilon = 1e-2 as in Sec. 3.3.1.

    Minimises ``objective``: "C+-" (the paper's), or "C++" (the same local
    moves for the cost of Algorithm 1; Sec. 3.3.1 notes that the heuristic
    serves other objectives, C++ among them).  Starts from ``start`` (default: the degree
    ordering).  Returns the rank array and the objective before each pass and
    after the last one.
    """
    obj = _OBJECTIVES[objective]
    n = off.shape[0] - 1
    rank = np.array(order_degree(off) if start is None else start, dtype=np.uint32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    trace = np.zeros(max_iter + 1, dtype=np.int64)
    it = _helper().tls_order_neigh(n, _p(off), _p(adj), _p(rank), eps, max_iter, _p(trace), obj)
    return rank, [int(x) for x in trace[: it + 1]]


def neigh_move_one(off: np.ndarray, adj: np.ndarray, rank: np.ndarray, u: int,
                   objective: str = "C+-") -> np.ndarray:
    """One Neigh update of vertex ``u`` (the move shown in Fig. 3)."""
    obj = _OBJECTIVES[objective]
    n = off.shape[0] - 1
    r = np.array(rank, dtype=np.uint32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    _helper().tls_neigh_move_one(n, _p(off), _p(adj), _p(r), int(u), obj)
    return r
