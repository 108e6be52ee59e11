"""GB300-native triangle listing with a given vertex ordering (arXiv:2203.04774).

Python binding of ``libtl.so`` (C ABI in ``include/tl.h``).  The functions
``tl_*`` below marshal arguments and call the library; every step of the
listing path runs in the library's CUDA kernels.  PyTorch is used only to
hold device memory and to name streams.

There is no CPU fallback: if ``libtl.so`` is missing, ``lib()`` raises.
Build it with ``python -c "import __graft_entry__ as g; g.build()"``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtl.so")

TL_OK, TL_EINVAL, TL_ENOMEM, TL_ECUDA, TL_ESTATE, TL_ECALLBACK, TL_ETIMEOUT = range(7)
TL_APP, TL_APM, TL_AMM = 0, 1, 2
TL_MIN_CHUNK_BYTES = 12 << 20
STATUS_NAMES = {0: "TL_OK", 1: "TL_EINVAL", 2: "TL_ENOMEM", 3: "TL_ECUDA", 4: "TL_ESTATE",
                5: "TL_ECALLBACK", 6: "TL_ETIMEOUT"}

# Every symbol the header declares, with its ctypes signature.
_P, _U32, _U64, _I, _SZ = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                           ctypes.c_size_t)
CONSUMER = ctypes.CFUNCTYPE(ctypes.c_int, _P, _U64, _U64, _P)


class CountHashState(ctypes.Structure):
    _fields_ = [("count", _U64), ("hash", _U64), ("stream", _P), ("scratch", _P)]


class CountHashNoallocState(ctypes.Structure):
    _fields_ = [("dev_out", _P), ("stream", _P)]


TL_NOALLOC_MAX_TRIPLES = 1 << 28


class CountHashPartsState(ctypes.Structure):
    _fields_ = [("vbase", _P), ("k", _U32), ("counts", _P), ("hashes", _P), ("stream", _P)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", _SZ), ("max_batch", _U32), ("workers", _U32),
                ("chunk_bytes", _SZ)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", _I), ("batch_size", _U32), ("triangles", _U64), ("hash", _U64),
                ("t_submit_ns", _U64), ("t_admit_ns", _U64), ("t_done_ns", _U64),
                ("tuning_entry", ctypes.c_int32)]


TL_KERNELS = 5  # small, medium, narrow, mid, large


class ListStats(ctypes.Structure):
    _fields_ = [("launches", _U64), ("chunks", _U64), ("triangles", _U64), ("probes", _U64),
                ("tasks", _U64 * TL_KERNELS), ("kernel_ms", ctypes.c_double * TL_KERNELS),
                ("kernel_probes", _U64 * TL_KERNELS), ("kernel_triangles", _U64 * TL_KERNELS),
                ("bucketize_ms", ctypes.c_double), ("consumer_ms", ctypes.c_double),
                ("wall_ms", ctypes.c_double)]


class Tuning(ctypes.Structure):
    """tl_tuning: the work split of the listing kernels (speed only)."""
    _fields_ = [("small_max_p", _U32), ("medium_max_p", _U32), ("narrow_max_p", _U32),
                ("mid_max_p", _U32), ("warp_work", _U32), ("narrow_piece", _U32),
                ("mid_piece", _U32),
                ("large_per_p", _U32), ("large_min", _U32), ("large_max", _U32),
                ("narrow_keep_mib", _U32), ("narrow_cold_first", _U32),
                ("large_hash_max_p", _U32)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class TuningEntry(ctypes.Structure):
    """tl_tuning_entry: one row of a server's work-split table."""
    _fields_ = [("alg", _I), ("profile_p", ctypes.c_double * 33),
                ("profile_w", ctypes.c_double * 48), ("log2_m", ctypes.c_double),
                ("tuning", Tuning)]


SIGNATURES = {
    "tl_graph_load": ([ctypes.POINTER(_P), _U32, _P, _U64, _I, _P], _I),
    "tl_graph_load_parts": ([ctypes.POINTER(_P), _U32, _P, _P, _P, _I, _P], _I),
    "tl_graph_union": ([ctypes.POINTER(_P), _P, _P, _U32, _P], _I),
    "tl_graph_size": ([_P, ctypes.POINTER(_U32), ctypes.POINTER(_U64)], _I),
    "tl_order_apply": ([_P, _P, _I], _I),
    "tl_order_compute": ([_P, _I, _P, _I], _I),
    "tl_cost": ([_P, _I, ctypes.POINTER(_U64)], _I),
    "tl_list_triangles": ([_P, _I, _SZ, _P, _P, ctypes.POINTER(_U64)], _I),
    "tl_list_triangles_range": ([_P, _I, _U32, _U32, _SZ, _P, _P, ctypes.POINTER(_U64),
                                 ctypes.POINTER(_U64)], _I),
    "tl_count_hash": ([_P, _U64, _U64, _P], _I),
    "tl_count_hash_release": ([ctypes.POINTER(CountHashState)], None),
    "tl_graph_csr": ([_P, _I, _P, _P], _I),
    "tl_default_tuning": ([ctypes.POINTER(Tuning)], _I),
    "tl_work_profile": ([_P, _I, _U32, _U32, _P], _I),
    "tl_set_tuning": ([_P, ctypes.POINTER(Tuning)], _I),
    "tl_get_tuning": ([_P, ctypes.POINTER(Tuning)], _I),
    "tl_server_create": ([ctypes.POINTER(_P), ctypes.POINTER(ServerConfig)], _I),
    "tl_server_add_graph": ([_P, _P, ctypes.POINTER(_U32)], _I),
    "tl_server_add_ordering": ([_P, _U32, _P, _I, ctypes.POINTER(_U32)], _I),
    "tl_server_submit": ([_P, _U32, _U32, _I, ctypes.POINTER(_U64)], _I),
    "tl_server_wait": ([_P, _U64, ctypes.POINTER(RequestResult)], _I),
    "tl_server_footprint": ([_P, _U32, ctypes.POINTER(_U64), ctypes.POINTER(_U64)], _I),
    "tl_server_free": ([_P], None),
    "tl_server_set_tuning_table": ([_P, _P, _U32], _I),
    "tl_server_now_ns": ([], _U64),
    "tl_count_hash_noalloc": ([_P, _U64, _U64, _P], _I),
    "tl_count_hash_parts": ([_P, _U64, _U64, _P], _I),
    "tl_last_list_stats": ([_P, ctypes.POINTER(ListStats)], _I),
    "tl_kernel_launches": ([], _U64),
    "tl_graph_free": ([_P], None),
    "tl_last_error": ([], ctypes.c_char_p),
    "tl_version": ([], ctypes.c_char_p),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: the CUDA library must be built first "
                    "(__graft_entry__.build()); there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


class TLError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().tl_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status: int, where: str) -> None:
    if status != TL_OK:
        raise TLError(status, where)


def _ptr_and_flag(x):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            x = x.contiguous()
            return x.data_ptr(), int(x.is_cuda), x
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(x, dtype=np.uint32)
    return a.ctypes.data, 0, a


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---- functions with the C names ---------------------------------------------

def tl_graph_load(n: int, edges, stream=None) -> ctypes.c_void_p:
    """Load an undirected graph from uint32 pairs [m, 2] (host numpy or device torch)."""
    ptr, on_dev, keep = _ptr_and_flag(edges)
    m_in = int(np.prod(keep.shape)) // 2
    h = _P()
    _check(lib().tl_graph_load(ctypes.byref(h), n, ptr, m_in, on_dev, _stream_handle(stream)),
           "tl_graph_load")
    return h


def tl_graph_load_parts(n, m_in, edges, stream=None) -> ctypes.c_void_p:
    """Disjoint union of k graphs from one concatenated pair list with part-local ids.

    ``n`` and ``m_in`` are sequences of k part sizes and pair counts; ``edges``
    holds the parts' pairs one part after the other ([sum m_in, 2], host numpy
    or device torch)."""
    nn = np.ascontiguousarray(n, dtype=np.uint32)
    mm = np.ascontiguousarray(m_in, dtype=np.uint64)
    if nn.shape != mm.shape or nn.ndim != 1:
        raise ValueError("n and m_in must be 1-d sequences of equal length")
    ptr, on_dev, keep = _ptr_and_flag(edges)
    if int(np.prod(keep.shape)) != 2 * int(mm.sum()):
        raise ValueError("edges must hold 2 * sum(m_in) ids")
    h = _P()
    _check(lib().tl_graph_load_parts(ctypes.byref(h), len(nn), nn.ctypes.data, mm.ctypes.data,
                                     ptr, on_dev, _stream_handle(stream)),
           "tl_graph_load_parts")
    return h


def tl_graph_union(graphs, ranks=None, stream=None) -> ctypes.c_void_p:
    """Disjoint union of loaded graphs (handles), each under ranks[i] (a device
    torch uint32/int32 tensor of its n_i ranks) or its current ordering (None)."""
    k = len(graphs)
    harr = (_P * k)(*[g.value if isinstance(g, _P) else g for g in graphs])
    keep = []
    rarr = None
    if ranks is not None:
        if len(ranks) != k:
            raise ValueError("ranks must have one entry per graph")
        rarr = (_P * k)()
        for i, r in enumerate(ranks):
            if r is None:
                continue
            ptr, on_dev, kp = _ptr_and_flag(r)
            if not on_dev:
                raise ValueError("ranks must be device tensors")
            keep.append(kp)
            rarr[i] = ptr
    h = _P()
    _check(lib().tl_graph_union(ctypes.byref(h), harr, rarr, k, _stream_handle(stream)),
           "tl_graph_union")
    return h


def tl_graph_size(g) -> tuple[int, int]:
    n, m = _U32(), _U64()
    _check(lib().tl_graph_size(g, ctypes.byref(n), ctypes.byref(m)), "tl_graph_size")
    return int(n.value), int(m.value)


def tl_order_apply(g, rank) -> None:
    ptr, on_dev, keep = _ptr_and_flag(rank)
    _check(lib().tl_order_apply(g, ptr, on_dev), "tl_order_apply")


TL_ORDER_DEGREE, TL_ORDER_SPLIT, TL_ORDER_CORE = 0, 1, 2


def tl_order_compute(g, kind: int, rank=None):
    """Degree or Split ordering computed on the device.  With ``rank`` None a
    host uint32 array is returned; else ``rank`` (numpy or torch, n uint32)
    is filled in place."""
    if rank is None:
        n, _ = tl_graph_size(g)
        rank = np.empty(n, dtype=np.uint32)
    ptr, on_dev, keep = _ptr_and_flag(rank)
    _check(lib().tl_order_compute(g, kind, ptr, on_dev), "tl_order_compute")
    return rank


def tl_cost(g, alg: int) -> int:
    c = _U64()
    _check(lib().tl_cost(g, alg, ctypes.byref(c)), "tl_cost")
    return int(c.value)


def _consumer_ptr(cb):
    if cb is None:
        return None, None
    if isinstance(cb, CONSUMER):
        return ctypes.cast(cb, _P), cb
    if isinstance(cb, int):
        return cb, None
    wrapped = CONSUMER(cb)
    return ctypes.cast(wrapped, _P), wrapped


def tl_list_triangles(g, alg: int, chunk_bytes: int = TL_MIN_CHUNK_BYTES, cb=None,
                      user=None) -> int:
    cbp, keep = _consumer_ptr(cb)
    nt = _U64()
    _check(lib().tl_list_triangles(g, alg, chunk_bytes, cbp, user, ctypes.byref(nt)),
           "tl_list_triangles")
    return int(nt.value)


def tl_list_triangles_range(g, alg: int, x_begin: int, x_end: int,
                            chunk_bytes: int = TL_MIN_CHUNK_BYTES, cb=None,
                            user=None) -> tuple[int, int]:
    cbp, keep = _consumer_ptr(cb)
    nt, npb = _U64(), _U64()
    _check(lib().tl_list_triangles_range(g, alg, x_begin, x_end, chunk_bytes, cbp, user,
                                         ctypes.byref(nt), ctypes.byref(npb)),
           "tl_list_triangles_range")
    return int(nt.value), int(npb.value)


def tl_graph_csr(g, direction: int) -> tuple[np.ndarray, np.ndarray]:
    n, m = tl_graph_size(g)
    off = np.empty(n + 1, dtype=np.uint64)
    adj = np.empty(max(m, 1), dtype=np.uint32)
    _check(lib().tl_graph_csr(g, direction, off.ctypes.data, adj.ctypes.data), "tl_graph_csr")
    return off, adj[:m]


def tl_last_list_stats(g) -> dict:
    st = ListStats()
    _check(lib().tl_last_list_stats(g, ctypes.byref(st)), "tl_last_list_stats")
    return {"launches": int(st.launches), "chunks": int(st.chunks),
            "triangles": int(st.triangles), "probes": int(st.probes),
            "tasks": [int(v) for v in st.tasks],
            "kernel_ms": [float(v) for v in st.kernel_ms],
            "kernel_probes": [int(v) for v in st.kernel_probes],
            "kernel_triangles": [int(v) for v in st.kernel_triangles],
            "bucketize_ms": float(st.bucketize_ms), "consumer_ms": float(st.consumer_ms),
            "wall_ms": float(st.wall_ms)}


TL_PROFILE_BINS_P, TL_PROFILE_BINS_W = 33, 48


def tl_work_profile(g, alg: int, x_begin: int = 0, x_end: int | None = None) -> np.ndarray:
    """uint64 [TL_PROFILE_BINS_P, TL_PROFILE_BINS_W]: summed tests W_x of the
    B vertices by bit length of their probe-set size p_x and of W_x."""
    if x_end is None:
        x_end = tl_graph_size(g)[0]
    h = np.zeros(TL_PROFILE_BINS_P * TL_PROFILE_BINS_W, dtype=np.uint64)
    _check(lib().tl_work_profile(g, alg, x_begin, x_end, h.ctypes.data), "tl_work_profile")
    return h.reshape(TL_PROFILE_BINS_P, TL_PROFILE_BINS_W)


def tl_default_tuning() -> dict:
    t = Tuning()
    _check(lib().tl_default_tuning(ctypes.byref(t)), "tl_default_tuning")
    return t.as_dict()


def tl_set_tuning(g, tuning: dict | None) -> None:
    """Set the work split of later listings on g (None: the defaults).  Keys
    missing from `tuning` keep the graph's current values."""
    if tuning is None:
        _check(lib().tl_set_tuning(g, None), "tl_set_tuning")
        return
    t = Tuning()
    _check(lib().tl_get_tuning(g, ctypes.byref(t)), "tl_get_tuning")
    for k, v in tuning.items():
        setattr(t, k, int(v))
    _check(lib().tl_set_tuning(g, ctypes.byref(t)), "tl_set_tuning")


def tl_get_tuning(g) -> dict:
    t = Tuning()
    _check(lib().tl_get_tuning(g, ctypes.byref(t)), "tl_get_tuning")
    return t.as_dict()


def tl_kernel_launches() -> int:
    return int(lib().tl_kernel_launches())


def tl_graph_free(g) -> None:
    if g:
        lib().tl_graph_free(g)


def tl_count_hash_ptr() -> int:
    """Address of the library's count + hash consumer (pass as ``cb``)."""
    return ctypes.cast(lib().tl_count_hash, _P).value


# ---- conveniences -----------------------------------------------------------

class _DevView:
    """Exposes a device buffer of triples through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {
            "shape": (n, 3), "typestr": "<u4", "data": (ptr, False), "version": 2}


class Collect:
    """Consumer that copies every chunk to host memory (tests, small graphs)."""

    def __init__(self):
        self.parts: list[np.ndarray] = []
        self.calls = 0
        self.error: BaseException | None = None
        self.fn = CONSUMER(self._on_chunk)

    def _on_chunk(self, ptr, n, idx, user):
        try:
            import torch
            self.calls += 1
            if n:
                t = torch.as_tensor(_DevView(ptr, n), device="cuda")
                self.parts.append(t.cpu().numpy().copy())
            return 0
        except BaseException as e:  # surfaced by the caller after the C call returns
            self.error = e
            return 1

    def triples(self) -> np.ndarray:
        if not self.parts:
            return np.zeros((0, 3), dtype=np.uint32)
        return np.concatenate(self.parts).astype(np.uint32)


class CountHash:
    """The library's device count + hash consumer."""

    def __init__(self, stream=None):
        self.state = CountHashState(0, 0, _stream_handle(stream), None)

    @property
    def user(self):
        return ctypes.cast(ctypes.pointer(self.state), _P)

    def reset(self):
        self.state.count = 0
        self.state.hash = 0

    def release(self):
        lib().tl_count_hash_release(ctypes.byref(self.state))


class CountHashParts:
    """The library's per-part count + hash consumer for a disjoint union.

    ``sizes`` are the parts' vertex counts n_i; the offsets, counts and hashes
    live in device tensors owned by this object."""

    def __init__(self, sizes, stream=None, device="cuda"):
        import torch
        sizes = np.asarray(sizes, dtype=np.int64)
        vb = np.zeros(len(sizes) + 1, dtype=np.int64)
        np.cumsum(sizes, out=vb[1:])
        self.vbase = torch.as_tensor(vb, device=device)
        self.counts = torch.zeros(len(sizes), dtype=torch.int64, device=device)
        self.hashes = torch.zeros(len(sizes), dtype=torch.int64, device=device)
        self.state = CountHashPartsState(self.vbase.data_ptr(), len(sizes),
                                         self.counts.data_ptr(), self.hashes.data_ptr(),
                                         _stream_handle(stream))

    @property
    def user(self):
        return ctypes.cast(ctypes.pointer(self.state), _P)

    @staticmethod
    def fn() -> int:
        return ctypes.cast(lib().tl_count_hash_parts, _P).value

    def reset(self):
        self.counts.zero_()
        self.hashes.zero_()

    def results(self) -> tuple[np.ndarray, np.ndarray]:
        """(counts, hashes) as uint64 numpy arrays, one entry per part."""
        return (self.counts.cpu().numpy().view(np.uint64).copy(),
                self.hashes.cpu().numpy().view(np.uint64).copy())


class Graph:
    """A graph handle: load, order, cost, list (thin wrapper over tl_*)."""

    def __init__(self, n: int, edges, stream=None):
        self.n = n
        self.h = tl_graph_load(n, edges, stream)

    @classmethod
    def _wrap(cls, h) -> "Graph":
        g = cls.__new__(cls)
        g.h = h
        g.n = tl_graph_size(h)[0]
        return g

    @classmethod
    def load_parts(cls, n, m_in, edges, stream=None) -> "Graph":
        """Disjoint union of graphs given as one concatenated pair list."""
        return cls._wrap(tl_graph_load_parts(n, m_in, edges, stream))

    @classmethod
    def union(cls, graphs, ranks=None, stream=None) -> "Graph":
        """Disjoint union of Graph objects under the given (or current) orderings."""
        return cls._wrap(tl_graph_union([g.h for g in graphs], ranks, stream))

    def order_compute(self, kind: int, rank=None):
        """Device ordering (TL_ORDER_DEGREE / _SPLIT / _CORE) as ranks; a new
        CUDA int32 tensor unless ``rank`` is given."""
        if rank is None:
            import torch
            rank = torch.empty(self.n, dtype=torch.int32, device="cuda")
        return tl_order_compute(self.h, kind, rank)

    def list_count_hash_parts(self, alg: int, sizes, chunk_bytes: int = TL_MIN_CHUNK_BYTES,
                              x_begin: int = 0, x_end: int | None = None, stream=None):
        """(triangles, per-part counts, per-part hashes, probes) of a union."""
        ch = CountHashParts(sizes, stream)
        nt, npb = tl_list_triangles_range(self.h, alg, x_begin,
                                          self.n if x_end is None else x_end, chunk_bytes,
                                          ch.fn(), ch.user)
        c, h = ch.results()
        return nt, c, h, npb

    def __del__(self):
        self.free()

    def free(self):
        h = getattr(self, "h", None)
        if h:
            tl_graph_free(h)
        self.h = None

    @property
    def m(self) -> int:
        return tl_graph_size(self.h)[1]

    def order_apply(self, rank) -> None:
        tl_order_apply(self.h, rank)

    def cost(self, alg: int) -> int:
        return tl_cost(self.h, alg)

    def csr(self, direction: int):
        return tl_graph_csr(self.h, direction)

    def list_collect(self, alg: int, chunk_bytes: int = TL_MIN_CHUNK_BYTES,
                     x_begin: int = 0, x_end: int | None = None):
        c = Collect()
        try:
            nt, npb = tl_list_triangles_range(self.h, alg, x_begin,
                                              self.n if x_end is None else x_end, chunk_bytes,
                                              c.fn, None)
        except TLError:
            if c.error is not None:
                raise c.error
            raise
        return c.triples(), nt, npb, c.calls

    def list_count_hash(self, alg: int, chunk_bytes: int = TL_MIN_CHUNK_BYTES,
                        x_begin: int = 0, x_end: int | None = None, stream=None):
        ch = CountHash(stream)
        try:
            nt, npb = tl_list_triangles_range(self.h, alg, x_begin,
                                              self.n if x_end is None else x_end, chunk_bytes,
                                              tl_count_hash_ptr(), ch.user)
            return nt, int(ch.state.count), int(ch.state.hash), npb
        finally:
            ch.release()


class Server:
    """Request loop over device-resident graphs (tl_server_*): continuous
    batching into disjoint unions, admission by estimated device footprint."""

    def __init__(self, hbm_budget_bytes: int, max_batch: int = 256, workers: int = 2,
                 chunk_bytes: int = 64 << 20):
        cfg = ServerConfig(hbm_budget_bytes, max_batch, workers, chunk_bytes)
        self.h = _P()
        _check(lib().tl_server_create(ctypes.byref(self.h), ctypes.byref(cfg)),
               "tl_server_create")
        self._graphs = []  # registered graphs stay alive as long as the server

    def add_graph(self, g: "Graph") -> int:
        gid = _U32()
        _check(lib().tl_server_add_graph(self.h, g.h, ctypes.byref(gid)), "tl_server_add_graph")
        self._graphs.append(g)
        return int(gid.value)

    def add_ordering(self, graph_id: int, rank) -> int:
        ptr, on_dev, keep = _ptr_and_flag(rank)
        oid = _U32()
        _check(lib().tl_server_add_ordering(self.h, graph_id, ptr, on_dev, ctypes.byref(oid)),
               "tl_server_add_ordering")
        return int(oid.value)

    def footprint(self, graph_id: int) -> tuple[int, int]:
        """(bytes charged per request on graph_id, bytes charged per batch)."""
        r, b = _U64(), _U64()
        _check(lib().tl_server_footprint(self.h, graph_id, ctypes.byref(r), ctypes.byref(b)),
               "tl_server_footprint")
        return int(r.value), int(b.value)

    def set_tuning_table(self, entries: list | None) -> None:
        """Work splits by degree profile for later batches: entries in the form
        of autotune.py's table (None or [] restores the defaults)."""
        names = {"A++": TL_APP, "A+-": TL_APM, "A--": TL_AMM}
        arr = (TuningEntry * max(1, len(entries or [])))()
        defaults = Tuning()
        _check(lib().tl_default_tuning(ctypes.byref(defaults)), "tl_default_tuning")
        for k, e in enumerate(entries or []):
            arr[k].alg = names[e["alg"]]
            for i, v in enumerate(e["profile"]["p"]):
                arr[k].profile_p[i] = v
            for i, v in enumerate(e["profile"]["w"]):
                arr[k].profile_w[i] = v
            arr[k].log2_m = float(np.log2(max(e["profile"]["m"], 1)))
            t = Tuning.from_buffer_copy(defaults)
            for f, v in e["tuning"].items():
                setattr(t, f, int(v))
            arr[k].tuning = t
        _check(lib().tl_server_set_tuning_table(self.h, arr, len(entries or [])),
               "tl_server_set_tuning_table")

    def submit(self, graph_id: int, ordering_id: int, alg: int) -> int:
        rid = _U64()
        _check(lib().tl_server_submit(self.h, graph_id, ordering_id, alg, ctypes.byref(rid)),
               "tl_server_submit")
        return int(rid.value)

    def wait(self, request_id: int) -> dict:
        r = RequestResult()
        _check(lib().tl_server_wait(self.h, request_id, ctypes.byref(r)), "tl_server_wait")
        return {"status": int(r.status), "batch_size": int(r.batch_size),
                "triangles": int(r.triangles), "hash": int(r.hash),
                "t_submit_ns": int(r.t_submit_ns), "t_admit_ns": int(r.t_admit_ns),
                "t_done_ns": int(r.t_done_ns), "tuning_entry": int(r.tuning_entry)}

    @staticmethod
    def now_ns() -> int:
        return int(lib().tl_server_now_ns())

    def close(self):
        h = getattr(self, "h", None)
        if h:
            lib().tl_server_free(h)
        self.h = None
        self._graphs = []

    def __del__(self):
        self.close()
