"""Python binding of libgpm.so (include/gpm.h): argument marshalling only.

Every count and listing runs in the library's CUDA kernels; this module only
converts numpy arrays / torch tensors to pointers, torch streams to
cudaStream_t handles, and status codes to exceptions. There is no CPU
fallback: importing this module raises if libgpm.so has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2011_03135_b300.build` "
                      "(the library has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

GPM_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "NOT_SORTED", -3: "SELF_LOOP", -4: "DUPLICATE", -5: "ASYMMETRIC",
    -6: "DISCONNECTED_PATTERN", -7: "K_TOO_LARGE", -8: "OOM", -9: "DEVICE", -10: "TIMEOUT", -11: "BUSY",
    -12: "UNSUPPORTED", -13: "OVERFLOW", -14: "OUT_OF_RANGE",
}
GRAPH_VALIDATE = 1
GRAPH_DEVICE_INPUT = 2
STRATEGY_CLIQUE_DAG, STRATEGY_LOCAL_COUNT, STRATEGY_EDGE, STRATEGY_ENUMERATE, STRATEGY_GUIDED = 1, 2, 3, 4, 5
MOTIF4_NAMES = ("3-star", "4-path", "tailed-triangle", "4-cycle", "diamond", "4-clique")
MOTIF3_NAMES = ("wedge", "triangle")


class GpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("max_degree", ctypes.c_uint32), ("nnz", ctypes.c_uint64),
                ("dag_arcs", ctypes.c_uint64), ("max_out_degree", ctypes.c_uint32), ("prepared", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64)]


class PatternInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("n_edges", ctypes.c_uint32), ("induced", ctypes.c_uint32),
                ("is_clique", ctypes.c_uint32), ("strategy", ctypes.c_uint32), ("motif_index", ctypes.c_uint32),
                ("automorphisms", ctypes.c_uint64), ("n_sb_pairs", ctypes.c_uint32),
                ("sb_pairs", ctypes.c_uint32 * 56), ("matching_order", ctypes.c_uint32 * 8),
                ("min_degree", ctypes.c_uint32 * 8)]


class Query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("kind", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


QUERY_MOTIF3, QUERY_MOTIF4, QUERY_TC, QUERY_CLIQUE4, QUERY_CLIQUE5 = 3, 4, 5, 6, 7
QUERY_WIDTH = {QUERY_MOTIF3: 2, QUERY_MOTIF4: 6, QUERY_TC: 1, QUERY_CLIQUE4: 1, QUERY_CLIQUE5: 1}


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("reserved0", ctypes.c_uint32), ("arena_bytes", ctypes.c_uint64),
                ("ring_items", ctypes.c_uint64), ("reserved", ctypes.c_uint64 * 4)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("graph", ctypes.c_uint32), ("kind", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("ncounts", ctypes.c_uint32), ("counts", ctypes.c_uint64 * 6)]


class Options(ctypes.Structure):
    _fields_ = [("warp_max_degree", ctypes.c_uint32), ("cta_max_degree", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("c4_hub_bound", ctypes.c_uint32),
                ("batch_direct_us", ctypes.c_uint32), ("c4_range_bound", ctypes.c_uint32),
                ("c4_range_width", ctypes.c_uint32), ("c4_pull_bound", ctypes.c_uint32)]


_vp, _u32, _u64, _i = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_U64P = ctypes.POINTER(ctypes.c_uint64)
_SIGS = {
    "gpm_graph_create": [_vp, _vp, _u32, _u64, _u32, _vp, ctypes.POINTER(_vp)],
    "gpm_graph_destroy": [_vp],
    "gpm_graph_prepare": [_vp, _vp],
    "gpm_graph_info": [_vp, ctypes.POINTER(GraphInfo)],
    "gpm_pattern_spec": [_u32, _vp, _i, ctypes.POINTER(_vp)],
    "gpm_pattern_clique": [_u32, ctypes.POINTER(_vp)],
    "gpm_pattern_motifs": [_u32, _vp, ctypes.POINTER(_u32)],
    "gpm_pattern_destroy": [_vp],
    "gpm_pattern_info": [_vp, ctypes.POINTER(PatternInfo)],
    "gpm_count": [_vp, _vp, _u32, _vp, _vp],
    "gpm_count_async": [_vp, _vp, _u32, _vp, _vp],
    "gpm_count_roots": [_vp, _vp, _u32, _u32, _u32, _vp, _vp],
    "gpm_count_enumerate": [_vp, _vp, _u32, _vp, _vp],
    "gpm_count_guided": [_vp, _vp, _u32, _vp, _vp],
    "gpm_count_cliques": [_vp, _u32, _u32, _u32, _vp, _vp],
    "gpm_exists": [_vp, _vp, _vp, _vp, _vp],
    "gpm_list": [_vp, _vp, _vp, _u64, _U64P, _U64P, _vp],
    "gpm_graph_reset": [_vp],
    "gpm_graph_set_orientation": [_vp, _u32],
    "gpm_graph_core_numbers": [_vp, _vp, _vp],
    "gpm_profile_enable": [_i],
    "gpm_profile_reset": [],
    "gpm_profile_report": [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
    "gpm_batch_create": [_vp, _u32, ctypes.POINTER(_vp)],
    "gpm_batch_run": [_vp, _vp, _vp],
    "gpm_batch_direct": [_vp, ctypes.POINTER(_u32), _U64P],
    "gpm_batch_info": [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_u32),
                       ctypes.POINTER(_u32)],
    "gpm_batch_destroy": [_vp],
    "gpm_count_batch": [_vp, _u32, _vp, _vp],
    "gpm_count_cycles4_noalloc": [_vp, _vp, _u32, _vp, _vp],
    "gpm_server_start": [_vp, _u32, ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)],
    "gpm_server_submit": [_vp, _u32, _u32, _u64],
    "gpm_server_poll": [_vp, ctypes.POINTER(Completion), _u32, ctypes.POINTER(_u32)],
    "gpm_server_stats": [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32)],
    "gpm_server_stop": [_vp],
    "gpm_set_options": [ctypes.POINTER(Options)],
    "gpm_get_options": [ctypes.POINTER(Options)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.gpm_last_error.argtypes = []
_lib.gpm_last_error.restype = ctypes.c_char_p
_lib.gpm_version.argtypes = []
_lib.gpm_version.restype = ctypes.c_char_p
_lib.gpm_kernel_launches.argtypes = []
_lib.gpm_kernel_launches.restype = ctypes.c_uint64


def _check(rc: int):
    if rc != GPM_OK:
        raise GpmError(rc, _lib.gpm_last_error().decode(errors="replace"))


def version() -> str:
    return _lib.gpm_version().decode()


def _stream(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _ptr(x):
    """(address, is_device, keepalive) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            x = np.ascontiguousarray(x)
        return x.ctypes.data, False, x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr(), x.is_cuda, x
    raise TypeError(f"expected a numpy array or a torch tensor, got {type(x)}")


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(_lib.gpm_kernel_launches())


def profile_enable(on: bool = True):
    _check(_lib.gpm_profile_enable(int(bool(on))))


def profile_reset():
    _check(_lib.gpm_profile_reset())


def profile_report() -> dict:
    """{kernel: {"launches": L, "ms": T}} summed since the last reset (call after synchronising)."""
    import json
    need = ctypes.c_size_t(0)
    _check(_lib.gpm_profile_report(None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value + 16)
    _check(_lib.gpm_profile_report(buf, len(buf), ctypes.byref(need)))
    return json.loads(buf.value.decode())


def set_options(warp_max_degree: int = 0, cta_max_degree: int = 0, blocks_per_sm: int = 0, c4_hub_bound: int = 0,
                batch_direct_us: int = 0, c4_range_bound: int = 0, c4_range_width: int = 0, c4_pull_bound: int = 0):
    o = Options(warp_max_degree, cta_max_degree, blocks_per_sm, c4_hub_bound, batch_direct_us, c4_range_bound,
                c4_range_width, c4_pull_bound)
    _check(_lib.gpm_set_options(ctypes.byref(o)))


def get_options() -> dict:
    o = Options()
    _check(_lib.gpm_get_options(ctypes.byref(o)))
    return dict(warp_max_degree=o.warp_max_degree, cta_max_degree=o.cta_max_degree, blocks_per_sm=o.blocks_per_sm,
                c4_hub_bound=o.c4_hub_bound, batch_direct_us=o.batch_direct_us, c4_range_bound=o.c4_range_bound,
                c4_range_width=o.c4_range_width, c4_pull_bound=o.c4_pull_bound)


class Graph:
    """A device-resident graph (library-owned copy of a symmetric sorted CSR)."""

    def __init__(self, rowptr, col, n: int | None = None, validate: bool = True, stream=None):
        rp, rp_dev, self._k1 = _ptr(rowptr)
        cp, cp_dev, self._k2 = _ptr(col)
        if rp_dev != cp_dev:
            raise ValueError("rowptr and col must both be host or both be device arrays")
        if n is None:
            n = len(rowptr) - 1
        nnz = int(col.shape[0]) if hasattr(col, "shape") else len(col)
        if isinstance(rowptr, np.ndarray) and rowptr.dtype != np.uint64:
            raise TypeError("rowptr must be uint64")
        if isinstance(col, np.ndarray) and col.dtype != np.uint32:
            raise TypeError("col must be uint32")
        flags = (GRAPH_VALIDATE if validate else 0) | (GRAPH_DEVICE_INPUT if rp_dev else 0)
        h = _vp()
        _check(_lib.gpm_graph_create(rp, cp if nnz else None, n, nnz, flags, _stream(stream), ctypes.byref(h)))
        self._h = h
        self.n = n
        self.nnz = nnz
        self._k1 = self._k2 = None

    @classmethod
    def from_host(cls, g, validate: bool = True, stream=None):
        """From an object with .rowptr (uint64) and .col (uint32) numpy arrays."""
        return cls(g.rowptr, g.col, g.n, validate=validate, stream=stream)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("graph has been destroyed")
        return self._h

    def prepare(self, stream=None):
        _check(_lib.gpm_graph_prepare(self.handle, _stream(stream)))
        return self

    def reset(self):
        """Drop the orientation so the next count rebuilds it (buffers are kept)."""
        _check(_lib.gpm_graph_reset(self.handle))
        return self

    def set_orientation(self, mode: str):
        """Order of the orientation: "degree" (default) or "core" (core numbers)."""
        modes = {"degree": 0, "core": 1}
        if mode not in modes:
            raise ValueError("orientation is 'degree' or 'core'")
        _check(_lib.gpm_graph_set_orientation(self.handle, modes[mode]))
        return self

    def core_numbers(self, stream=None) -> np.ndarray:
        """Core number of every vertex (k-core peeling on the device), as a host array."""
        out = np.zeros(max(self.n, 1), dtype=np.uint32)
        _check(_lib.gpm_graph_core_numbers(self.handle, out.ctypes.data, _stream(stream)))
        return out[: self.n]

    def info(self) -> dict:
        i = GraphInfo()
        _check(_lib.gpm_graph_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in GraphInfo._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.gpm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Pattern:
    """A planned pattern (library-owned)."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def spec(cls, adj, induced: bool = True):
        a = np.ascontiguousarray(np.asarray(adj, dtype=np.uint8))
        k = a.shape[0]
        h = _vp()
        _check(_lib.gpm_pattern_spec(k, a.ctypes.data, int(bool(induced)), ctypes.byref(h)))
        return cls(h)

    @classmethod
    def clique(cls, k: int):
        h = _vp()
        _check(_lib.gpm_pattern_clique(k, ctypes.byref(h)))
        return cls(h)

    @classmethod
    def motifs(cls, k: int):
        arr = (_vp * 32)()
        npat = _u32(0)
        _check(_lib.gpm_pattern_motifs(k, arr, ctypes.byref(npat)))
        return [cls(_vp(arr[i])) for i in range(npat.value)]

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = PatternInfo()
        _check(_lib.gpm_pattern_info(self._h, ctypes.byref(i)))
        return dict(k=i.k, n_edges=i.n_edges, induced=i.induced, is_clique=i.is_clique, strategy=i.strategy,
                    motif_index=i.motif_index, automorphisms=i.automorphisms,
                    sb_pairs=[(i.sb_pairs[2 * j], i.sb_pairs[2 * j + 1]) for j in range(i.n_sb_pairs)],
                    matching_order=list(i.matching_order[: i.k]), min_degree=list(i.min_degree[: i.k]))

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.gpm_pattern_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _handles(patterns: Sequence[Pattern]):
    arr = (_vp * len(patterns))()
    for i, p in enumerate(patterns):
        arr[i] = p.handle
    return arr


def count(graph: Graph, patterns: Sequence[Pattern], stream=None) -> list:
    """Exact counts (host), one per pattern."""
    out = np.zeros(len(patterns), dtype=np.uint64)
    _check(_lib.gpm_count(graph.handle, _handles(patterns), len(patterns), out.ctypes.data, _stream(stream)))
    return [int(x) for x in out]


def count_async(graph: Graph, patterns: Sequence[Pattern], out, stream=None):
    """Enqueue the counts into a device tensor (uint64 / int64, len >= npat); no synchronisation."""
    p, dev, _keep = _ptr(out)
    if not dev:
        raise ValueError("count_async needs a device output tensor")
    _check(_lib.gpm_count_async(graph.handle, _handles(patterns), len(patterns), p, _stream(stream)))


def count_enumerate(graph: Graph, patterns: Sequence[Pattern], stream=None) -> list:
    """Counts by pattern-oblivious enumeration with connectivity codes (all patterns with the same k = 3, 4, 5)."""
    out = np.zeros(len(patterns), dtype=np.uint64)
    _check(_lib.gpm_count_enumerate(graph.handle, _handles(patterns), len(patterns), out.ctypes.data,
                                    _stream(stream)))
    return [int(x) for x in out]


def count_guided(graph: Graph, patterns: Sequence[Pattern], stream=None) -> list:
    """Counts by the pattern-guided search (any connected pattern with 3..8 vertices)."""
    out = np.zeros(len(patterns), dtype=np.uint64)
    _check(_lib.gpm_count_guided(graph.handle, _handles(patterns), len(patterns), out.ctypes.data,
                                 _stream(stream)))
    return [int(x) for x in out]


def count_roots(graph: Graph, patterns: Sequence[Pattern], root_lo: int, root_hi: int, stream=None) -> list:
    """Counts of embeddings whose root vertex lies in [root_lo, root_hi)."""
    out = np.zeros(len(patterns), dtype=np.uint64)
    _check(_lib.gpm_count_roots(graph.handle, _handles(patterns), len(patterns), root_lo, root_hi,
                                out.ctypes.data, _stream(stream)))
    return [int(x) for x in out]


def count_cliques(graph: Graph, k: int, root_lo: int = 0, root_hi: int | None = None, stream=None) -> int:
    """Number of k-cliques (k = 3..9) whose root vertex lies in [root_lo, root_hi)."""
    out = ctypes.c_uint64(0)
    hi = graph.n if root_hi is None else root_hi
    _check(_lib.gpm_count_cliques(graph.handle, k, root_lo, hi, ctypes.byref(out), _stream(stream)))
    return int(out.value)


def exists(graph: Graph, pattern: Pattern, stream=None):
    """(found, witness): whether the graph holds an embedding of the pattern,
    and one such embedding (pattern vertex order) or None; stops at the first match."""
    k = pattern.info()["k"]
    found = ctypes.c_int(0)
    w = np.zeros(k, dtype=np.uint32)
    _check(_lib.gpm_exists(graph.handle, pattern.handle, ctypes.byref(found), w.ctypes.data, _stream(stream)))
    return bool(found.value), (w if found.value else None)


def list_embeddings(graph: Graph, pattern: Pattern, cap: int, out=None, stream=None):
    """List up to `cap` embeddings. Returns (tuples[written, k], total).

    `out` may be a preallocated uint32 numpy array / torch tensor (host or
    device) with room for cap*k entries; by default a host array is returned.
    """
    k = pattern.info()["k"]
    if out is None:
        out = np.zeros((max(cap, 1), k), dtype=np.uint32)
    p, _dev, _keep = _ptr(out)
    written, total = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_lib.gpm_list(graph.handle, pattern.handle, p if cap else None, cap, ctypes.byref(written),
                         ctypes.byref(total), _stream(stream)))
    return out[: written.value], int(total.value)


def _queries(queries):
    arr = (Query * len(queries))()
    for i, (g, kind) in enumerate(queries):
        arr[i].graph = g.handle
        arr[i].kind = kind
    return arr


class Batch:
    """Many (graph, kind) count queries run by one persistent kernel replayed from a CUDA graph."""

    def __init__(self, queries):
        self._queries = list(queries)
        self._arr = _queries(self._queries)
        h = _vp()
        _check(_lib.gpm_batch_create(self._arr, len(self._queries), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None) -> list:
        out = np.zeros(6 * len(self._queries), dtype=np.uint64)
        _check(_lib.gpm_batch_run(self._h, out.ctypes.data, _stream(stream)))
        return [[int(x) for x in out[6 * i: 6 * i + QUERY_WIDTH[k]]] for i, (_, k) in enumerate(self._queries)]

    def info(self) -> dict:
        a, b, c, d = _u32(), _u32(), _u32(), _u32()
        _check(_lib.gpm_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        nd, gk = _u32(), ctypes.c_uint64()
        _check(_lib.gpm_batch_direct(self._h, ctypes.byref(nd), ctypes.byref(gk)))
        return dict(items=a.value, roots_per_item=b.value, verts_per_item=c.value, grid=d.value,
                    direct_queries=nd.value, graph_kernels=gk.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.gpm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count_batch(queries, stream=None) -> list:
    """One-shot batched counts for [(Graph, QUERY_*), ...]."""
    arr = _queries(queries)
    out = np.zeros(6 * len(queries), dtype=np.uint64)
    _check(_lib.gpm_count_batch(arr, len(queries), out.ctypes.data, _stream(stream)))
    return [[int(x) for x in out[6 * i: 6 * i + QUERY_WIDTH[k]]] for i, (_, k) in enumerate(queries)]


def plain_patterns(kind):
    """The patterns a one-query-per-call gpm_count needs for a batch query kind."""
    if kind == QUERY_MOTIF3:
        return Pattern.motifs(3)
    if kind == QUERY_MOTIF4:
        return Pattern.motifs(4)
    return [Pattern.clique({QUERY_TC: 3, QUERY_CLIQUE4: 4, QUERY_CLIQUE5: 5}[kind])]


class Server:
    """Continuous-batching request loop over resident graphs (see gpm_server_start)."""

    def __init__(self, graphs, max_inflight: int = 256, arena_bytes: int = 0, ring_items: int = 0):
        self._graphs = list(graphs)
        arr = (_vp * len(self._graphs))()
        for i, g in enumerate(self._graphs):
            arr[i] = g.handle
        o = ServerOpts(max_inflight, 0, arena_bytes, ring_items)
        h = _vp()
        _check(_lib.gpm_server_start(arr, len(self._graphs), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._buf = (Completion * 4096)()

    def submit(self, graph: int, kind: int, tag: int):
        _check(_lib.gpm_server_submit(self._h, graph, kind, tag))

    def poll(self) -> list:
        """[(tag, graph, kind, status, counts)] of requests finished since the last poll."""
        n = _u32(0)
        _check(_lib.gpm_server_poll(self._h, self._buf, len(self._buf), ctypes.byref(n)))
        out = []
        for i in range(n.value):
            c = self._buf[i]
            out.append((int(c.tag), int(c.graph), int(c.kind), int(c.status),
                        [int(c.counts[j]) for j in range(c.ncounts)]))
        return out

    def stats(self) -> dict:
        a, b = _u32(), _u32()
        _check(_lib.gpm_server_stats(self._h, ctypes.byref(a), ctypes.byref(b)))
        return dict(inflight=a.value, pending=b.value)

    def stop(self):
        if getattr(self, "_h", None) is not None:
            _check(_lib.gpm_server_stop(self._h))
            self._h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
