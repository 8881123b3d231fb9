"""CPU oracle for graph pattern mining -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The library's product path never loads
it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain single-threaded C, exact integer
counts with 128-bit accumulation and overflow detection); this module only
marshals numpy arrays through ctypes. See ``oracle.c`` for the definition each
function follows and the paper passage it restates.

Parity status: every function here is pinned by the not-gpu tests (closed
forms, brute force on tiny graphs, the paper's worked examples); none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_E_ARG, ORC_E_OOM, ORC_E_OVERFLOW, ORC_E_CAP = 0, -1, -2, -3, -4

# Motif output order for k = 4 and k = 3 (by edge count, then as listed).
MOTIF4_NAMES = ("3-star", "4-path", "tailed-triangle", "4-cycle", "diamond", "4-clique")
MOTIF3_NAMES = ("wedge", "triangle")


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (host gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
            U64P = ctypes.POINTER(ctypes.c_uint64)
            sig = {
                "orc_automorphisms": ([u32, vp], u64),
                "orc_bf_induced": ([u32, vp, vp, u32, vp, U64P], ctypes.c_int),
                "orc_bf_noninduced": ([u32, vp, vp, u32, vp, U64P], ctypes.c_int),
                "orc_bf_maps": ([u32, vp, vp, u32, vp, vp, u64, U64P], ctypes.c_int),
                "orc_out_degrees": ([u32, vp, vp, vp], ctypes.c_int),
                "orc_cliques": ([u32, vp, vp, u32, u32, u32, U64P], ctypes.c_int),
                "orc_triangles": ([u32, vp, vp, U64P], ctypes.c_int),
                "orc_core_numbers": ([u32, vp, vp, vp], ctypes.c_int),
                "orc_core_order": ([u32, vp, vp, vp], ctypes.c_int),
                "orc_motifs5": ([u32, vp, vp, vp, vp], ctypes.c_int),
                "orc_motifs5_roots": ([u32, vp, vp, u32, u32, vp, vp], ctypes.c_int),
                "orc_cliques_keyed": ([u32, vp, vp, vp, u32, u32, u32, U64P], ctypes.c_int),
                "orc_diamonds": ([u32, vp, vp, u32, u32, U64P], ctypes.c_int),
                "orc_cycles4": ([u32, vp, vp, u32, u32, U64P], ctypes.c_int),
                "orc_noninduced_terms": ([u32, vp, vp, u32, vp], ctypes.c_int),
                "orc_motifs": ([u32, vp, vp, u32, vp], ctypes.c_int),
                "orc_eq1_local_wedges": ([ctypes.c_int64, ctypes.c_int64, ctypes.c_int64], ctypes.c_int64),
                "orc_edge_wedges_direct": ([vp, vp, u32, u32, U64P], ctypes.c_int),
                "orc_connectivity_code": ([vp, vp, vp, u32, U64P], ctypes.c_int),
                "orc_code_to_adjacency": ([u32, u64, vp], ctypes.c_int),
                "orc_connectivity_map_lookup": ([vp, vp, vp, u32, u32], u64),
                "orc_orders_satisfying": ([u32, vp, u32], u64),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _csr(g):
    rp = np.ascontiguousarray(g.rowptr, dtype=np.uint64)
    col = np.ascontiguousarray(g.col, dtype=np.uint32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.uint32)
    return rp, col


def _check(rc, what):
    if rc != ORC_OK:
        raise OracleError(f"{what}: oracle error {rc}")


def _adj(k, padj):
    a = np.ascontiguousarray(np.asarray(padj, dtype=np.uint8).reshape(k, k))
    return a


# ---------------- patterns ----------------

def automorphisms(padj) -> int:
    a = np.asarray(padj, dtype=np.uint8)
    k = a.shape[0]
    a = np.ascontiguousarray(a)
    return int(_load().orc_automorphisms(k, a.ctypes.data))


def orders_satisfying(k: int, pairs) -> int:
    p = np.ascontiguousarray(np.asarray(pairs, dtype=np.uint32).reshape(-1, 2))
    if p.size == 0:
        p = np.zeros((1, 2), dtype=np.uint32)
        return int(_load().orc_orders_satisfying(k, p.ctypes.data, 0))
    return int(_load().orc_orders_satisfying(k, p.ctypes.data, p.shape[0]))


# ---------------- tier 1: brute force ----------------

def bf_induced(g, padj) -> int:
    a = _adj(len(padj), padj)
    rp, col = _csr(g)
    out = ctypes.c_uint64(0)
    _check(_load().orc_bf_induced(g.n, rp.ctypes.data, col.ctypes.data, a.shape[0], a.ctypes.data,
                                  ctypes.byref(out)), "bf_induced")
    return int(out.value)


def bf_noninduced(g, padj) -> int:
    a = _adj(len(padj), padj)
    rp, col = _csr(g)
    out = ctypes.c_uint64(0)
    _check(_load().orc_bf_noninduced(g.n, rp.ctypes.data, col.ctypes.data, a.shape[0], a.ctypes.data,
                                     ctypes.byref(out)), "bf_noninduced")
    return int(out.value)


def bf_maps(g, padj, cap: int = 1 << 22) -> np.ndarray:
    """Every injective map of the pattern into G that sends pattern edges to graph edges."""
    a = _adj(len(padj), padj)
    k = a.shape[0]
    rp, col = _csr(g)
    buf = np.zeros((max(cap, 1), k), dtype=np.uint32)
    nm = ctypes.c_uint64(0)
    _check(_load().orc_bf_maps(g.n, rp.ctypes.data, col.ctypes.data, k, a.ctypes.data, buf.ctypes.data, cap,
                               ctypes.byref(nm)), "bf_maps")
    return buf[: nm.value].copy()


def bf_subgraph_set(g, padj) -> set:
    """The set of distinct edge-induced embeddings of P in G, each as a frozenset of edges."""
    a = np.asarray(padj, dtype=np.uint8)
    k = a.shape[0]
    pedges = [(i, j) for i in range(k) for j in range(i + 1, k) if a[i, j]]
    out = set()
    for f in bf_maps(g, a):
        out.add(frozenset((min(f[i], f[j]), max(f[i], f[j])) for i, j in pedges))
    return out


# ---------------- tier 2: exact plain algorithms ----------------

def out_degrees(g) -> np.ndarray:
    rp, col = _csr(g)
    od = np.zeros(max(g.n, 1), dtype=np.uint32)
    _check(_load().orc_out_degrees(g.n, rp.ctypes.data, col.ctypes.data, od.ctypes.data), "out_degrees")
    return od[: g.n]


def cliques(g, k: int, root_lo: int = 0, root_hi: int | None = None) -> int:
    rp, col = _csr(g)
    hi = g.n if root_hi is None else root_hi
    out = ctypes.c_uint64(0)
    _check(_load().orc_cliques(g.n, rp.ctypes.data, col.ctypes.data, k, root_lo, hi, ctypes.byref(out)),
           "cliques")
    return int(out.value)


def core_numbers(g) -> np.ndarray:
    """Core number of every vertex (the key of the core value based orientation)."""
    rp, col = _csr(g)
    out = np.zeros(max(g.n, 1), dtype=np.uint32)
    _check(_load().orc_core_numbers(g.n, rp.ctypes.data, col.ctypes.data, out.ctypes.data), "core_numbers")
    return out[: g.n]


def core_order(g) -> np.ndarray:
    """Round of the level-synchronous peel that takes each vertex (the degeneracy order)."""
    rp, col = _csr(g)
    out = np.zeros(max(g.n, 1), dtype=np.uint32)
    _check(_load().orc_core_order(g.n, rp.ctypes.data, col.ctypes.data, out.ctypes.data), "core_order")
    return out[: g.n]


def cliques_keyed(g, key, k: int, root_lo: int = 0, root_hi: int | None = None) -> int:
    """k-cliques whose first vertex in the order (key, id) lies in [root_lo, root_hi)."""
    rp, col = _csr(g)
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    hi = g.n if root_hi is None else root_hi
    out = ctypes.c_uint64(0)
    _check(_load().orc_cliques_keyed(g.n, rp.ctypes.data, col.ctypes.data, key.ctypes.data, k, root_lo, hi,
                                     ctypes.byref(out)), "cliques_keyed")
    return int(out.value)


def triangles(g) -> int:
    rp, col = _csr(g)
    out = ctypes.c_uint64(0)
    _check(_load().orc_triangles(g.n, rp.ctypes.data, col.ctypes.data, ctypes.byref(out)), "triangles")
    return int(out.value)


def diamonds(g, root_lo: int = 0, root_hi: int | None = None) -> int:
    rp, col = _csr(g)
    hi = g.n if root_hi is None else root_hi
    out = ctypes.c_uint64(0)
    _check(_load().orc_diamonds(g.n, rp.ctypes.data, col.ctypes.data, root_lo, hi, ctypes.byref(out)),
           "diamonds")
    return int(out.value)


def cycles4(g, root_lo: int = 0, root_hi: int | None = None) -> int:
    rp, col = _csr(g)
    hi = g.n if root_hi is None else root_hi
    out = ctypes.c_uint64(0)
    _check(_load().orc_cycles4(g.n, rp.ctypes.data, col.ctypes.data, root_lo, hi, ctypes.byref(out)),
           "cycles4")
    return int(out.value)


def noninduced_terms(g, k: int) -> list:
    rp, col = _csr(g)
    out = np.zeros(6, dtype=np.uint64)
    _check(_load().orc_noninduced_terms(g.n, rp.ctypes.data, col.ctypes.data, k, out.ctypes.data),
           "noninduced_terms")
    return [int(x) for x in out[: (2 if k == 3 else 6)]]


def motifs(g, k: int) -> list:
    """Induced counts of every connected k-vertex pattern (k = 3: wedge, triangle; k = 4: see MOTIF4_NAMES)."""
    rp, col = _csr(g)
    out = np.zeros(6, dtype=np.uint64)
    _check(_load().orc_motifs(g.n, rp.ctypes.data, col.ctypes.data, k, out.ctypes.data), "motifs")
    return [int(x) for x in out[: (2 if k == 3 else 6)]]


def motifs5(g, root_lo: int = 0, root_hi: int | None = None):
    """(counts, class_masks): induced counts of the 21 connected 5-vertex
    patterns and each class's canonical adjacency mask (bit of pair (a, b),
    a < b, in lexicographic pair order), ordered by edge count, then mask.
    With a root range, only the subgraphs whose smallest vertex lies in it."""
    rp, col = _csr(g)
    out = np.zeros(21, dtype=np.uint64)
    masks = np.zeros(21, dtype=np.uint32)
    hi = g.n if root_hi is None else root_hi
    _check(_load().orc_motifs5_roots(g.n, rp.ctypes.data, col.ctypes.data, root_lo, hi, out.ctypes.data,
                                     masks.ctypes.data), "motifs5")
    return [int(x) for x in out], [int(m) for m in masks]


# ---------------- worked examples ----------------

def eq1_local_wedges(deg_u: int, deg_v: int, c_tri: int) -> int:
    return int(_load().orc_eq1_local_wedges(deg_u, deg_v, c_tri))


def edge_wedges_direct(g, u: int, v: int) -> int:
    rp, col = _csr(g)
    out = ctypes.c_uint64(0)
    _check(_load().orc_edge_wedges_direct(rp.ctypes.data, col.ctypes.data, u, v, ctypes.byref(out)),
           "edge_wedges_direct")
    return int(out.value)


def connectivity_code(g, emb) -> str:
    rp, col = _csr(g)
    e = np.ascontiguousarray(np.asarray(emb, dtype=np.uint32))
    code = ctypes.c_uint64(0)
    nbits = _load().orc_connectivity_code(rp.ctypes.data, col.ctypes.data, e.ctypes.data, len(e),
                                          ctypes.byref(code))
    return format(code.value, f"0{nbits}b") if nbits else ""


def code_to_adjacency(k: int, code: str) -> np.ndarray:
    adj = np.zeros((k, k), dtype=np.uint8)
    _load().orc_code_to_adjacency(k, int(code, 2), adj.ctypes.data)
    return adj


def connectivity_map_lookup(g, emb, v: int) -> list:
    rp, col = _csr(g)
    e = np.ascontiguousarray(np.asarray(emb, dtype=np.uint32))
    bits = int(_load().orc_connectivity_map_lookup(rp.ctypes.data, col.ctypes.data, e.ctypes.data, len(e), v))
    return [i for i in range(len(e)) if bits >> i & 1]


# ---------------- named patterns (k x k adjacency, vertex order as documented) ----------------

def pattern(k: int, edges) -> np.ndarray:
    a = np.zeros((k, k), dtype=np.uint8)
    for i, j in edges:
        a[i, j] = a[j, i] = 1
    return a


def clique_pattern(k: int) -> np.ndarray:
    return pattern(k, [(i, j) for i in range(k) for j in range(i + 1, k)])


# 4-vertex connected patterns in MOTIF4_NAMES order
MOTIF4_PATTERNS = (
    pattern(4, [(0, 1), (0, 2), (0, 3)]),                          # 3-star, centre 0
    pattern(4, [(0, 1), (1, 2), (2, 3)]),                          # 4-path
    pattern(4, [(0, 1), (0, 2), (1, 2), (2, 3)]),                  # tailed triangle, tail at 2
    pattern(4, [(0, 2), (2, 1), (1, 3), (3, 0)]),                  # 4-cycle 0-2-1-3-0
    pattern(4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)]),          # diamond, shared edge (0,1)
    clique_pattern(4),                                             # 4-clique
)
MOTIF3_PATTERNS = (
    pattern(3, [(0, 1), (0, 2)]),                                  # wedge, centre 0
    clique_pattern(3),                                             # triangle
)
DIAMOND = MOTIF4_PATTERNS[4]
CYCLE4 = MOTIF4_PATTERNS[3]
