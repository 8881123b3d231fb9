"""Seeded synthetic input graphs (host side, shared by the oracle tests and the CUDA path).

Nothing here mines patterns: it samples graphs and assembles the symmetric,
loop-free, duplicate-free, sorted CSR that the paper assumes of its inputs
(Section 6, Table of input graphs). The sampling code is C (``graphgen.c``),
loaded through ctypes and compiled on first use with the host ``gcc`` when the
shared library is missing.

Every function returns ``Graph(n, rowptr: uint64[n+1], col: uint32[nnz])``.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so next to it (host gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P64 = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64))
            P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))
            U64P = ctypes.POINTER(ctypes.c_uint64)
            lib.gg_free.argtypes = [ctypes.c_void_p]
            lib.gg_free.restype = None
            lib.gg_csr_from_edges.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                              P64, P32, U64P]
            lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, P64, P32, U64P]
            lib.gg_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.c_int, P64, P32, U64P, ctypes.POINTER(ctypes.c_double)]
            lib.gg_erdos_renyi.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int,
                                           P64, P32, U64P]
            for f in (lib.gg_csr_from_edges, lib.gg_rmat, lib.gg_chung_lu, lib.gg_erdos_renyi):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Undirected simple graph as a symmetric sorted CSR (host numpy arrays)."""

    n: int
    rowptr: np.ndarray  # uint64[n+1]
    col: np.ndarray  # uint32[nnz], nnz = 2 * (number of undirected edges)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[int(self.rowptr[v]):int(self.rowptr[v + 1])]

    def digest(self) -> str:
        h = hashlib.sha256()
        h.update(np.uint64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.rowptr).tobytes())
        h.update(np.ascontiguousarray(self.col).tobytes())
        return h.hexdigest()[:16]

    def edges(self) -> np.ndarray:
        """Undirected edges (u < v) as an int64 array of shape (m, 2)."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr).astype(np.int64))
        dst = self.col.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)


def _take(rc, n, rp, cp, nnz, name, meta=None) -> Graph:
    lib = _load()
    if rc != 0:
        raise ValueError(f"graph generator failed with code {rc}")
    try:
        rowptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
        col = np.ctypeslib.as_array(cp, shape=(max(int(nnz.value), 1),))[: int(nnz.value)].copy()
    finally:
        lib.gg_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.gg_free(ctypes.cast(cp, ctypes.c_void_p))
    return Graph(n, rowptr.astype(np.uint64), col.astype(np.uint32), name, meta or {})


def _out():
    return ctypes.POINTER(ctypes.c_uint64)(), ctypes.POINTER(ctypes.c_uint32)(), ctypes.c_uint64(0)


def from_edges(n: int, edges, name: str = "edges") -> Graph:
    """CSR from an undirected edge list (symmetrised, loops and duplicates dropped)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if e.size and (e.min() < 0 or e.max() >= n):
        raise ValueError("edge endpoint out of range")
    src = np.ascontiguousarray(e[:, 0].astype(np.uint32))
    dst = np.ascontiguousarray(e[:, 1].astype(np.uint32))
    rp, cp, nnz = _out()
    rc = _load().gg_csr_from_edges(n, src.ctypes.data, dst.ctypes.data, len(src), ctypes.byref(rp),
                                   ctypes.byref(cp), ctypes.byref(nnz))
    return _take(rc, n, rp, cp, nnz, name)


def rmat(scale: int, edge_factor: float = 16.0, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 1,
         permute: bool = True) -> Graph:
    """R-MAT graph with 2**scale vertices from edge_factor * 2**scale edge samples."""
    a, b, c, _ = abcd
    rp, cp, nnz = _out()
    rc = _load().gg_rmat(scale, float(edge_factor), a, b, c, seed, int(permute), ctypes.byref(rp),
                         ctypes.byref(cp), ctypes.byref(nnz))
    return _take(rc, 1 << scale, rp, cp, nnz, f"rmat-s{scale}-ef{edge_factor:g}-seed{seed}",
                 dict(kind="rmat", scale=scale, edge_factor=edge_factor, abcd=tuple(abcd), seed=seed))


def chung_lu(n: int, dbar: float = 24.0, gamma: float = 2.1, seed: int = 3, permute: bool = True) -> Graph:
    """Chung-Lu power-law graph: mean expected degree dbar, exponent gamma, cutoff sqrt(n*dbar)."""
    rp, cp, nnz = _out()
    wmax = ctypes.c_double(0.0)
    rc = _load().gg_chung_lu(n, float(dbar), float(gamma), seed, int(permute), ctypes.byref(rp),
                             ctypes.byref(cp), ctypes.byref(nnz), ctypes.byref(wmax))
    return _take(rc, n, rp, cp, nnz, f"chunglu-n{n}-d{dbar:g}-g{gamma:g}-seed{seed}",
                 dict(kind="chung_lu", dbar=dbar, gamma=gamma, seed=seed, max_weight=wmax.value))


def erdos_renyi(n: int, p: float, seed: int = 1, permute: bool = False) -> Graph:
    """G(n, p) random graph."""
    rp, cp, nnz = _out()
    rc = _load().gg_erdos_renyi(n, float(p), seed, int(permute), ctypes.byref(rp), ctypes.byref(cp),
                                ctypes.byref(nnz))
    return _take(rc, n, rp, cp, nnz, f"er-n{n}-p{p:g}-seed{seed}", dict(kind="er", p=p, seed=seed))


# ---------------- small structured graphs (closed-form test cases) ----------------

def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def complete_multipartite(parts) -> Graph:
    owner = []
    for pi, s in enumerate(parts):
        owner += [pi] * s
    n = len(owner)
    e = [(i, j) for i in range(n) for j in range(i + 1, n) if owner[i] != owner[j]]
    return from_edges(n, e, "K_" + ",".join(map(str, parts)))


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"C{n}")


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"P{n}")


def star(leaves: int) -> Graph:
    return from_edges(leaves + 1, [(0, i) for i in range(1, leaves + 1)], f"S{leaves}")


def petersen() -> Graph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return from_edges(10, outer + spokes + inner, "petersen")


def empty(n: int) -> Graph:
    return from_edges(n, np.zeros((0, 2), dtype=np.int64), f"E{n}")


def random_small(n: int, p: float, seed: int) -> Graph:
    """Dense-ish G(n,p) with a random vertex labelling, for brute-force parity cases."""
    g = erdos_renyi(n, p, seed=seed, permute=True)
    g.name = f"gnp-n{n}-p{p:g}-s{seed}"
    return g


# ---------------- the benchmark workloads ----------------

def workload_tc_rmat14() -> Graph:
    """Triangle counting input: R-MAT scale 14, edge factor 16, (0.57,0.19,0.19,0.05), seed 1."""
    return rmat(14, 16.0, (0.57, 0.19, 0.19, 0.05), seed=1)


def workload_clique_rmat21() -> Graph:
    """k-clique input: R-MAT scale 21, edge factor 16, (0.57,0.19,0.19,0.05), seed 2."""
    return rmat(21, 16.0, (0.57, 0.19, 0.19, 0.05), seed=2)


def workload_clique6_rmat20() -> Graph:
    """Large-k clique input: R-MAT scale 20, edge factor 16, (0.57,0.19,0.19,0.05), seed 2."""
    return rmat(20, 16.0, (0.57, 0.19, 0.19, 0.05), seed=2)


def workload_clique789_chung_lu1m() -> Graph:
    """Large-k clique input (k = 7, 8, 9): Chung-Lu, 1,048,576 vertices, mean degree 24, exponent 2.1, seed 3."""
    return chung_lu(1 << 20, 24.0, 2.1, seed=3)


def workload_sl_chung_lu4m() -> Graph:
    """Subgraph-listing input: Chung-Lu, 4,194,304 vertices, mean degree 24, exponent 2.1, seed 3."""
    return chung_lu(1 << 22, 24.0, 2.1, seed=3)


def workload_motif5_er1m() -> Graph:
    """5-vertex motif input: Erdos-Renyi G(n, p), n = 1,048,576, mean degree 8 (p = 8 / (n - 1)), seed 7,
    ids permuted."""
    n = 1 << 20
    return erdos_renyi(n, 8.0 / (n - 1), seed=7, permute=True)


def batch_query_specs(nq: int = 512, base_seed: int = 1000, log2n_range=(10, 20), dbar_range=(8.0, 64.0)):
    """Seeded descriptions of the mixed 3-/4-motif batch.

    Query i: graph type ER or R-MAT (50/50), motif size 3 or 4 (50/50),
    log2(n) uniform in log2n_range (integral for R-MAT), mean degree
    log-uniform in dbar_range; p = dbar/(n-1) for ER, edge factor dbar/2 for
    R-MAT; graph seed base_seed + i.
    """
    rng = np.random.Generator(np.random.PCG64(base_seed))
    specs = []
    for i in range(nq):
        kind = "er" if rng.random() < 0.5 else "rmat"
        k = 3 if rng.random() < 0.5 else 4
        l2 = rng.uniform(log2n_range[0], log2n_range[1])
        dbar = math.exp(rng.uniform(math.log(dbar_range[0]), math.log(dbar_range[1])))
        if kind == "rmat":
            scale = int(round(l2))
            specs.append(dict(kind="rmat", k=k, scale=scale, n=1 << scale, edge_factor=dbar / 2.0,
                              seed=base_seed + i))
        else:
            n = int(round(2.0 ** l2))
            specs.append(dict(kind="er", k=k, n=n, p=min(1.0, dbar / (n - 1)), seed=base_seed + i))
    return specs


def graph_from_spec(s) -> Graph:
    if s["kind"] == "rmat":
        return rmat(s["scale"], s["edge_factor"], (0.57, 0.19, 0.19, 0.05), seed=s["seed"])
    if s["kind"] == "er":
        return erdos_renyi(s["n"], s["p"], seed=s["seed"], permute=True)
    raise ValueError(s)


# ---------------- parallel generation of many graphs ----------------

def _gen_worker(spec):
    from multiprocessing import shared_memory
    g = graph_from_spec(spec)
    shm = shared_memory.SharedMemory(create=True, size=max(1, g.rowptr.nbytes + g.col.nbytes))
    buf = np.ndarray((g.rowptr.nbytes + g.col.nbytes,), dtype=np.uint8, buffer=shm.buf)
    buf[: g.rowptr.nbytes] = g.rowptr.view(np.uint8)
    buf[g.rowptr.nbytes:] = g.col.view(np.uint8)
    name = shm.name
    shm.close()
    return name, g.n, int(g.col.size), g.name


def generate_many(specs, procs: int | None = None):
    """Graphs for a list of specs, generated in a spawn-started process pool.

    Start it before any CUDA work in the calling process (spawn is used, so
    the workers never inherit a CUDA context). Returns Graphs in spec order.
    """
    import multiprocessing as mp
    from multiprocessing import shared_memory
    procs = procs or max(1, min(len(specs), os.cpu_count() or 1))
    out = [None] * len(specs)
    # largest first for balance
    order = sorted(range(len(specs)), key=lambda i: -specs[i].get("n", 0) * specs[i].get("edge_factor", 1.0))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        for i, (name, n, nnz, gname) in zip(order, pool.imap(_gen_worker, [specs[i] for i in order])):
            shm = shared_memory.SharedMemory(name=name)
            try:
                raw = np.ndarray((8 * (n + 1) + 4 * nnz,), dtype=np.uint8, buffer=shm.buf)
                rowptr = raw[: 8 * (n + 1)].view(np.uint64).copy()
                col = raw[8 * (n + 1):].view(np.uint32).copy()
            finally:
                shm.close()
                shm.unlink()
            out[i] = Graph(n, rowptr, col, gname, dict(specs[i]))
    return out
