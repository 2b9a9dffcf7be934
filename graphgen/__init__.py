"""Seeded synthetic graph inputs: R-MAT and 2-D grids as CSR, edge weights, sources.

This package only *produces* inputs (it holds none of the traversal
arithmetic); the CPU oracle tests and the CUDA path both consume its arrays.
The recipe follows the paper's dataset rules (Sec. 7, "Datasets"): R-MAT with
edge factor 16 and initiator a=.57, b=.19, c=.19, d=.05; every graph made
undirected with self-loops and duplicate edges removed; weights uniform
integers (1..64 in the paper).

The C source is compiled on first use (gcc, OpenMP) into ``_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_OUT = os.path.join(_HERE, "_build", "libgraphgen.so")
_lock = threading.Lock()
_lib = None

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (idempotent)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u32, u64, dbl = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_double)
            vp = ctypes.c_void_p
            pp = ctypes.POINTER(ctypes.c_void_p)
            lib.gg_rmat.argtypes = [i32, i32, u64, dbl, dbl, dbl, vp, pp]
            lib.gg_rmat.restype = i64
            lib.gg_grid.argtypes = [i32, dbl, u64, vp, pp]
            lib.gg_grid.restype = i64
            lib.gg_from_edges.argtypes = [i32, i64, vp, vp, vp, pp]
            lib.gg_from_edges.restype = i64
            lib.gg_weights.argtypes = [i32, vp, vp, u32, u32, u64, vp]
            lib.gg_weights.restype = None
            lib.gg_sources.argtypes = [i32, vp, i32, u64, vp]
            lib.gg_sources.restype = i32
            lib.gg_free.argtypes = [vp]
            lib.gg_free.restype = None
            _lib = lib
    return _lib


@dataclass
class CSR:
    """Host CSR graph: int32 row offsets R (n+1), int32 columns C (m), optional uint32 W."""
    R: np.ndarray
    C: np.ndarray
    W: np.ndarray | None = None
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.R.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.C.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.R.astype(np.int64))


def _take_csr(n: int, m: int, R64: np.ndarray, cptr: ctypes.c_void_p, name: str) -> CSR:
    lib = _load()
    if m < 0:
        raise MemoryError("graph generation failed")
    if m >= 2**31:
        lib.gg_free(cptr)
        raise ValueError(f"{name}: m={m} does not fit int32 row offsets")
    C = np.empty(m, dtype=np.int32)
    if m:
        ctypes.memmove(C.ctypes.data, cptr.value, m * 4)
    lib.gg_free(cptr)
    return CSR(R=R64.astype(np.int32), C=C, name=name)


def rmat(scale: int, ef: int = 16, seed: int = 1, abcd=RMAT_ABCD) -> CSR:
    """Undirected R-MAT graph with 2**scale vertices and ef * 2**scale draws."""
    lib = _load()
    n = 1 << scale
    R = np.empty(n + 1, dtype=np.int64)
    cptr = ctypes.c_void_p()
    a, b, c, _ = abcd
    m = lib.gg_rmat(scale, ef, seed, a, b, c, R.ctypes.data, ctypes.byref(cptr))
    return _take_csr(n, m, R, cptr, f"rmat_s{scale}_ef{ef}_seed{seed}")


def grid(W: int, p_del: float = 0.0, seed: int = 3) -> CSR:
    """W x W 4-neighbour grid with each undirected edge deleted with probability p_del."""
    lib = _load()
    n = W * W
    R = np.empty(n + 1, dtype=np.int64)
    cptr = ctypes.c_void_p()
    m = lib.gg_grid(W, float(p_del), seed, R.ctypes.data, ctypes.byref(cptr))
    return _take_csr(n, m, R, cptr, f"grid_{W}x{W}_del{p_del}_seed{seed}")


def from_edges(n: int, src, dst, name: str = "edges") -> CSR:
    """Symmetric, self-loop-free, duplicate-free CSR with sorted rows from an edge list."""
    lib = _load()
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    R = np.empty(n + 1, dtype=np.int64)
    cptr = ctypes.c_void_p()
    m = lib.gg_from_edges(n, len(s), s.ctypes.data, d.ctypes.data, R.ctypes.data,
                          ctypes.byref(cptr))
    if m < 0:
        raise ValueError("edge endpoint out of range")
    return _take_csr(n, m, R, cptr, name)


def directed(n: int, src, dst, name: str = "directed") -> CSR:
    """Directed CSR from (src, dst) pairs; rows sorted, duplicates and self-loops kept."""
    s = np.asarray(src, dtype=np.int64)
    d = np.asarray(dst, dtype=np.int64)
    order = np.lexsort((d, s))
    s, d = s[order], d[order]
    R = np.zeros(n + 1, dtype=np.int64)
    np.add.at(R, s + 1, 1)
    R = np.cumsum(R)
    return CSR(R=R.astype(np.int32), C=d.astype(np.int32), name=name)


def weights(g: CSR, lo: int, hi: int, seed: int) -> np.ndarray:
    """uint32 weights uniform in [lo, hi], symmetric: w(u,v) == w(v,u)."""
    lib = _load()
    R64 = g.R.astype(np.int64)
    W = np.empty(g.m, dtype=np.uint32)
    if g.m:
        lib.gg_weights(g.n, R64.ctypes.data, g.C.ctypes.data, lo, hi, seed, W.ctypes.data)
    return W


def sources(g: CSR, k: int, seed: int) -> np.ndarray:
    """k distinct sources uniform over vertices of degree >= 1 (seeded rejection sampling)."""
    lib = _load()
    R64 = g.R.astype(np.int64)
    out = np.empty(max(k, 1), dtype=np.int32)
    got = lib.gg_sources(g.n, R64.ctypes.data, k, seed, out.ctypes.data)
    return out[:got].copy()


def max_degree_vertex(g: CSR) -> int:
    """Smallest vertex id among those of maximum degree."""
    return int(np.argmax(g.degrees()))


def csr_digest(g: CSR) -> str:
    """Stable content hash of a CSR (for determinism checks and caching)."""
    import hashlib
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.R).tobytes())
    h.update(np.ascontiguousarray(g.C).tobytes())
    if g.W is not None:
        h.update(np.ascontiguousarray(g.W).tobytes())
    return h.hexdigest()[:16]


# ---- the named workloads -------------------------------------------------

def rmat_weighted(scale: int, ef: int = 16, seed: int = 2, wlo: int = 1, whi: int = 64) -> CSR:
    g = rmat(scale, ef, seed)
    g.W = weights(g, wlo, whi, seed)
    return g


def grid_weighted(W: int, p_del: float = 0.1, seed: int = 3, wlo: int = 1, whi: int = 1000) -> CSR:
    g = grid(W, p_del, seed)
    g.W = weights(g, wlo, whi, seed)
    return g
