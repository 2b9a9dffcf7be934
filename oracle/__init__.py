"""CPU oracle for the frontier-traversal hot path (test infrastructure only).

Plain, slow, obviously correct C (``oracle.c``) behind a ctypes wrapper.  Only
the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package; the product library never does, and the two
share no code.  Functions cite the passage of the paper they follow:

* ``bfs``            — Sec. 6.1 (BFS depth / predecessor), FIFO queue BFS.
* ``dijkstra``       — Sec. 3 SSSP example and Alg. 1 (labels, preds, relax on
                       strict improvement), binary-heap Dijkstra with 64-bit keys.
* ``bellman_ford``, ``floyd_warshall`` — brute-force cross-checks.
* ``advance``        — Sec. 4.1: concatenation of neighbour lists in input order.
* ``advance_bfs``, ``advance_relax``, ``pull`` — the fused functors of
                       Sec. 6.1, Alg. 1 and Alg. 2 (Reverse_Advance).
* ``filter_unique``, ``filter_unvisited``, ``filter_near_far`` — Sec. 4.2,
                       Alg. 2 GenerateUnvisitedFrontier, Sec. 5.1.5 near/far.
* ``bfs_certificate``, ``sssp_certificate`` — textbook optimality conditions.
* ``bc_source``, ``bc`` — Sec. 6.3, Brandes' path counts (int64) and dependencies.
* ``cc``             — Sec. 6.4, component labels (smallest vertex id of the component).
* ``segmented_intersect`` — Sec. 4.3, neighbour-list intersections of item pairs.
* ``triangles``      — Sec. 6.6, triangles by their definition (each once, u < v < w).
* ``multisplit``     — Sec. 5.1.5's near/far split generalised to K buckets.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
(closed forms, scipy's independent csgraph routines, brute force, hand-worked
golden graphs); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

INF32 = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile oracle.c (plain -O2, no OpenMP: the oracle is single-threaded)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
            vp = ctypes.c_void_p
            sig = {
                "orc_bfs": ([i32, vp, vp, i32, vp, vp], i64),
                "orc_bfs_min_parent": ([i32, vp, vp, vp, vp], None),
                "orc_dijkstra": ([i32, vp, vp, vp, i32, vp, vp], i32),
                "orc_sssp_min_parent": ([i32, vp, vp, vp, vp, i32, vp], None),
                "orc_bellman_ford": ([i32, vp, vp, vp, i32, vp], None),
                "orc_floyd_warshall": ([i32, vp, vp, vp, vp], None),
                "orc_advance": ([vp, vp, vp, i64, i32, vp, i64], i64),
                "orc_advance_bfs": ([vp, vp, vp, i64, i32, vp, vp, vp], i64),
                "orc_pull": ([vp, vp, vp, i64, i32, vp, vp, vp, vp, vp], i64),
                "orc_advance_relax": ([i32, vp, vp, vp, vp, i64, vp, vp, vp], i64),
                "orc_filter_unique": ([i32, vp, i64, vp], i64),
                "orc_filter_unvisited": ([i32, vp, vp], i64),
                "orc_filter_near_far": ([i32, vp, i64, vp, u32, vp, vp, vp], i64),
                "orc_bfs_certificate": ([i32, vp, vp, i32, vp, vp], i32),
                "orc_sssp_certificate": ([i32, vp, vp, vp, i32, vp, vp], i32),
                "orc_bfs_multi": ([i32, vp, vp, vp, i32, vp], i32),
                "orc_bc_source": ([i32, vp, vp, i32, vp, vp, vp], i32),
                "orc_bc": ([i32, vp, vp, vp, i32, vp], i32),
                "orc_cc": ([i32, vp, vp, vp], i64),
                "orc_segmented_intersect": ([vp, vp, vp, vp, i64, vp, vp, i64], i64),
                "orc_triangles": ([i32, vp, vp, vp], i64),
                "orc_multisplit": ([i32, vp, i64, vp, u32, u32, i32, vp, vp], i64),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def bfs(R, C, src: int):
    """Queue BFS (Sec. 6.1).  Returns (depth, pred) int32 arrays; -1 = unreachable."""
    R, C = _i32(R), _i32(C)
    n = len(R) - 1
    depth = np.empty(n, np.int32)
    pred = np.empty(n, np.int32)
    if _load().orc_bfs(n, _p(R), _p(C), src, _p(depth), _p(pred)) < 0:
        raise ValueError("bad BFS arguments")
    return depth, pred


def bfs_min_parent(R, C, depth):
    """Smallest-id parent one level up for every reached vertex (canonical BFS tree)."""
    R, C, depth = _i32(R), _i32(C), _i32(depth)
    pred = np.empty(len(R) - 1, np.int32)
    _load().orc_bfs_min_parent(len(R) - 1, _p(R), _p(C), _p(depth), _p(pred))
    return pred


def dijkstra(R, C, W, src: int):
    """Binary-heap Dijkstra (Alg. 1 semantics).  Returns (dist uint32, pred int32, overflow)."""
    R, C, W = _i32(R), _i32(C), _u32(W)
    n = len(R) - 1
    dist = np.empty(n, np.uint32)
    pred = np.empty(n, np.int32)
    rc = _load().orc_dijkstra(n, _p(R), _p(C), _p(W), src, _p(dist), _p(pred))
    if rc < 0:
        raise ValueError("bad SSSP arguments")
    return dist, pred, bool(rc)


def sssp_min_parent(R, C, W, dist, src: int):
    """Smallest-id tight predecessor for every reached vertex (canonical SSSP tree)."""
    R, C, W, dist = _i32(R), _i32(C), _u32(W), _u32(dist)
    pred = np.empty(len(R) - 1, np.int32)
    _load().orc_sssp_min_parent(len(R) - 1, _p(R), _p(C), _p(W), _p(dist), src, _p(pred))
    return pred


def bellman_ford(R, C, W, src: int):
    """Bellman-Ford distances as uint64 (2**64-1 = unreachable); W None = unit weights."""
    R, C = _i32(R), _i32(C)
    W = None if W is None else _u32(W)
    n = len(R) - 1
    d = np.empty(n, np.uint64)
    _load().orc_bellman_ford(n, _p(R), _p(C), _p(W), src, _p(d))
    return d


def floyd_warshall(R, C, W=None):
    """All-pairs distances (n x n uint64, 2**64-1 = no path); W None = unit weights."""
    R, C = _i32(R), _i32(C)
    W = None if W is None else _u32(W)
    n = len(R) - 1
    D = np.empty((n, n), np.uint64)
    _load().orc_floyd_warshall(n, _p(R), _p(C), _p(W), _p(D))
    return D


def advance(R, C, frontier, edge_ids: bool = False):
    """Concatenated neighbour lists (V->V) or edge ids (V->E) in input order (Sec. 4.1)."""
    R, C, F = _i32(R), _i32(C), _i32(frontier)
    total = int(np.sum(R[F + 1].astype(np.int64) - R[F])) if len(F) else 0
    out = np.empty(max(total, 1), np.int32)
    k = _load().orc_advance(_p(R), _p(C), _p(F), len(F), int(edge_ids), _p(out), total)
    return out[:k].copy()


def advance_bfs(R, C, frontier, level: int, depth, pred):
    """Push advance with the BFS visit functor; updates depth/pred copies, returns (out, depth, pred)."""
    R, C, F = _i32(R), _i32(C), _i32(frontier)
    depth = _i32(depth).copy()
    pred = _i32(pred).copy()
    out = np.empty(max(len(depth), 1), np.int32)
    k = _load().orc_advance_bfs(_p(R), _p(C), _p(F), len(F), level, _p(depth), _p(pred), _p(out))
    return out[:k].copy(), depth, pred


def pull(R, C, candidates, level: int, depth, pred):
    """Pull step (Alg. 2 Reverse_Advance).  Returns (active, unvisited, depth, pred)."""
    R, C, F = _i32(R), _i32(C), _i32(candidates)
    depth = _i32(depth).copy()
    pred = _i32(pred).copy()
    act = np.empty(max(len(F), 1), np.int32)
    unv = np.empty(max(len(F), 1), np.int32)
    nu = ctypes.c_int64()
    na = _load().orc_pull(_p(R), _p(C), _p(F), len(F), level, _p(depth), _p(pred), _p(act),
                          _p(unv), ctypes.byref(nu))
    return act[:na].copy(), unv[:nu.value].copy(), depth, pred


def advance_relax(R, C, W, frontier, dist, pred):
    """Jacobi relax step (Alg. 1 Update_Label/Set_Pred).  Returns (improved, dist, pred)."""
    R, C, W, F = _i32(R), _i32(C), _u32(W), _i32(frontier)
    n = len(R) - 1
    dist = _u32(dist).copy()
    pred = _i32(pred).copy()
    out = np.empty(max(n, 1), np.int32)
    k = _load().orc_advance_relax(n, _p(R), _p(C), _p(W), _p(F), len(F), _p(dist), _p(pred),
                                  _p(out))
    if k == -1:
        raise OverflowError("distance does not fit below UINT32_MAX")
    return out[:k].copy(), dist, pred


def filter_unique(n: int, items):
    """Exact filter: first occurrence of each item in [0, n), input order kept."""
    a = _i32(items)
    out = np.empty(max(len(a), 1), np.int32)
    k = _load().orc_filter_unique(n, _p(a), len(a), _p(out))
    return out[:k].copy()


def filter_unvisited(depth):
    """Unvisited frontier: ascending ids with depth == -1."""
    d = _i32(depth)
    out = np.empty(max(len(d), 1), np.int32)
    k = _load().orc_filter_unvisited(len(d), _p(d), _p(out))
    return out[:k].copy()


def filter_near_far(n: int, items, dist, threshold: int):
    """Stable split by dist < threshold.  Returns (near, far)."""
    a, d = _i32(items), _u32(dist)
    near = np.empty(max(len(a), 1), np.int32)
    far = np.empty(max(len(a), 1), np.int32)
    fl = ctypes.c_int64()
    k = _load().orc_filter_near_far(n, _p(a), len(a), _p(d), threshold, _p(near), _p(far),
                                    ctypes.byref(fl))
    return near[:k].copy(), far[:fl.value].copy()


def bfs_certificate(R, C, src: int, depth, pred=None) -> int:
    """0 if (depth, pred) is a valid BFS answer, else the code of the first violated rule."""
    R, C, depth = _i32(R), _i32(C), _i32(depth)
    pred = None if pred is None else _i32(pred)
    return int(_load().orc_bfs_certificate(len(R) - 1, _p(R), _p(C), src, _p(depth), _p(pred)))


def sssp_certificate(R, C, W, src: int, dist, pred=None) -> int:
    """0 if (dist, pred) is a valid SSSP answer, else the code of the first violated rule."""
    R, C, W, dist = _i32(R), _i32(C), _u32(W), _u32(dist)
    pred = None if pred is None else _i32(pred)
    return int(_load().orc_sssp_certificate(len(R) - 1, _p(R), _p(C), _p(W), src, _p(dist),
                                            _p(pred)))


def bfs_multi(R, C, srcs):
    """k independent queue-BFS depth arrays, shape (k, n)."""
    R, C, S = _i32(R), _i32(C), _i32(srcs)
    n = len(R) - 1
    depth = np.empty((len(S), n), np.int32)
    if _load().orc_bfs_multi(n, _p(R), _p(C), _p(S), len(S), _p(depth)) < 0:
        raise ValueError("bad multi-source BFS arguments")
    return depth


def bc_source(R, C, src: int):
    """Brandes' single-source pass (Sec. 6.3).  Returns (depth int32, sigma int64,
    delta float64, overflow); sigma counts shortest paths, delta is the dependency."""
    R, C = _i32(R), _i32(C)
    n = len(R) - 1
    depth = np.empty(n, np.int32)
    sigma = np.empty(n, np.int64)
    delta = np.empty(n, np.float64)
    rc = _load().orc_bc_source(n, _p(R), _p(C), src, _p(depth), _p(sigma), _p(delta))
    if rc < 0:
        raise ValueError("bad BC arguments")
    return depth, sigma, delta, bool(rc)


def bc(R, C, srcs):
    """Betweenness centrality over the given sources (ordered pairs): float64 array."""
    R, C, S = _i32(R), _i32(C), _i32(srcs)
    n = len(R) - 1
    out = np.empty(n, np.float64)
    rc = _load().orc_bc(n, _p(R), _p(C), _p(S), len(S), _p(out))
    if rc < 0:
        raise ValueError("bad BC arguments")
    if rc > 0:
        raise OverflowError("a shortest-path count exceeds INT64_MAX")
    return out


def cc(R, C):
    """Component labels (smallest vertex id of each component) and the component count."""
    R, C = _i32(R), _i32(C)
    n = len(R) - 1
    label = np.empty(max(n, 1), np.int32)
    k = _load().orc_cc(n, _p(R), _p(C), _p(label))
    if k < 0:
        raise MemoryError("oracle CC")
    return label[:n].copy(), int(k)


def segmented_intersect(R, C, a, b, items: bool = True):
    """Per-pair intersection sizes of N(a[i]) and N(b[i]) and, with items, the
    intersections concatenated in pair order.  Returns (counts int64, items or None, total)."""
    R, C, A, B = _i32(R), _i32(C), _i32(a), _i32(b)
    counts = np.empty(max(len(A), 1), np.int64)
    lib = _load()
    total = lib.orc_segmented_intersect(_p(R), _p(C), _p(A), _p(B), len(A), _p(counts), None, 0)
    out = None
    if items:
        out = np.empty(max(total, 1), np.int32)
        lib.orc_segmented_intersect(_p(R), _p(C), _p(A), _p(B), len(A), _p(counts), _p(out),
                                    total)
        out = out[:total].copy()
    return counts[:len(A)].copy(), out, int(total)


def triangles(R, C):
    """(total triangles, per-vertex triangle counts int64) of an undirected graph."""
    R, C = _i32(R), _i32(C)
    n = len(R) - 1
    per = np.empty(max(n, 1), np.int64)
    t = _load().orc_triangles(n, _p(R), _p(C), _p(per))
    if t < 0:
        raise MemoryError("oracle triangles")
    return int(t), per[:n].copy()


def multisplit(n: int, items, dist, base: int, delta: int, K: int):
    """Stable K-way split by bucket min(K-1, (dist - base) // delta) (0 below base).
    Returns (items by bucket, bucket lengths int64[K])."""
    a, d = _i32(items), _u32(dist)
    out = np.empty(max(len(a), 1), np.int32)
    bl = np.empty(K, np.int64)
    w = _load().orc_multisplit(n, _p(a), len(a), _p(d), base, delta, K, _p(out), _p(bl))
    return out[:w].copy(), bl
