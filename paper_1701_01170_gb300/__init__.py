"""Python binding of the GB300 frontier-traversal library (include/gr.h).

Argument marshalling only: every function below forwards to the entry point
of the same name in libgr.so (plain device pointers, sizes and a
cudaStream_t); all traversal work runs in the library's CUDA kernels.  There
is no CPU fallback: if libgr.so is missing or fails to load, importing the
library raises.

Device memory and streams come from PyTorch tensors; a tensor argument must
be a contiguous CUDA tensor of the dtype stated in gr.h.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

c_i32, c_i64, c_u32, c_f32, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                    ctypes.c_float, ctypes.c_void_p)

# status codes (gr.h)
GR_OK = 0
GR_ERR_INVALID_ARG = -1
GR_ERR_OOM = -2
GR_ERR_CUDA = -3
GR_ERR_CAPACITY = -4
GR_ERR_OVERFLOW = -5
GR_ERR_TIMEOUT = -6
GR_ERR_INVALID_GRAPH = -7
GR_ERR_UNSUPPORTED = -8
GR_INF_DIST = 0xFFFFFFFF

GR_BORROW, GR_COPY, GR_SYMMETRIC = 0, 1, 2
GR_OP_BFS, GR_OP_SSSP = 1, 2
GR_V2V, GR_V2E, GR_PUSH, GR_PULL, GR_ORDERED, GR_UNORDERED, GR_IDEMPOTENT = 0, 1, 0, 2, 0, 4, 8
GR_FN_NONE, GR_FN_BFS_VISIT, GR_FN_SSSP_RELAX = 0, 1, 2
GR_FILTER_EXACT_UNIQUE, GR_FILTER_CULL, GR_FILTER_UNVISITED, GR_FILTER_NEAR_FAR = 0, 1, 2, 3
GR_FILTER_MULTISPLIT = 4
GR_DIR_AUTO, GR_DIR_PUSH, GR_DIR_PULL = 0, 1, 2


class gr_bfs_opts(ctypes.Structure):
    _fields_ = [("direction", c_i32), ("do_a", c_f32), ("do_b", c_f32), ("big_degree", c_i32),
                ("blocks_per_sm", c_i32), ("spin_limit", c_u32), ("ws", c_vp),
                ("level_stats", c_vp), ("max_levels", c_i32), ("max_blocks", c_i32),
                ("bulk_edges", c_i64)]


class gr_sssp_opts(ctypes.Structure):
    _fields_ = [("delta", c_u32), ("big_degree", c_i32), ("blocks_per_sm", c_i32),
                ("spin_limit", c_u32), ("ws", c_vp), ("level_stats", c_vp), ("max_levels", c_i32),
                ("bulk_rows", c_i32), ("max_blocks", c_i32), ("levels", c_i32)]


class gr_bfs_state(ctypes.Structure):
    _fields_ = [("depth", c_vp), ("pred", c_vp), ("level", c_i32)]


class gr_sssp_state(ctypes.Structure):
    _fields_ = [("key", c_vp), ("threshold", c_u32)]


class gr_multisplit_state(ctypes.Structure):
    _fields_ = [("key", c_vp), ("base", c_u32), ("delta", c_u32), ("buckets", c_i32),
                ("bucket_len", c_vp)]


class gr_msbfs_opts(ctypes.Structure):
    _fields_ = [("direction", c_i32), ("push_ratio", c_f32), ("snapshot_levels", c_i32)]


class gr_job(ctypes.Structure):
    _fields_ = [("g", c_vp), ("op", c_i32), ("src", c_i32), ("out", c_vp), ("pred", c_vp),
                ("do_a", c_f32), ("do_b", c_f32), ("big_degree", c_i32), ("delta", c_u32)]


class gr_batch_opts(ctypes.Structure):
    _fields_ = [("cluster_size", c_i32), ("clusters_per_sm", c_i32), ("use_graph", c_i32),
                ("spin_limit", c_u32)]


class gr_bc_opts(ctypes.Structure):
    _fields_ = [("big_degree", c_i32), ("blocks_per_sm", c_i32), ("spin_limit", c_u32),
                ("ws", c_vp)]


class gr_cc_opts(ctypes.Structure):
    _fields_ = [("big_degree", c_i32), ("blocks_per_sm", c_i32), ("spin_limit", c_u32),
                ("ws", c_vp)]


class gr_run_stats(ctypes.Structure):
    _fields_ = [("levels", c_i32), ("reserved", c_i32), ("edges", c_i64), ("vertices", c_i64),
                ("updates", c_i64)]


class GrError(RuntimeError):
    """A non-GR_OK status from the library."""

    def __init__(self, status: int, where: str = ""):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


_lib = None

_SIGNATURES = {
    "gr_status_str": ([c_i32], ctypes.c_char_p),
    "gr_version": ([], c_i32),
    "gr_graph_create_csr": ([c_i32, c_i64, c_vp, c_vp, c_vp, c_u32, c_vp,
                             ctypes.POINTER(c_vp)], c_i32),
    "gr_graph_destroy": ([c_vp], c_i32),
    "gr_graph_info": ([c_vp, c_vp, c_vp, c_vp, c_vp], c_i32),
    "gr_graph_footprint": ([c_vp, c_i32, ctypes.POINTER(ctypes.c_size_t)], c_i32),
    "gr_workspace_create": ([c_vp, c_i32, ctypes.POINTER(c_vp)], c_i32),
    "gr_workspace_destroy": ([c_vp], c_i32),
    "gr_workspace_create_async": ([c_vp, c_i32, c_vp, ctypes.POINTER(c_vp)], c_i32),
    "gr_workspace_destroy_async": ([c_vp, c_vp], c_i32),
    "gr_sync_status": ([c_vp, c_vp, c_vp], c_i32),
    "gr_last_run_stats": ([c_vp, c_vp, ctypes.POINTER(gr_run_stats), c_vp], c_i32),
    "gr_advance": ([c_vp, c_vp, c_i64, c_vp, c_i32, c_i32, c_vp, c_vp, c_i64, c_vp, c_vp], c_i32),
    "gr_filter": ([c_vp, c_vp, c_i64, c_vp, c_i32, c_vp, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp,
                   c_vp], c_i32),
    "gr_bfs_opts_default": ([ctypes.POINTER(gr_bfs_opts)], None),
    "gr_bfs": ([c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(gr_bfs_opts), c_vp], c_i32),
    "gr_sssp_opts_default": ([ctypes.POINTER(gr_sssp_opts)], None),
    "gr_sssp": ([c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(gr_sssp_opts), c_vp], c_i32),
    "gr_msbfs_opts_default": ([ctypes.POINTER(gr_msbfs_opts)], None),
    "gr_bfs_multi": ([c_vp, c_vp, c_i32, c_vp, ctypes.POINTER(gr_msbfs_opts), c_vp], c_i32),
    "gr_batch_opts_default": ([ctypes.POINTER(gr_batch_opts)], None),
    "gr_batch_create": ([c_vp, c_i32, ctypes.POINTER(gr_batch_opts), ctypes.POINTER(c_vp)], c_i32),
    "gr_batch_run": ([c_vp, c_vp], c_i32),
    "gr_batch_status": ([c_vp, c_vp, c_vp], c_i32),
    "gr_batch_info": ([c_vp, c_vp, c_vp, c_vp], c_i32),
    "gr_batch_destroy": ([c_vp], c_i32),
    "gr_bfs_static": ([c_i32, c_i64, c_vp, c_vp, c_u32, c_i32, c_vp, c_vp, c_vp, c_vp], c_i32),
    "gr_bc_opts_default": ([ctypes.POINTER(gr_bc_opts)], None),
    "gr_bc": ([c_vp, c_i32, c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(gr_bc_opts), c_vp], c_i32),
    "gr_cc_opts_default": ([ctypes.POINTER(gr_cc_opts)], None),
    "gr_cc": ([c_vp, c_vp, c_vp, ctypes.POINTER(gr_cc_opts), c_vp], c_i32),
    "gr_segmented_intersect": ([c_vp, c_vp, c_vp, c_i64, c_vp, c_vp, c_vp, c_i64, c_vp, c_vp,
                                c_vp], c_i32),
    "gr_triangle_count": ([c_vp, c_vp, c_vp, c_vp, c_vp], c_i32),
}
GR_STATIC_MAX_VERTICES = 1 << 20
GR_STATIC_MAX_EDGES = 1 << 25


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgr.so (raises if it is absent; never falls back to other code)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("GR_LIBRARY", _build.LIB)   # an alternative build of libgr.so
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    missing = [name for name in _SIGNATURES if not hasattr(lib, name)]
    if missing:
        raise RuntimeError(f"{path} does not export {', '.join(missing)}: rebuild it")
    for name, (args, res) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_str(s: int) -> str:
    return load().gr_status_str(s).decode()


def _check(st: int, where: str):
    if st != GR_OK:
        raise GrError(st, where)


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (or an int address / None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return c_vp(t)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return c_vp(t.data_ptr())


def _buf32(t, count: int, what: str):
    """Device pointer of a 4-byte-element CUDA tensor holding at least `count` elements.

    The kernels write `count` 32-bit values through the pointer, so a smaller
    or narrower tensor is rejected here instead of being overrun on the
    device.  An int (a raw device address) is passed through unchecked.
    """
    if t is None or isinstance(t, int):
        return _ptr(t)
    if t.element_size() != 4:
        raise ValueError(f"{what}: expected a 32-bit tensor, got {t.dtype}")
    if t.numel() < count:
        raise ValueError(f"{what}: needs {count} elements, the tensor has {t.numel()}")
    return _ptr(t)


def _graph_n(g) -> int:
    n = c_i32()
    _check(load().gr_graph_info(c_vp(g), ctypes.byref(n), None, None, None), "gr_graph_info")
    return n.value


def _stream(stream):
    import torch
    if stream is None:
        return c_vp(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return c_vp(stream)
    return c_vp(stream.cuda_stream)


# ---- entry points (same names as gr.h) ------------------------------------

def gr_version() -> int:
    return load().gr_version()


def gr_graph_create_csr(n, m, row_offsets, cols, weights=None, flags=0, stream=None):
    """Returns an opaque graph handle (int).  row_offsets/cols/weights: CUDA tensors."""
    h = c_vp()
    st = load().gr_graph_create_csr(n, m, _ptr(row_offsets), _ptr(cols), _ptr(weights), flags,
                                    _stream(stream), ctypes.byref(h))
    _check(st, "gr_graph_create_csr")
    return h.value


def gr_graph_destroy(g):
    _check(load().gr_graph_destroy(c_vp(g)), "gr_graph_destroy")


def gr_graph_info(g):
    n, m, fl, md = c_i32(), c_i64(), c_u32(), c_i32()
    _check(load().gr_graph_info(c_vp(g), ctypes.byref(n), ctypes.byref(m), ctypes.byref(fl),
                                ctypes.byref(md)), "gr_graph_info")
    return {"n": n.value, "m": m.value, "flags": fl.value, "max_degree": md.value}


def gr_graph_footprint(g, op) -> int:
    b = ctypes.c_size_t()
    _check(load().gr_graph_footprint(c_vp(g), op, ctypes.byref(b)), "gr_graph_footprint")
    return b.value


def gr_workspace_create(g, ops=GR_OP_BFS | GR_OP_SSSP):
    h = c_vp()
    _check(load().gr_workspace_create(c_vp(g), ops, ctypes.byref(h)), "gr_workspace_create")
    return h.value


def gr_workspace_destroy(ws):
    _check(load().gr_workspace_destroy(c_vp(ws)), "gr_workspace_destroy")


def gr_workspace_create_async(g, ops=GR_OP_BFS | GR_OP_SSSP, stream=None):
    """Stream-ordered workspace: allocated and initialised on `stream`, no device wait."""
    h = c_vp()
    _check(load().gr_workspace_create_async(c_vp(g), ops, _stream(stream), ctypes.byref(h)),
           "gr_workspace_create_async")
    return h.value


def gr_workspace_destroy_async(ws, stream=None):
    """Release a stream-ordered workspace after the work queued on `stream`."""
    _check(load().gr_workspace_destroy_async(c_vp(ws), _stream(stream)),
           "gr_workspace_destroy_async")


def gr_sync_status(g, ws=None, stream=None) -> int:
    """Device-detected status since the last call (0 = GR_OK); does not raise."""
    return load().gr_sync_status(c_vp(g), c_vp(ws) if ws else None, _stream(stream))


def gr_last_run_stats(g, ws=None, stream=None) -> dict:
    """Counters of the last BFS / SSSP run on a workspace (synchronous)."""
    st = gr_run_stats()
    _check(load().gr_last_run_stats(c_vp(g), c_vp(ws) if ws else None, ctypes.byref(st),
                                    _stream(stream)), "gr_last_run_stats")
    return {"levels": st.levels, "edges": st.edges, "vertices": st.vertices,
            "updates": st.updates}


def gr_advance(g, inp, in_len, out, out_len, mode=0, functor=GR_FN_NONE, state=None,
               in_len_dev=None, out_cap=None, stream=None):
    """One advance step; out_len is a 1-element int64 CUDA tensor (written on device)."""
    cap = out.numel() if out_cap is None and out is not None else (out_cap or 0)
    st = load().gr_advance(c_vp(g), _ptr(inp), in_len, _ptr(in_len_dev), mode, functor,
                           ctypes.byref(state) if state is not None else None, _ptr(out), cap,
                           _ptr(out_len), _stream(stream))
    _check(st, "gr_advance")


def gr_filter(g, inp, in_len, out, out_len, mode=GR_FILTER_EXACT_UNIQUE, state=None,
              far=None, far_len=None, in_len_dev=None, out_cap=None, far_cap=None, stream=None):
    cap = out.numel() if out_cap is None and out is not None else (out_cap or 0)
    fcap = far.numel() if far_cap is None and far is not None else (far_cap or 0)
    st = load().gr_filter(c_vp(g), _ptr(inp), in_len, _ptr(in_len_dev), mode,
                          ctypes.byref(state) if state is not None else None, _ptr(out), cap,
                          _ptr(out_len), _ptr(far), fcap, _ptr(far_len), _stream(stream))
    _check(st, "gr_filter")


def _opts(struct, default_fn: str, kw):
    """The library's defaults for `struct`, then the given fields (unknown names raise)."""
    o = struct()
    getattr(load(), default_fn)(ctypes.byref(o))
    names = {f[0] for f in struct._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"{struct.__name__} has no field {k!r}")
        setattr(o, k, v)
    return o


def bfs_opts(**kw) -> gr_bfs_opts:
    return _opts(gr_bfs_opts, "gr_bfs_opts_default", kw)


def sssp_opts(**kw) -> gr_sssp_opts:
    return _opts(gr_sssp_opts, "gr_sssp_opts_default", kw)


def gr_bfs(g, src, depth, pred=None, opts=None, stream=None):
    n = _graph_n(g)
    st = load().gr_bfs(c_vp(g), src, _buf32(depth, n, "depth"), _buf32(pred, n, "pred"),
                       ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "gr_bfs")


def gr_sssp(g, src, dist, pred=None, opts=None, stream=None):
    n = _graph_n(g)
    st = load().gr_sssp(c_vp(g), src, _buf32(dist, n, "dist"), _buf32(pred, n, "pred"),
                        ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "gr_sssp")


def msbfs_opts(**kw) -> gr_msbfs_opts:
    return _opts(gr_msbfs_opts, "gr_msbfs_opts_default", kw)


def gr_bfs_multi(g, srcs, depth, opts=None, stream=None):
    """k-source bit-parallel BFS; srcs is a host int sequence, depth a CUDA int32 (k*n) tensor."""
    import numpy as np
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    depth_p = _buf32(depth, len(s) * _graph_n(g), "depth")
    st = load().gr_bfs_multi(c_vp(g), s.ctypes.data_as(c_vp), len(s), depth_p,
                             ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "gr_bfs_multi")


def batch_opts(**kw) -> gr_batch_opts:
    return _opts(gr_batch_opts, "gr_batch_opts_default", kw)


def gr_batch_create(jobs, opts=None):
    """jobs: a sequence of gr_job structures.  Returns an opaque batch handle."""
    arr = (gr_job * len(jobs))(*jobs)
    h = c_vp()
    _check(load().gr_batch_create(ctypes.cast(arr, c_vp), len(jobs),
                                  ctypes.byref(opts) if opts is not None else None,
                                  ctypes.byref(h)), "gr_batch_create")
    return h.value


def gr_batch_run(b, stream=None):
    _check(load().gr_batch_run(c_vp(b), _stream(stream)), "gr_batch_run")


def gr_batch_status(b, njobs=None, stream=None):
    """(first error code, per-job status list or None)."""
    import numpy as np
    arr = None if njobs is None else np.zeros(njobs, np.int32)
    st = load().gr_batch_status(c_vp(b), arr.ctypes.data_as(c_vp) if arr is not None else None,
                                _stream(stream))
    return st, (None if arr is None else arr.tolist())


def gr_batch_info(b):
    c, cs, sb = c_i32(), c_i32(), ctypes.c_size_t()
    _check(load().gr_batch_info(c_vp(b), ctypes.byref(c), ctypes.byref(cs), ctypes.byref(sb)),
           "gr_batch_info")
    return {"clusters": c.value, "cluster_size": cs.value, "scratch_bytes": sb.value}


def gr_batch_destroy(b):
    _check(load().gr_batch_destroy(c_vp(b)), "gr_batch_destroy")


def bc_opts(**kw) -> gr_bc_opts:
    return _opts(gr_bc_opts, "gr_bc_opts_default", kw)


def _buf(t, count: int, size: int, what: str):
    """Device pointer of a CUDA tensor of `size`-byte elements holding at least `count`."""
    if t is None or isinstance(t, int):
        return _ptr(t)
    if t.element_size() != size:
        raise ValueError(f"{what}: expected {8 * size}-bit elements, got {t.dtype}")
    if t.numel() < count:
        raise ValueError(f"{what}: needs {count} elements, the tensor has {t.numel()}")
    return _ptr(t)


def gr_bc(g, src, depth=None, sigma=None, delta=None, bc=None, opts=None, stream=None):
    """Brandes' pass for one source: depth int32, sigma int64, delta float64 (each n or
    None) and bc float64 (n, accumulated) are CUDA tensors."""
    n = _graph_n(g)
    st = load().gr_bc(c_vp(g), src, _buf(depth, n, 4, "depth"), _buf(sigma, n, 8, "sigma"),
                      _buf(delta, n, 8, "delta"), _buf(bc, n, 8, "bc"),
                      ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "gr_bc")


def cc_opts(**kw) -> gr_cc_opts:
    return _opts(gr_cc_opts, "gr_cc_opts_default", kw)


def gr_cc(g, comp, num_components=None, opts=None, stream=None):
    """Component labels (smallest vertex id per component) into comp (int32, n); the
    component count into num_components (a 1-element int32 CUDA tensor) if given."""
    n = _graph_n(g)
    st = load().gr_cc(c_vp(g), _buf(comp, n, 4, "comp"), _buf(num_components, 1, 4, "count"),
                      ctypes.byref(opts) if opts is not None else None, _stream(stream))
    _check(st, "gr_cc")


def gr_segmented_intersect(g, a, b, length, counts=None, total=None, out=None, out_len=None,
                           out_cap=None, ws=None, stream=None):
    """Per-pair neighbour-list intersections; a, b int32 CUDA tensors, counts int64 (length),
    total / out_len 1-element int64 tensors, out int32 tensor."""
    cap = out.numel() if out is not None and out_cap is None else (out_cap or 0)
    st = load().gr_segmented_intersect(c_vp(g), _buf(a, length, 4, "a"), _buf(b, length, 4, "b"),
                                       length, _buf(counts, length, 8, "counts"),
                                       _buf(total, 1, 8, "total"), _buf(out, 0, 4, "out"), cap,
                                       _buf(out_len, 1, 8, "out_len"), c_vp(ws) if ws else None,
                                       _stream(stream))
    _check(st, "gr_segmented_intersect")


def gr_triangle_count(g, total, per_vertex=None, ws=None, stream=None):
    """Triangles of a symmetric graph into total (1-element int64 CUDA tensor); optional
    per-vertex counts (int64, n)."""
    n = _graph_n(g)
    st = load().gr_triangle_count(c_vp(g), _buf(total, 1, 8, "total"),
                                  _buf(per_vertex, n, 8, "per_vertex"), c_vp(ws) if ws else None,
                                  _stream(stream))
    _check(st, "gr_triangle_count")


def gr_bfs_static(n, m, row_offsets, cols, src, depth, pred=None, status=None, flags=0,
                  stream=None):
    """BFS that allocates nothing: scratch lives in the library's static device array.

    For callers that may not allocate device memory at call time (allocator
    callbacks, latency-critical threads, runtimes owning all device memory).
    Calls share that array, so they must not overlap on the GPU.
    """
    st = load().gr_bfs_static(n, m, _ptr(row_offsets), _ptr(cols), flags, src, _ptr(depth),
                              _ptr(pred), _ptr(status), _stream(stream))
    _check(st, "gr_bfs_static")


# ---- convenience: a graph resident in device memory ------------------------

class Graph:
    """A device-resident CSR graph plus its library handle.

    Holds the device tensors (the handle borrows them) so that they live as
    long as the handle.  `csr` is any object with int32 numpy arrays R, C and
    optionally uint32 W (e.g. graphgen.CSR).
    """

    def __init__(self, R, C, W=None, symmetric=True, device="cuda", stream=None):
        import numpy as np
        import torch
        self.n = int(len(R) - 1)
        self.m = int(len(C))
        self.R = torch.from_numpy(np.ascontiguousarray(R, dtype=np.int32)).to(device)
        self.C = torch.from_numpy(np.ascontiguousarray(C, dtype=np.int32)).to(device)
        self.W = None
        if W is not None:
            w = np.ascontiguousarray(W, dtype=np.uint32).view(np.int32)
            self.W = torch.from_numpy(w).to(device)
        torch.cuda.synchronize()
        flags = GR_SYMMETRIC if symmetric else 0
        self.handle = gr_graph_create_csr(self.n, self.m, self.R, self.C, self.W, flags, stream)

    @classmethod
    def from_csr(cls, csr, symmetric=True, **kw):
        return cls(csr.R, csr.C, getattr(csr, "W", None), symmetric=symmetric, **kw)

    def info(self):
        return gr_graph_info(self.handle)

    def sync_status(self, ws=None, stream=None) -> int:
        return gr_sync_status(self.handle, ws, stream)

    def close(self):
        if getattr(self, "handle", None):
            gr_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass
