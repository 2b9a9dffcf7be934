"""Shared helpers of the GPU tests: marshalling between numpy and CUDA tensors."""
import numpy as np

import graphgen as gg


def dev(a, dtype=None):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    t = torch.from_numpy(a).cuda()
    return t if dtype is None else t.to(dtype)


def host(t, dtype=None):
    a = t.cpu().numpy()
    return a if dtype is None else a.view(dtype)


def empty_i32(n):
    import torch
    return torch.empty(max(n, 1), dtype=torch.int32, device="cuda")


def len_tensor():
    import torch
    return torch.zeros(1, dtype=torch.int64, device="cuda")


def pack_keys(dist, pred):
    """key = dist << 32 | (uint32) pred, the SSSP state layout of gr.h."""
    d = np.asarray(dist, dtype=np.uint64)
    p = np.asarray(pred, dtype=np.int64).astype(np.uint32).astype(np.uint64)
    return (d << np.uint64(32)) | p


def unpack_keys(keys):
    k = np.asarray(keys).view(np.uint64)
    return (k >> np.uint64(32)).astype(np.uint32), (k & np.uint64(0xFFFFFFFF)).astype(
        np.uint32).view(np.int32)


def undirected(n, pairs):
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return gg.from_edges(n, pairs[:, 0], pairs[:, 1])


def star_plus(deg):
    """Vertex 0 joined to deg leaves, each leaf joined to a second hub n-1."""
    n = deg + 2
    pairs = [(0, i) for i in range(1, deg + 1)] + [(i, n - 1) for i in range(1, deg + 1, 3)]
    return undirected(n, pairs)
