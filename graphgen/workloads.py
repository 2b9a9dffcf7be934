"""Named synthetic workloads built from the generators (inputs only, no traversal arithmetic).

* ``batch_graphs`` / ``batch_jobs``: many uneven R-MAT graphs with a job
  list of BFS/SSSP queries, 50/50 — the batched configuration.
* ``serving_graphs``: the resident graph set of the serving configuration.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import CSR, grid_weighted, rmat_weighted, sources

OP_BFS, OP_SSSP = 1, 2


@dataclass
class BatchGraph:
    scale: int
    ef: int
    seed: int
    csr: CSR


def batch_graphs(count: int = 64, seed: int = 5, scale_lo: int = 10, scale_hi: int = 18,
                 ef_lo: int = 8, ef_hi: int = 32, base_seed: int = 1000) -> list[BatchGraph]:
    """`count` R-MAT graphs, scale ~ U{scale_lo..scale_hi}, ef ~ U{ef_lo..ef_hi}, weights U[1,64].

    Graph i uses generator seed base_seed + i; the (scale, ef) draws come from
    numpy's default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    scales = rng.integers(scale_lo, scale_hi + 1, count)
    efs = rng.integers(ef_lo, ef_hi + 1, count)
    out = []
    for i in range(count):
        g = rmat_weighted(int(scales[i]), int(efs[i]), base_seed + i, 1, 64)
        out.append(BatchGraph(int(scales[i]), int(efs[i]), base_seed + i, g))
    return out


def batch_jobs(graphs: list[BatchGraph], njobs: int = 512, seed: int = 5):
    """(graph index, op, source) triples: BFS and SSSP alternate, graphs and sources random."""
    rng = np.random.default_rng(seed + 1)
    picks = rng.integers(0, len(graphs), njobs)
    jobs = []
    per_graph: dict[int, np.ndarray] = {}
    for j in range(njobs):
        gi = int(picks[j])
        if gi not in per_graph:
            per_graph[gi] = sources(graphs[gi].csr, 64, seed=seed * 7919 + gi)
        cand = per_graph[gi]
        src = int(cand[int(rng.integers(0, len(cand)))])
        jobs.append((gi, OP_BFS if j % 2 == 0 else OP_SSSP, src))
    return jobs


def serving_graphs(small: bool = False):
    """The serving set: R-MAT s18/20/22/24 (ef 16, weights U[1,64]) and grids
    1024^2..8192^2 (10 % deletion, weights U[1,1000]).  `small` shrinks every
    graph (scales 12-15, grids 64-512) for tests."""
    if small:
        rm = [(12, 16), (13, 16), (14, 16), (15, 16)]
        gw = [64, 128, 256, 512]
    else:
        rm = [(18, 16), (20, 16), (22, 16), (24, 16)]
        gw = [1024, 2048, 4096, 8192]
    out = []
    for s, ef in rm:
        out.append((f"rmat_s{s}", rmat_weighted(s, ef, 2, 1, 64)))
    for w in gw:
        out.append((f"grid_{w}", grid_weighted(w, 0.1, 3, 1, 1000)))
    return out
