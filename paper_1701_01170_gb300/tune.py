"""Autotuner for the per-level strategy knobs of BFS, SSSP and batched jobs.

The paper fixes its strategy switches by hand (average degree 5 and frontier
size 4096 choose the load balancer, Sec. 5.1.3; do_a / do_b choose push or
pull, Sec. 5.1.4, whose best values it shows differ per graph).  Here every
knob that changes only speed, never results, is searched by measurement on
the graph at hand and cached by a graph signature:

* BFS: do_a, do_b (Eq. 5-6: when a level goes pull / back to push),
  big_degree (rows at least this long are expanded as edge chunks shared by
  the whole grid instead of by one warp), blocks_per_sm (grid shape).
* SSSP: delta (near/far bucket width, Sec. 5.1.5) and big_degree.
* Batches: cluster size (CTAs that run one job together) and resident
  clusters per SM.

Timing uses CUDA events on the launching stream after warm-up; candidates
are compared on the same sample of sources.
"""
from __future__ import annotations

import json
import os
import statistics
from dataclasses import asdict, dataclass, field

from . import (GR_OP_BFS, GR_OP_SSSP, batch_opts, bfs_opts, gr_batch_create, gr_batch_destroy,
               gr_batch_run, gr_batch_status, gr_bfs, gr_graph_info, gr_sssp, gr_sync_status,
               sssp_opts)

BFS_GRID = {
    "do_a": [0.002, 0.01, 0.05, 0.2],
    "do_b": [0.0, 0.05],
    "big_degree": [64, 256, 1024],
    "blocks_per_sm": [0, 2],
}
SSSP_DELTA_FACTORS = [0.25, 0.5, 1.0, 2.0, 4.0, 8.0]
BATCH_CLUSTERS = [1, 2, 4, 8]


@dataclass
class BfsChoice:
    do_a: float = 0.05
    do_b: float = 0.05
    big_degree: int = 256
    blocks_per_sm: int = 0
    ms: float = float("nan")

    def opts(self, **kw):
        return bfs_opts(do_a=self.do_a, do_b=self.do_b, big_degree=self.big_degree,
                        blocks_per_sm=self.blocks_per_sm, **kw)


@dataclass
class SsspChoice:
    delta: int = 0
    big_degree: int = 1024
    ms: float = float("nan")

    def opts(self, **kw):
        return sssp_opts(delta=self.delta, big_degree=self.big_degree, **kw)


@dataclass
class TuneCache:
    path: str | None = None
    entries: dict = field(default_factory=dict)

    @classmethod
    def load(cls, path: str | None):
        c = cls(path=path)
        if path and os.path.exists(path):
            with open(path) as f:
                c.entries = json.load(f)
        return c

    def save(self):
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def signature(graph_handle) -> str:
    """Graph features the choices depend on: size, density and degree skew."""
    info = gr_graph_info(graph_handle)
    return f"n{info['n']}_m{info['m']}_dmax{info['max_degree']}_f{info['flags']}"


def _time(fn, reps: int, warm: int = 2) -> float:
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        s.record()
        fn()
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def tune_bfs(graph, sources, reps: int = 3, cache: TuneCache | None = None,
             grid: dict | None = None) -> BfsChoice:
    """Pick the fastest BFS knobs over `sources` (results are identical for all)."""
    import itertools

    import torch
    key = "bfs:" + signature(graph.handle)
    if cache and key in cache.entries:
        return BfsChoice(**cache.entries[key])
    grid = grid or BFS_GRID
    depth = torch.empty(graph.n, dtype=torch.int32, device="cuda")
    best = None
    for da, db, bd, bps in itertools.product(grid["do_a"], grid["do_b"], grid["big_degree"],
                                             grid["blocks_per_sm"]):
        if db > da:
            continue
        c = BfsChoice(da, db, bd, bps)
        o = c.opts()

        def run():
            for s in sources:
                gr_bfs(graph.handle, int(s), depth, None, o)

        c.ms = _time(run, reps) / max(1, len(sources))
        if best is None or c.ms < best.ms:
            best = c
    if gr_sync_status(graph.handle) != 0:
        raise RuntimeError("BFS failed while tuning")
    if cache is not None:
        cache.entries[key] = asdict(best)
        cache.save()
    return best


def default_delta(graph) -> int:
    """The library's own default bucket width (256 * mean weight / mean degree)."""
    import numpy as np
    w = graph.W.to(dtype=__import__("torch").int64) & 0xFFFFFFFF
    m = max(graph.m, 1)
    deg = (graph.R[1:] - graph.R[:-1])
    nz = int((deg > 0).sum().item())
    mean_w = float(w.sum().item()) / m
    return max(1, int(256.0 * mean_w / (m / max(nz, 1))))


def tune_sssp(graph, sources, reps: int = 2, cache: TuneCache | None = None,
              factors=None, bigs=(256, 1024)) -> SsspChoice:
    import torch
    key = "sssp:" + signature(graph.handle)
    if cache and key in cache.entries:
        return SsspChoice(**cache.entries[key])
    base = default_delta(graph)
    dist = torch.empty(graph.n, dtype=torch.int32, device="cuda")
    best = None
    for f in factors or SSSP_DELTA_FACTORS:
        for bd in bigs:
            c = SsspChoice(max(1, int(base * f)), bd)
            o = c.opts()

            def run():
                for s in sources:
                    gr_sssp(graph.handle, int(s), dist, None, o)

            c.ms = _time(run, reps, warm=1) / max(1, len(sources))
            if best is None or c.ms < best.ms:
                best = c
    if gr_sync_status(graph.handle) != 0:
        raise RuntimeError("SSSP failed while tuning")
    if cache is not None:
        cache.entries[key] = asdict(best)
        cache.save()
    return best


def tune_batch(jobs, reps: int = 3, clusters=None, per_sm=(0,)) -> tuple[dict, float]:
    """Pick cluster size / residency for a job list (gr_job structures); returns (opts, ms)."""
    best = None
    for cs in clusters or BATCH_CLUSTERS:
        for ps in per_sm:
            try:
                b = gr_batch_create(jobs, batch_opts(cluster_size=cs, clusters_per_sm=ps))
            except RuntimeError:
                continue
            ms = _time(lambda: gr_batch_run(b), reps, warm=1)
            st, _ = gr_batch_status(b)
            gr_batch_destroy(b)
            if st != 0:
                raise RuntimeError(f"batch failed while tuning (status {st})")
            if best is None or ms < best[1]:
                best = ({"cluster_size": cs, "clusters_per_sm": ps}, ms)
    return best


BATCH_BFS_BIG = [64, 256, 1024]
BATCH_BFS_DO = [(0.01, 0.01), (0.05, 0.05), (0.2, 0.05)]
BATCH_SSSP_BIG = [256, 1024, 4096]
BATCH_DELTA_FACTORS = [0.5, 1.0, 2.0]


def tune_batch_strategy(jobs, graphs_by_handle=None, reps: int = 3):
    """Choose the batch's launch shape and per-level strategy by measuring the batch itself.

    Coordinate search, each candidate timed as a whole batch launch: the cluster size (CTAs
    per job), then for the BFS jobs the split threshold (warp batches vs grid-shared edge
    chunks) and the push/pull switch factors (Eq. 5-6), then for the SSSP jobs the split
    threshold and the near/far bucket width (a factor on each graph's default; needs
    `graphs_by_handle`).  The jobs are updated in place with the winners; returns
    (batch opts, ms per launch, chosen settings).  Results do not depend on any of these.
    """
    opts, best_ms = tune_batch(jobs, reps=reps)
    chosen = {"cluster_size": opts["cluster_size"]}

    def measure():
        b = gr_batch_create(jobs, batch_opts(**opts))
        ms = _time(lambda: gr_batch_run(b), reps, warm=1)
        st, _ = gr_batch_status(b)
        gr_batch_destroy(b)
        if st != 0:
            raise RuntimeError(f"batch failed while tuning (status {st})")
        return ms

    def search(name, values, apply):
        nonlocal best_ms
        best_v = None
        for v in values:
            apply(v)
            ms = measure()
            if ms < best_ms:
                best_ms, best_v = ms, v
        if best_v is not None:
            apply(best_v)
            chosen[name] = best_v
        else:
            apply(None)

    bfs = [j for j in jobs if j.op == GR_OP_BFS]
    sssp = [j for j in jobs if j.op == GR_OP_SSSP]
    saved_bfs = [(j.big_degree, j.do_a, j.do_b) for j in bfs]
    saved_sssp = [(j.big_degree, j.delta) for j in sssp]

    def set_bfs_big(v):
        for j, sv in zip(bfs, saved_bfs):
            j.big_degree = sv[0] if v is None else v

    def set_bfs_do(v):
        for j, sv in zip(bfs, saved_bfs):
            j.do_a, j.do_b = (sv[1], sv[2]) if v is None else v

    def set_sssp_big(v):
        for j, sv in zip(sssp, saved_sssp):
            j.big_degree = sv[0] if v is None else v

    base_delta = {}
    if graphs_by_handle:
        for j in sssp:
            if j.g not in base_delta:
                base_delta[j.g] = default_delta(graphs_by_handle[j.g])

    def set_delta(v):
        for j, sv in zip(sssp, saved_sssp):
            j.delta = sv[1] if v is None else max(1, int(base_delta[j.g] * v))

    if bfs:
        search("bfs_big_degree", BATCH_BFS_BIG, set_bfs_big)
        saved_bfs = [(j.big_degree, j.do_a, j.do_b) for j in bfs]
        search("bfs_do", BATCH_BFS_DO, set_bfs_do)
    if sssp:
        search("sssp_big_degree", BATCH_SSSP_BIG, set_sssp_big)
        saved_sssp = [(j.big_degree, j.delta) for j in sssp]
        if base_delta:
            search("sssp_delta_factor", BATCH_DELTA_FACTORS, set_delta)
    return opts, best_ms, chosen


def tune_jobs(jobs, graphs_by_handle, sample_sources: int = 2, cache: TuneCache | None = None):
    """Fill each job's per-level knobs from the tuned choice of its graph.

    graphs_by_handle maps a graph handle to its Graph object.  Returns the
    jobs with do_a / do_b / big_degree / delta set.
    """
    import numpy as np
    chosen: dict[tuple, object] = {}
    for j in jobs:
        key = (j.g, j.op)
        if key in chosen:
            continue
        G = graphs_by_handle[j.g]
        srcs = [j.src] + [int(s) for s in np.random.default_rng(0).integers(0, G.n, sample_sources)]
        if j.op == GR_OP_BFS:
            chosen[key] = tune_bfs(G, srcs[:sample_sources], cache=cache,
                                   grid={**BFS_GRID, "blocks_per_sm": [0]})
        else:
            chosen[key] = tune_sssp(G, srcs[:sample_sources], cache=cache, reps=1,
                                    factors=[0.5, 1.0, 4.0], bigs=(1024,))
    for j in jobs:
        c = chosen[(j.g, j.op)]
        if j.op == GR_OP_BFS:
            j.do_a, j.do_b, j.big_degree = c.do_a, c.do_b, c.big_degree
        elif j.op == GR_OP_SSSP:
            j.delta, j.big_degree = c.delta, c.big_degree
    return jobs
