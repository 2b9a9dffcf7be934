"""Serving loop: continuous batching of BFS / SSSP queries over device-resident graphs.

Requests (graph, op, source) arrive over time.  The dispatcher admits them
as soon as a lane is idle and the lane's scratch for that graph fits the
HBM budget (the footprint model of the paper's memory discussion, Sec. 7:
per-query bytes from gr_graph_footprint), and groups BFS requests that are
waiting on the same low-diameter graph into one bit-parallel multi-source
unit (gr_bfs_multi, up to 256 sources).  Lanes are worker threads, each with
its own CUDA stream and workspaces, so units from different lanes overlap on
the GPU.  Requests that arrive while others run join the queue and are
admitted as lanes and memory free up (continuous batching).

Latency of a request = completion time - arrival time, where completion
includes copying its result (depth or dist) back to pinned host memory.

The policy (`Dispatcher`) is plain Python and runs against any backend; the
GPU backend (`GpuBackend`) executes units through the C ABI.
"""
from __future__ import annotations

import collections
import statistics
import threading
import time
from dataclasses import dataclass, field

OP_BFS, OP_SSSP = 1, 2


@dataclass
class Request:
    rid: int
    graph: str
    op: int
    src: int
    t_arrival: float
    t_start: float | None = None
    t_done: float | None = None
    result: object = None          # host numpy array (depth or dist)
    status: int = 0
    lane: int = -1                 # the lane that ran it


@dataclass
class Unit:
    """What one lane runs at once: one query, or several BFS queries as one MS-BFS."""
    graph: str
    op: int
    requests: list
    multi: bool = False


@dataclass
class GraphInfo:
    name: str
    n: int
    bytes_bfs: int                 # per-query workspace bytes (BFS)
    bytes_sssp: int
    bytes_multi: int               # multi-source scratch + output, allocated once per graph
    multi_ok: bool                 # low diameter: group BFS requests into MS-BFS
    max_group: int = 256           # sources per MS-BFS unit (bounded by output bytes)


class Dispatcher:
    """Admission and grouping policy (no GPU calls).

    The memory model: each lane keeps at most one workspace per graph it has
    served (reused), plus one multi-source scratch per graph.  A unit is
    admitted on an idle lane when the bytes it would add keep the total under
    `budget`; otherwise the lane evicts its own least recently used
    workspaces first, then those of other idle lanes (nothing runs on them),
    and if that is not enough the unit waits for running lanes to finish.
    """

    def __init__(self, graphs: dict[str, GraphInfo], lanes: int, budget: int,
                 max_group: int = 256):
        self.graphs = graphs
        self.nlanes = lanes
        self.budget = budget
        self.max_group = max_group
        self.pending: collections.deque[Request] = collections.deque()
        self.lane_ws: list[collections.OrderedDict] = [collections.OrderedDict()
                                                       for _ in range(lanes)]
        self.multi_alloc: set[str] = set()
        self.multi_busy: set[str] = set()
        self.used = 0
        self.evictions = 0

    def ws_bytes(self, g: str, op: int) -> int:
        gi = self.graphs[g]
        return gi.bytes_bfs if op == OP_BFS else gi.bytes_sssp

    def admit(self, lane: int, idle=()) -> tuple[Unit | None, list]:
        """Next unit for an idle lane and the (lane, (graph, op)) workspaces to evict
        first: the lane's own, least recently used first, then those of the other
        lanes in `idle`."""
        if not self.pending:
            return None, []
        others = [l for l in idle if l != lane]
        for idx, r in enumerate(self.pending):
            gi = self.graphs[r.graph]
            multi = r.op == OP_BFS and gi.multi_ok and r.graph not in self.multi_busy
            if multi:
                need = 0 if r.graph in self.multi_alloc else gi.bytes_multi
            else:
                need = 0 if (r.graph, r.op) in self.lane_ws[lane] else self.ws_bytes(r.graph, r.op)
            evict = []
            free = self.budget - self.used
            if need > free:
                for l in [lane] + others:
                    for key, b in self.lane_ws[l].items():   # least recently used first
                        if l == lane and key == (r.graph, r.op):
                            continue
                        evict.append((l, key))
                        free += b
                        if need <= free:
                            break
                    if need <= free:
                        break
                if need > free:
                    continue                      # try a later request that fits
            for l, key in evict:
                self.used -= self.lane_ws[l].pop(key)
                self.evictions += 1
            if multi:
                group = [r]
                rest = collections.deque()
                for j, q in enumerate(self.pending):
                    if j == idx:
                        continue
                    if (len(group) < min(self.max_group, gi.max_group) and q.graph == r.graph
                            and q.op == OP_BFS):
                        group.append(q)
                    else:
                        rest.append(q)
                self.pending = rest
                if r.graph not in self.multi_alloc:
                    self.multi_alloc.add(r.graph)
                    self.used += need
                self.multi_busy.add(r.graph)
                return Unit(r.graph, OP_BFS, group, multi=True), evict
            del self.pending[idx]
            key = (r.graph, r.op)
            if key in self.lane_ws[lane]:
                self.lane_ws[lane].move_to_end(key)
            else:
                self.lane_ws[lane][key] = need
                self.used += need
            return Unit(r.graph, r.op, [r]), evict
        return None, []

    def release(self, unit: Unit):
        if unit.multi:
            self.multi_busy.discard(unit.graph)


class GpuBackend:
    """Executes units through the C ABI; one CUDA stream and workspace set per lane."""

    MULTI_OUT_BYTES = 256 << 20

    def __init__(self, graphs: dict, lanes: int, blocks_per_sm: int = 1, bfs_opts=None,
                 sssp_opts=None, multi_out_bytes: int | None = None):
        import torch

        from . import (GR_OP_BFS, GR_OP_SSSP, bfs_opts as _bo, gr_graph_footprint,
                       sssp_opts as _so)
        self.torch = torch
        if multi_out_bytes:
            self.MULTI_OUT_BYTES = int(multi_out_bytes)
        self.graphs = graphs                     # name -> Graph
        self.streams = [torch.cuda.Stream() for _ in range(lanes)]
        self.ws = [dict() for _ in range(lanes)]
        self.blocks_per_sm = blocks_per_sm
        self.bfs_opts = bfs_opts or {}
        self.sssp_opts = sssp_opts or {}
        self._bo, self._so = _bo, _so
        nmax = max(G.n for G in graphs.values())
        self.dev_out = [torch.empty(nmax, dtype=torch.int32, device="cuda") for _ in range(lanes)]
        self.host_out = [torch.empty(nmax, dtype=torch.int32).pin_memory() for _ in range(lanes)]
        # MS-BFS output: at most MULTI_OUT_BYTES per unit (k * n * 4 bytes)
        self.multi_host = [torch.empty(self.MULTI_OUT_BYTES // 4, dtype=torch.int32).pin_memory()
                           for _ in range(lanes)]
        self.multi_out: dict[str, object] = {}
        self.footprint = {name: (gr_graph_footprint(G.handle, GR_OP_BFS),
                                 gr_graph_footprint(G.handle, GR_OP_SSSP))
                          for name, G in graphs.items()}
        self.graph_blocks: dict[str, int] = {}   # name -> CTA cap of its queries (0: none)
        self.evicted = 0                          # workspaces released by evictions

    def calibrate(self, names, srcs: dict, slack: float = 1.5):
        """Cap the CTAs of a graph's queries at SMs / lanes when that costs a query at
        most `slack` times its full-GPU time (latency-bound, high-diameter graphs), so
        that the lanes run such queries side by side instead of one at a time."""
        from . import gr_bfs
        torch = self.torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        cap = max(1, sms // len(self.streams))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

        def once(G, src, opts):
            out = self.dev_out[0][:G.n]
            gr_bfs(G.handle, src, out, None, opts)       # warm
            ev[0].record()
            gr_bfs(G.handle, src, out, None, opts)
            ev[1].record()
            ev[1].synchronize()
            return ev[0].elapsed_time(ev[1])

        for name in names:
            G = self.graphs[name]
            full = once(G, srcs[name], self._bo(blocks_per_sm=self.blocks_per_sm))
            capped = once(G, srcs[name], self._bo(blocks_per_sm=self.blocks_per_sm,
                                                  max_blocks=cap))
            self.graph_blocks[name] = cap if capped <= slack * full else 0
        return dict(self.graph_blocks)

    def graph_infos(self, multi_names) -> dict[str, GraphInfo]:
        out = {}
        for name, G in self.graphs.items():
            fb, fs = self.footprint[name]
            k = self.multi_cap(name)
            out[name] = GraphInfo(name, G.n, fb, fs, 100 * G.n + k * 4 * G.n, name in multi_names, k)
        return out

    def multi_cap(self, name) -> int:
        return max(1, min(256, self.MULTI_OUT_BYTES // (4 * self.graphs[name].n)))

    def prepare_multi(self, names):
        """Allocate the multi-source scratch of each graph up front (first call allocates)."""
        from . import gr_bfs_multi
        torch = self.torch
        for name in names:
            G = self.graphs[name]
            buf = torch.empty(self.multi_cap(name) * G.n, dtype=torch.int32, device="cuda")
            self.multi_out[name] = buf
            gr_bfs_multi(G.handle, [0], buf)
        torch.cuda.synchronize()

    def evict(self, lane: int, keys):
        """Release workspaces, each in the order of the stream of the lane that holds it
        (`keys` are (lane, (graph, op)) pairs): the other lanes' streams keep running
        (nothing waits for the whole device)."""
        from . import gr_workspace_destroy_async
        for l, key in keys:
            ws = self.ws[l].pop(key, None)
            if ws:
                gr_workspace_destroy_async(ws, self.streams[l])
                self.evicted += 1

    def _workspace(self, lane, graph, op):
        from . import GR_OP_BFS, GR_OP_SSSP, gr_workspace_create_async
        key = (graph, op)
        if key not in self.ws[lane]:
            self.ws[lane][key] = gr_workspace_create_async(
                self.graphs[graph].handle, GR_OP_BFS if op == OP_BFS else GR_OP_SSSP,
                self.streams[lane])
        return self.ws[lane][key]

    def run(self, lane: int, unit: Unit, t0: float):
        """Run a unit to completion on the lane's stream (called on the lane's thread)."""
        from . import gr_bfs, gr_bfs_multi, gr_sssp, gr_sync_status
        torch = self.torch
        G = self.graphs[unit.graph]
        s = self.streams[lane]
        now = time.perf_counter() - t0
        for r in unit.requests:
            r.t_start = now
            r.lane = lane
        with torch.cuda.stream(s):
            if unit.multi:
                k = len(unit.requests)
                buf = self.multi_out[unit.graph]
                gr_bfs_multi(G.handle, [r.src for r in unit.requests], buf, stream=s)
                host = self.multi_host[lane][:k * G.n]
                host.copy_(buf[:k * G.n], non_blocking=True)
                s.synchronize()
                done = time.perf_counter() - t0
                h = host.numpy().reshape(k, G.n)
                for i, r in enumerate(unit.requests):
                    r.result = h[i].copy()
                    r.t_done = done
                return
            ws = self._workspace(lane, unit.graph, unit.op)
            r = unit.requests[0]
            out = self.dev_out[lane][:G.n]
            cap = self.graph_blocks.get(unit.graph, 0)
            if unit.op == OP_BFS:
                gr_bfs(G.handle, r.src, out, None,
                       self._bo(ws=ws, blocks_per_sm=self.blocks_per_sm, max_blocks=cap,
                                **self.bfs_opts), s)
            else:
                gr_sssp(G.handle, r.src, out, None,
                        self._so(ws=ws, blocks_per_sm=self.blocks_per_sm, max_blocks=cap,
                                 **self.sssp_opts), s)
            hv = self.host_out[lane][:G.n]
            hv.copy_(out, non_blocking=True)
            s.synchronize()
            r.status = gr_sync_status(G.handle, ws, s)
            r.t_done = time.perf_counter() - t0
            r.result = hv.numpy().copy()

    def close(self):
        for lane in range(len(self.ws)):
            self.evict(lane, [(lane, k) for k in list(self.ws[lane].keys())])
        self.torch.cuda.synchronize()


def serve_trace(backend, trace: list[Request], lanes: int, budget: int, multi_names=(),
                max_group: int = 256) -> dict:
    """Replay a trace in real time through the dispatcher and lanes; returns statistics."""
    disp = Dispatcher(backend.graph_infos(set(multi_names)), lanes, budget, max_group)
    trace = sorted(trace, key=lambda r: r.t_arrival)
    lock = threading.Condition()
    idle = list(range(lanes))
    done_units = []
    t0 = time.perf_counter()

    def work(lane, unit):
        try:
            backend.run(lane, unit, t0)
        finally:
            with lock:
                disp.release(unit)
                idle.append(lane)
                done_units.append(unit)
                lock.notify_all()

    nxt = 0
    threads = []
    with lock:
        while nxt < len(trace) or disp.pending or len(idle) < lanes:
            now = time.perf_counter() - t0
            while nxt < len(trace) and trace[nxt].t_arrival <= now:
                disp.pending.append(trace[nxt])
                nxt += 1
            started = False
            progress = True
            while idle and disp.pending and progress:
                progress = False
                for lane in reversed(idle):
                    unit, evict = disp.admit(lane, idle)
                    if unit is None:
                        continue
                    idle.remove(lane)
                    backend.evict(lane, evict)
                    th = threading.Thread(target=work, args=(lane, unit), daemon=True)
                    th.start()
                    threads.append(th)
                    started = progress = True
                    break
            if started:
                continue
            if disp.pending and len(idle) == lanes:
                # every lane is idle and nothing fits even after evicting all
                # their workspaces: waiting cannot help
                raise RuntimeError("serve_trace: a pending request exceeds the memory budget")
            wait = 0.05
            if nxt < len(trace):
                wait = max(0.0, min(wait, trace[nxt].t_arrival - (time.perf_counter() - t0)))
            lock.wait(timeout=wait)
    for th in threads:
        th.join()
    return summarize(trace, time.perf_counter() - t0, disp)


def serve_serial(backend, trace: list[Request]) -> dict:
    """The one-query-at-a-time plain path: arrival order, no overlap, no grouping."""
    trace = sorted(trace, key=lambda r: r.t_arrival)
    t0 = time.perf_counter()
    for r in trace:
        now = time.perf_counter() - t0
        if now < r.t_arrival:
            time.sleep(r.t_arrival - now)
        backend.run(0, Unit(r.graph, r.op, [r]), t0)
    return summarize(trace, time.perf_counter() - t0, None)


def summarize(trace, wall: float, disp) -> dict:
    lat = sorted((r.t_done - r.t_arrival) * 1e3 for r in trace if r.t_done is not None)
    if not lat:
        return {"completed": 0}

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]

    span = max(r.t_done for r in trace) - min(r.t_arrival for r in trace)
    out = {"completed": len(lat), "queries_per_s": len(lat) / span if span > 0 else None,
           "p50_ms": pct(50), "p99_ms": pct(99), "mean_ms": statistics.mean(lat),
           "wall_s": wall, "errors": sum(1 for r in trace if r.status != 0)}
    if disp is not None:
        out["evictions"] = disp.evictions
    return out


def poisson_trace(graph_names, rate: float, count: int, seed: int, sources_of) -> list[Request]:
    """`count` requests, exponential inter-arrival times at `rate` per second; each picks a
    graph uniformly, BFS/SSSP 50/50 and a random non-isolated source (sources_of(name, rng))."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        g = graph_names[int(rng.integers(0, len(graph_names)))]
        op = OP_BFS if rng.random() < 0.5 else OP_SSSP
        out.append(Request(i, g, op, int(sources_of(g, rng)), t))
    return out
