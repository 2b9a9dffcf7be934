#!/usr/bin/env python3
"""Benchmark: traversal throughput (GTEPS) of direction-optimising BFS + SSSP.

Workload (the paper's R-MAT recipe, Sec. 7 "Datasets"): undirected R-MAT,
scale 22, edge factor 16, a/b/c/d = .57/.19/.19/.05, seed 2, uint32 weights
uniform in [1, 64]; int32 CSR.  One step = one gr_bfs (direction-optimising)
plus one gr_sssp from the same source; steps cycle over the highest-degree
vertex and 64 seeded random non-isolated sources.

GTEPS follows the paper's definition (Sec. 7 "Measurement methodology"): the
sum of neighbour-list lengths of all visited vertices, per query, divided by
the time.  A step's edges are that sum for its BFS plus that sum for its SSSP.

Arms:
  default           the CUDA library (libgr.so) through its C ABI;
  --impl reference  the CPU oracle (oracle/) on the host cores.
Run with torchrun for N > 1 GPUs: every rank runs independent queries on its
own GPU (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

SCALE, EF, SEED, WLO, WHI = 22, 16, 2, 1, 64
N_RANDOM_SOURCES = 64
METRIC = "GTEPS"
L2_FLUSH_BYTES = 512 << 20   # larger than the 129 MB L2


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1 + N_RANDOM_SOURCES,
                   help="timed steps; the default runs every source (hub + 64 random) once")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--scale", type=int, default=SCALE, help="R-MAT scale (22 = the named workload)")
    p.add_argument("--no-cpu-baseline", action="store_true",
                   help="skip the timed CPU-oracle sample (for profiler runs)")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--workload", choices=["s22", "s16", "grid", "msbfs", "batch", "serve", "ops",
                                          "push", "bc", "cc", "tc", "static"],
                   default="s22",
                   help="s22 (default, the headline workload) or one of the other configurations")
    p.add_argument("--rates", default="20,2000,5000,10000,20000,50000",
                   help="serve: Poisson arrival rates (requests/s); the first one is below "
                        "the service rate (unloaded latency), the others saturate it")
    p.add_argument("--requests", type=int, default=400, help="serve: requests per rate")
    p.add_argument("--no-extras", action="store_true",
                   help="s22: skip the push-only BFS, multi-source, batch and serving legs "
                        "(for profiler runs)")
    return p.parse_args()


def workload(scale):
    import graphgen as gg
    g = gg.rmat_weighted(scale, EF, SEED, WLO, WHI)
    hub = gg.max_degree_vertex(g)
    srcs = [hub] + [int(s) for s in gg.sources(g, N_RANDOM_SOURCES, seed=SEED)]
    return g, srcs


def config(g, args, n_gpus):
    return {
        "workload": f"rmat_s{args.scale}_ef{EF}_seed{SEED}: one direction-optimising BFS + one "
                    f"SSSP per step, sources = highest-degree vertex then {N_RANDOM_SOURCES} "
                    f"seeded random non-isolated vertices",
        "graph": {"n": g.n, "m_directed": g.m, "weights": f"uint32 U[{WLO},{WHI}]",
                  "csr": "int32 row offsets, int32 columns"},
        "sources": f"{1 + N_RANDOM_SOURCES} in a fixed list (the highest-degree vertex first); "
                   f"timed step k of rank r runs list entry (7r + k) mod {1 + N_RANDOM_SOURCES}, "
                   f"so rank 0 times the hub first; warm-up runs the last W entries; the "
                   f"line's sources_timed lists them",
        "l2": "flushed between steps (512 MB write, untimed); CSR is 1.04 GB > L2",
        "parallelism": f"replicas x{n_gpus} (independent queries per GPU)",
    }


def timed_sources(srcs, rank, steps):
    """List entries the timed steps of `rank` run, in order (the hub first on rank 0)."""
    k = rank_source_offset(rank)
    return [srcs[(k + i) % len(srcs)] for i in range(steps)]


def warmup_sources(srcs, warmup):
    """Warm-up runs the last entries of the list, so the timed steps keep the hub."""
    return [srcs[-1 - (i % len(srcs))] for i in range(warmup)]


# ---------------------------------------------------------------- clocks ---

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------- CPU baseline ---

def host_threads(g):
    cores = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 64 << 30
    per_query = 20 * g.m + 64 * g.n          # Dijkstra heap + arrays, with margin
    return max(1, min(cores, int(avail * 0.5 // per_query)))


def oracle_queries(g, srcs, threads):
    """Run BFS + Dijkstra of the oracle for each source, `threads` at a time.

    Returns (wall seconds, traversed edges).  ctypes releases the GIL while the
    C oracle runs, so the threads use separate host cores.
    """
    import concurrent.futures as cf

    import oracle
    deg = g.degrees()

    def one(src):
        d, _ = oracle.bfs(g.R, g.C, src)
        dist, _, _ = oracle.dijkstra(g.R, g.C, g.W, src)
        return int(deg[d >= 0].sum()) + int(deg[dist != oracle.INF32].sum())

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        edges = sum(ex.map(one, srcs))
    return time.perf_counter() - t0, edges


def cpu_baseline(g, srcs):
    """Throughput of the oracle on all host cores, plus its one-thread latency."""
    threads = host_threads(g)
    sample = [srcs[i % len(srcs)] for i in range(threads)]
    secs, edges = oracle_queries(g, sample, threads)
    secs1, _ = oracle_queries(g, [srcs[0]], 1)
    return {"value": edges / secs / 1e9, "unit": "GTEPS", "cores": threads, "kind": "oracle",
            "latency_ms_one_thread": secs1 * 1e3,
            "sample": f"{threads} BFS+SSSP query pairs (oracle queue BFS + binary-heap "
                      f"Dijkstra) on the same graph, one per host thread, {secs:.1f} s wall; "
                      f"latency: one pair from the highest-degree vertex on one thread"}


# -------------------------------------------------------------- helpers ---

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_source_offset(rank: int) -> int:
    """Replicas start at different sources so that ranks run different queries."""
    return rank * 7


def aggregate_ranks(dev_ms: float, edges: int, world: int):
    """(max timed milliseconds over ranks, total traversed edges over ranks).

    Replicas only: this is the one collective, and it runs after the timed
    region (the data path has none).
    """
    if world <= 1:
        return dev_ms, float(edges)
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([dev_ms, float(edges)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def emit(obj):
    print(json.dumps(obj), flush=True)


# ------------------------------------------------------- reference arm ---

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    g, srcs = workload(args.scale)
    threads = host_threads(g)
    per_step = threads
    k = 0
    for _ in range(args.warmup):
        oracle_queries(g, [srcs[(k + i) % len(srcs)] for i in range(per_step)], threads)
        k += per_step
    tot_s, tot_e = 0.0, 0
    for _ in range(args.steps):
        s, e = oracle_queries(g, [srcs[(k + i) % len(srcs)] for i in range(per_step)], threads)
        tot_s += s
        tot_e += e
        k += per_step
    val = tot_e / tot_s / 1e9
    emit({"impl": "reference", "metric": METRIC, "value": val, "unit": "GTEPS", "n_gpus": args.gpus,
          "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": tot_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "int32", "data": "synthetic",
          "config": config(g, args, args.gpus),
          "cpu_baseline": {"value": val, "unit": "GTEPS", "cores": threads, "kind": "oracle",
                           "sample": f"each step = {per_step} BFS+SSSP query pairs, one per "
                                     f"host thread"},
          "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                  "d2h_bytes_per_step": 0}})


# -------------------------------------------------------------- GPU arm ---

def algorithmic_bytes(kind, n, m_r=0, n_r=0, st=None):
    """Bytes one launch must move for its query, by the per-unit figures of the method.

    push_bfs: 4 B per column of a reached vertex (m_r: the sum of the degrees
              of the reached vertices), 24 B per reached vertex (frontier entry
              in and out, its two row offsets, its depth and pred writes), 8 B
              per vertex for the depth/pred initialisation: 4 m_r + 24 n_r + 8 n.
    bfs:      the direction-optimising launch counted from its own counters:
              push rows as above, pull levels 4 B per neighbour checked and 12 B
              per unvisited candidate (its row offsets and depth):
              4 edges + 12 rows + 12 discovered + 8 n.
    sssp:     the lower bound that relaxes every edge of a reached vertex once:
              8 B per edge (column + weight) and 28 B per vertex (key and stamp
              initialisation, key read and dist/pred write at unpack): 8 m_r + 28 n.
              Repeated relaxations are reported beside it, not counted in it.
    """
    if kind == "push_bfs":
        return 4 * m_r + 24 * n_r + 8 * n
    if kind == "bfs":
        return 4 * st["edges"] + 12 * st["vertices"] + 12 * st["updates"] + 8 * n
    return 8 * m_r + 28 * n


def profiled_traffic() -> dict:
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the hub-source
    launches, from the committed ncu summaries under profiles/, for the kernel versions they
    were captured on; None for a kernel whose sources changed since (digest mismatch)."""
    from paper_1701_01170_gb300 import _build
    out = {}
    for kind, fname in (("bfs", "bfs_persistent_rmat_s22.md"),
                        ("sssp", "sssp_persistent_rmat_s22.md"),
                        ("push_bfs", "bfs_persistent_push_rmat_s22.md")):
        cur = _build.source_digest("bfs" if kind == "push_bfs" else kind)
        path = os.path.join(ROOT, "profiles", fname)
        out[kind] = None
        try:
            fields = {}
            with open(path) as f:
                for line in f:
                    if line.startswith("- ") and ":" in line:
                        k, v = line[2:].split(":", 1)
                        v = v.strip()
                        if v.startswith("`"):        # a `quoted` value, then a comment
                            v = v[1:].split("`", 1)[0]
                        fields[k.strip()] = v
            if fields.get("kernel_source_digest") == cur:
                out[kind] = int(fields["traffic_bytes_per_launch"])
        except (OSError, KeyError, ValueError):
            pass
    return out


def roofline_entry(kernel, launch, byts, ms, hbm, peak_note, traffic, **extra):
    ach = byts / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": traffic, "peak_kind": peak_note, "kernel": kernel, "launch": launch,
            "algorithmic_bytes": byts, "launch_ms": ms, **extra}


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_1701_01170_gb300 as gr
    gr.load()
    dev = torch.device("cuda", torch.cuda.current_device())

    g, srcs = workload(args.scale)
    G = gr.Graph.from_csr(g)
    deg_t = torch.from_numpy(g.degrees().astype(np.int64)).to(dev)
    n = g.n
    depth = torch.empty(n, dtype=torch.int32, device=dev)
    bpred = torch.empty_like(depth)
    dist_t = torch.empty_like(depth)
    spred = torch.empty_like(depth)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    # BFS and SSSP run on workspaces of their own, so that each launch's work counters can
    # be read after the step
    ws_bfs = gr.gr_workspace_create(G.handle, gr.GR_OP_BFS)
    bopts = gr.bfs_opts(ws=ws_bfs)
    sopts = gr.sssp_opts()

    def reached_stats(t, sssp):
        r = (t != -1) if sssp else (t >= 0)
        return int((deg_t * r).sum().item()), int(r.sum().item())

    def step(src, evs):
        # the L2 flush runs on the GPU while the host prepares the first launch, so the
        # start event does not time host launch overhead
        flush.zero_()
        evs[0].record(stream)
        gr.gr_bfs(G.handle, src, depth, bpred, bopts, stream=stream)
        evs[1].record(stream)
        gr.gr_sssp(G.handle, src, dist_t, spred, sopts, stream=stream)
        evs[2].record(stream)

    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for src in warmup_sources(srcs, args.warmup):
        step(src, evs)
    torch.cuda.synchronize()
    st = G.sync_status()
    if st != gr.GR_OK:
        raise RuntimeError(f"warm-up failed: {gr.status_str(st)}")

    timed = timed_sources(srcs, rank, args.steps)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    t_bfs, t_sssp, e_bfs, e_sssp = [], [], 0, 0
    b_alg, s_alg = 0, 0            # algorithmic bytes of the timed launches
    s_relaxed, s_rows, s_mr, s_nr = 0, 0, 0, 0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for src in timed:
        step(src, evs)
        evs[2].synchronize()
        t_bfs.append(evs[0].elapsed_time(evs[1]))
        t_sssp.append(evs[1].elapsed_time(evs[2]))
        # untimed: edge counts, kernel counters (the next step's flush follows)
        eb, _ = reached_stats(depth, False)
        es, nrs = reached_stats(dist_t, True)
        e_bfs += eb
        e_sssp += es
        bst = gr.gr_last_run_stats(G.handle, ws_bfs)
        sst = gr.gr_last_run_stats(G.handle)
        b_alg += algorithmic_bytes("bfs", n, st=bst)
        s_alg += algorithmic_bytes("sssp", n, m_r=es, n_r=nrs)
        s_relaxed += sst["edges"]
        s_rows += sst["vertices"]
        s_mr += es
        s_nr += nrs
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    st = G.sync_status()
    if st != gr.GR_OK or gr.gr_sync_status(G.handle, ws_bfs) != gr.GR_OK:
        raise RuntimeError(f"timed steps failed: {gr.status_str(st)}")

    # the hub launches once more with per-level traces (untimed), then timed alone three
    # times: the launch the committed ncu summaries capture
    cap = 256
    lv_b = torch.zeros(4 * cap, dtype=torch.int32, device=dev)
    lv_s = torch.zeros(4 * cap, dtype=torch.int32, device=dev)
    hub = srcs[0]
    gr.gr_bfs(G.handle, hub, depth, bpred,
              gr.bfs_opts(ws=ws_bfs, level_stats=lv_b.data_ptr(), max_levels=cap), stream=stream)
    hub_bst = gr.gr_last_run_stats(G.handle, ws_bfs)
    gr.gr_sssp(G.handle, hub, dist_t, spred,
               gr.sssp_opts(level_stats=lv_s.data_ptr(), max_levels=cap), stream=stream)
    hub_sst = gr.gr_last_run_stats(G.handle)
    hub_ms_r, hub_n_r = reached_stats(dist_t, True)
    tb = lv_b.view(cap, 4)[:min(cap, hub_bst["levels"])].cpu().tolist()
    ts_ = lv_s.view(cap, 4)[:min(cap, hub_sst["levels"])].cpu().tolist()
    trace = {
        "bfs_hub_levels": [{"frontier": r[0], "pull": r[1], "m_f": r[2], "start_us": r[3] / 1e3}
                           for r in tb],
        "sssp_hub_steps": [{"near_rows": r[0], "split": r[1], "far": r[2], "start_us": r[3] / 1e3}
                           for r in ts_],
        "sssp_hub_rows_per_reached": hub_sst["vertices"] / max(1, hub_n_r),
        "sssp_hub_edges_relaxed_per_m_r": hub_sst["edges"] / max(1, hub_ms_r),
    }
    hub_bfs_ms, hub_sssp_ms = [], []
    for _ in range(3):
        step(hub, evs)
        evs[2].synchronize()
        hub_bfs_ms.append(evs[0].elapsed_time(evs[1]))
        hub_sssp_ms.append(evs[1].elapsed_time(evs[2]))

    dev_ms = sum(t_bfs) + sum(t_sssp)
    edges = e_bfs + e_sssp
    dev_ms_max, edges_all = aggregate_ranks(dev_ms, edges, ws)
    value = edges_all / (dev_ms_max / 1e3) / 1e9

    # ---- e2e: host buffers through the C ABI, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        if ws > 1:
            torch.distributed.barrier()      # replicas start their e2e regions together
        e2e = combine_e2e(run_e2e(gr, g, srcs, args, dev, rank), ws)

    # ---- roofline: algorithmic bytes of the timed launches over their summed event time
    hbm, peak_note = hbm_peak()
    traffic = profiled_traffic()
    roof = {
        "sssp": roofline_entry(
            "sssp_persistent", f"mean over the {len(timed)} timed launches", s_alg / len(timed),
            sum(t_sssp) / len(timed), hbm, peak_note, traffic.get("sssp"),
            formula="8 m_r + 28 n (every edge of a reached vertex relaxed once)",
            edges_relaxed_per_m_r=s_relaxed / max(1, s_mr),
            rows_opened_per_reached=s_rows / max(1, s_nr),
            hub={"algorithmic_bytes": algorithmic_bytes("sssp", n, m_r=hub_ms_r, n_r=hub_n_r),
                 "ms": statistics.median(hub_sssp_ms), "counters": hub_sst,
                 "m_r": hub_ms_r, "n_r": hub_n_r},
            traffic_launch="hub source (ncu, one launch)"),
        "bfs": roofline_entry(
            "bfs_persistent", f"mean over the {len(timed)} timed launches", b_alg / len(timed),
            sum(t_bfs) / len(timed), hbm, peak_note, traffic.get("bfs"),
            formula="4 edges + 12 rows + 12 discovered + 8 n from the launch's counters",
            hub={"algorithmic_bytes": algorithmic_bytes("bfs", n, st=hub_bst),
                 "ms": statistics.median(hub_bfs_ms), "counters": hub_bst},
            traffic_launch="hub source (ncu, one launch)"),
    }
    dominant = "sssp" if sum(t_sssp) >= sum(t_bfs) else "bfs"
    out = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": config(g, args, ws),
        "sources_timed": timed,
        "breakdown": {"bfs_ms_mean": statistics.mean(t_bfs), "sssp_ms_mean": statistics.mean(t_sssp),
                      "bfs_gteps": e_bfs / (sum(t_bfs) / 1e3) / 1e9,
                      "sssp_gteps": e_sssp / (sum(t_sssp) / 1e3) / 1e9,
                      "bfs_ms_median": statistics.median(t_bfs),
                      "sssp_ms_median": statistics.median(t_sssp),
                      "bfs_ms_p99": float(np.percentile(t_bfs, 99)),
                      "sssp_ms_p99": float(np.percentile(t_sssp, 99)),
                      "kernel_share": {"sssp_persistent": sum(t_sssp) / dev_ms,
                                       "bfs_persistent": sum(t_bfs) / dev_ms},
                      "wall_s_timed_loop": wall},
        "roofline": roof[dominant],
        "roofline_other": roof["bfs" if dominant == "sssp" else "sssp"],
        "clocks": clk,
        "trace": trace,
        "gpu_launches": 2 * args.steps,
        "e2e": e2e,
    }
    if rank == 0 and not args.no_extras:
        out["push_bfs"] = measure_push_bfs(gr, G, g, timed, depth, flush, hbm, peak_note,
                                           traffic.get("push_bfs"), deg_t, stream)
        # the next operator families on the same graph (Sec. 6.3, 6.4, 6.6)
        out["bc"] = measure_bc(gr, G, g, srcs[:4], flush, deg_t, hbm, peak_note)
        out["cc"] = measure_cc(gr, G, g, hub, flush, hbm, peak_note)
        out["tc"] = measure_tc(gr, G, g, flush, hbm, peak_note)
    gr.gr_workspace_destroy(ws_bfs)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(g, srcs)
    G.close()
    del G
    if rank == 0 and ws == 1 and not args.no_extras:
        # the batched and served forms, each against the plain one-query path on this GPU
        out["msbfs"] = measure_msbfs(gr, reps=3)
        out["batch"] = measure_batch(gr, reps=5)
        out["serve"] = measure_serve(gr, rates=[20.0, 2000.0], requests=160)
    if rank == 0:
        emit(out)
    if ws > 1:
        torch.distributed.destroy_process_group()


def measure_push_bfs(gr, G, g, sources, do_depth, flush, hbm, peak_note, traffic, deg_t,
                     stream):
    """Push-only BFS (advance + visit + cull fused, no pull levels) from the same sources:
    its HBM fraction against 4 m_r + 24 n_r + 8 n, the advance + filter figure of merit.
    Depths must equal the direction-optimising run's."""
    import torch
    n = g.n
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    opts = gr.bfs_opts(direction=gr.GR_DIR_PUSH)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def once(src):
        flush.zero_()
        e0.record(stream)
        gr.gr_bfs(G.handle, src, depth, None, opts, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    once(sources[0])
    tot_ms, tot_b, tot_e, same = 0.0, 0, 0, True
    per = []
    hub_ms = []
    for i, src in enumerate(sources):
        ms = once(src)
        r = depth >= 0
        m_r, n_r = int((deg_t * r).sum().item()), int(r.sum().item())
        b = algorithmic_bytes("push_bfs", n, m_r=m_r, n_r=n_r)
        gr.gr_bfs(G.handle, src, do_depth, None, stream=stream)      # direction-optimising
        same = same and bool(torch.equal(depth, do_depth))
        tot_ms += ms
        tot_b += b
        tot_e += m_r
        per.append(ms)
        if i == 0:
            hub_ms.append(ms)
            hub_b = b
    for _ in range(2):
        hub_ms.append(once(sources[0]))
    # per-level trace of the first source (untimed)
    cap = 256
    lv = torch.zeros(4 * cap, dtype=torch.int32, device="cuda")
    gr.gr_bfs(G.handle, sources[0], depth, None,
              gr.bfs_opts(direction=gr.GR_DIR_PUSH, level_stats=lv.data_ptr(), max_levels=cap),
              stream=stream)
    levels = gr.gr_last_run_stats(G.handle)["levels"]
    trace = [{"frontier": r[0], "m_f": r[2], "start_us": r[3] / 1e3}
             for r in lv.view(cap, 4)[:min(cap, levels)].cpu().tolist()]
    if G.sync_status() != gr.GR_OK:
        raise RuntimeError("push-only BFS failed")
    hub = roofline_entry("bfs_persistent (push only)", "first timed source", hub_b,
                         statistics.median(hub_ms), hbm, peak_note, traffic,
                         formula="4 m_r + 24 n_r + 8 n")
    return {"kernel": "bfs_persistent, direction = push only",
            "formula": "4 m_r + 24 n_r + 8 n (m_r: sum of degrees of reached vertices)",
            "sources": len(sources), "ms_mean": tot_ms / len(sources),
            "ms_median": statistics.median(per), "gteps": tot_e / (tot_ms / 1e3) / 1e9,
            "achieved": tot_b / (tot_ms / 1e3) / 1e9, "peak": hbm,
            "frac": tot_b / (tot_ms / 1e3) / 1e9 / hbm, "first_source": hub,
            "depths_identical_to_direction_optimising": same, "first_source_levels": trace}


def _timed(fn, flush, reps):
    """CUDA-event times of fn() (ms), each after an untimed L2 flush."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = []
    for _ in range(reps):
        flush.zero_()
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def measure_bc(gr, G, g, sources, flush, deg_t, hbm, peak_note):
    """Brandes' pass (gr_bc) per source.  Algorithmic bytes per source:
    8 m_r (the columns of the reached rows, read by both passes) + 52 n_r (per reached
    vertex: BFS-order entry written and read twice, row offsets twice, sigma read twice,
    delta written) + 44 n (depth, sigma and delta initialised; bc read and written, delta
    read).  Depths must equal gr_bfs's."""
    import torch
    n = g.n
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    sigma = torch.empty(n, dtype=torch.int64, device="cuda")
    delta = torch.empty(n, dtype=torch.float64, device="cuda")
    bc = torch.zeros(n, dtype=torch.float64, device="cuda")
    ref = torch.empty_like(depth)
    gr.gr_bc(G.handle, sources[0], depth, sigma, delta, bc)          # warm (allocates scratch)
    tot_ms, tot_b, tot_e, same, per = 0.0, 0, 0, True, []
    for src in sources:
        ms = statistics.median(_timed(lambda: gr.gr_bc(G.handle, src, depth, sigma, delta, bc),
                                      flush, 3))
        r = depth >= 0
        m_r, n_r = int((deg_t * r).sum().item()), int(r.sum().item())
        gr.gr_bfs(G.handle, src, ref, None)
        same = same and bool(torch.equal(depth, ref))
        b = 8 * m_r + 52 * n_r + 44 * n
        tot_ms += ms
        tot_b += b
        tot_e += 2 * m_r
        per.append({"source": int(src), "ms": ms, "m_r": m_r, "n_r": n_r,
                    "levels": gr.gr_last_run_stats(G.handle)["levels"]})
    ok = G.sync_status() == gr.GR_OK
    ach = tot_b / (tot_ms / 1e3) / 1e9
    return {"kernel": "bc_persistent", "sources": len(sources), "ms_mean": tot_ms / len(sources),
            "gteps": tot_e / (tot_ms / 1e3) / 1e9,
            "formula": "8 m_r + 52 n_r + 44 n per source (edges counted twice: both passes)",
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": None, "peak_kind": peak_note},
            "per_source": per, "depths_identical_to_bfs": same and ok}


def measure_cc(gr, G, g, hub, flush, hbm, peak_note):
    """Connected components (gr_cc).  Algorithmic bytes: 4 m (columns once) + 8 n (row
    offsets and labels) + 16 per hooked edge (written to and read from the filtered edge
    frontier as an 8-byte pair).  The hub's component must have as many vertices as a BFS
    from the hub reaches."""
    import torch
    comp = torch.empty(g.n, dtype=torch.int32, device="cuda")
    k = torch.zeros(1, dtype=torch.int32, device="cuda")
    gr.gr_cc(G.handle, comp, k)                                     # warm (allocates scratch)
    ms = statistics.median(_timed(lambda: gr.gr_cc(G.handle, comp, k), flush, 3))
    st = gr.gr_last_run_stats(G.handle)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    gr.gr_bfs(G.handle, hub, d, None)
    ok = G.sync_status() == gr.GR_OK and \
        int((comp == comp[hub]).sum().item()) == int((d >= 0).sum().item())
    b = 4 * g.m + 8 * g.n + 16 * st["updates"]
    ach = b / (ms / 1e3) / 1e9
    return {"kernel": "cc_persistent", "ms": ms, "components": int(k.item()),
            "hooking_iterations": st["levels"], "hooked_edges": st["updates"],
            "gteps": g.m / (ms / 1e3) / 1e9,
            "formula": "4 m + 8 n + 16 per hooked edge",
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": None, "peak_kind": peak_note},
            "hub_component_matches_bfs": ok}


def measure_tc(gr, G, g, flush, hbm, peak_note):
    """Triangle counting (gr_triangle_count, forward algorithm).  Streamed bytes: 12 m (the
    CSR columns read to orient the edges, the oriented graph's m/2 (source, column) pairs
    written and read); the intersections themselves re-read those rows from L2."""
    import torch
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    gr.gr_triangle_count(G.handle, total)                           # warm (allocates scratch)
    ms = statistics.median(_timed(lambda: gr.gr_triangle_count(G.handle, total), flush, 3))
    ok = G.sync_status() == gr.GR_OK
    b = 12 * g.m
    ach = b / (ms / 1e3) / 1e9
    return {"kernel": "tc_count (with tc_sources, scan, tc_compact)", "ms": ms,
            "triangles": int(total.item()), "triangles_per_s": int(total.item()) / (ms / 1e3),
            "oriented_edges_per_s": (g.m // 2) / (ms / 1e3),
            "formula": "12 m streamed", "status_ok": ok,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": None, "peak_kind": peak_note}}


def run_e2e(gr, g, srcs, args, dev, rank):
    """GTEPS through the public API from pinned host buffers.

    Every step copies the whole CSR (R, C, W) from pinned host memory into a
    graph's device arrays, runs gr_bfs + gr_sssp on it, and reads depth, pred,
    dist and pred back into pinned host memory.  Steps are pipelined over two
    graph buffers and three streams (upload, compute, read-back), so the upload
    of step k + 1 overlaps the queries of step k; the timed region runs from
    the first upload to the last read-back and holds every copy of every step.
    """
    import torch
    n = g.n
    hR = torch.from_numpy(g.R).pin_memory()
    hC = torch.from_numpy(g.C).pin_memory()
    hW = torch.from_numpy(g.W.view(np.int32)).pin_memory()
    Gs = [gr.Graph.from_csr(g), gr.Graph.from_csr(g)]
    steps = args.e2e_steps
    # one set of pinned result buffers per step: nothing runs on the host
    # between the steps; the results are checked after the loop
    outs_h = [[torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(4)]
              for _ in range(steps)]
    outs_d = [[torch.empty(n, dtype=torch.int32, device=dev) for _ in range(4)] for _ in range(2)]
    deg = g.degrees()
    up, comp, down = (torch.cuda.Stream() for _ in range(3))
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    k = rank_source_offset(rank)
    used = [srcs[(k + i) % len(srcs)] for i in range(steps)]
    # warm both buffers, the copy paths and the pinned result pages (untimed)
    for G, od in zip(Gs, outs_d):
        with torch.cuda.stream(up):
            G.R.copy_(hR, non_blocking=True)
            G.C.copy_(hC, non_blocking=True)
            G.W.copy_(hW, non_blocking=True)
        up.synchronize()
        gr.gr_bfs(G.handle, used[0], od[0], od[1])
        gr.gr_sssp(G.handle, used[0], od[2], od[3])
    with torch.cuda.stream(down):
        for oh in outs_h:
            for h, d in zip(oh, outs_d[0]):
                h.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    for i, src in enumerate(used):
        b = i & 1
        G, od = Gs[b], outs_d[b]
        if i >= 2:
            up.wait_event(ev[i - 2][2])      # buffer b's queries of step i - 2 are done
            comp.wait_event(ev[i - 2][3])    # and its results have been read back
        ev[i][0].record(up)
        with torch.cuda.stream(up):
            G.R.copy_(hR, non_blocking=True)
            G.C.copy_(hC, non_blocking=True)
            G.W.copy_(hW, non_blocking=True)
        ev[i][1].record(up)
        comp.wait_event(ev[i][1])
        gr.gr_bfs(G.handle, src, od[0], od[1], stream=comp)
        gr.gr_sssp(G.handle, src, od[2], od[3], stream=comp)
        ev[i][2].record(comp)
        down.wait_event(ev[i][2])
        with torch.cuda.stream(down):
            for h, d in zip(outs_h[i], od):
                h.copy_(d, non_blocking=True)
        ev[i][3].record(down)
    torch.cuda.synchronize()
    ms = ev[0][0].elapsed_time(ev[steps - 1][3])
    edges = 0
    parts = [0.0, 0.0, 0.0]
    for i in range(steps):
        parts[0] += ev[i][0].elapsed_time(ev[i][1])
        parts[2] += ev[i][2].elapsed_time(ev[i][3])
        d = outs_h[i][0].numpy()
        dist = outs_h[i][2].numpy()
        edges += int(deg[d >= 0].sum()) + int(deg[dist != -1].sum())
    for i in range(steps):
        parts[1] += ev[i][1].elapsed_time(ev[i][2])
    st = max(abs(G.sync_status()) for G in Gs)
    for G in Gs:
        G.close()
    if st != gr.GR_OK:
        raise RuntimeError(f"e2e failed: {gr.status_str(-st)}")
    return {"value": edges / (ms / 1e3) / 1e9, "unit": "GTEPS", "_ms": ms, "_edges": edges,
            "h2d_bytes_per_step": int(g.R.nbytes + g.C.nbytes + g.W.nbytes),
            "d2h_bytes_per_step": int(4 * n * 4), "steps": steps,
            "ms_per_step": ms / steps,
            "h2d_ms_per_step": parts[0] / steps,
            "upload_to_results_ms_per_step": parts[1] / steps,
            "d2h_ms_per_step": parts[2] / steps,
            "note": "whole CSR re-uploaded from pinned host memory and all four result arrays "
                    "read back every step; steps pipelined over two graph buffers and three "
                    "streams; ms_per_step = (last read-back end - first upload start) / steps"}


def hbm_peak():
    """(HBM GB/s, "measured" | "fallback"): the measured copy bandwidth of this GPU model, else
    the fallback figure of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        hbm = None
    return (hbm, "measured") if hbm else (6800.0, "fallback")


def ops_algorithmic_bytes(op, f, e, u):
    """Bytes a standalone operator must move: f frontier rows, e edges expanded, u outputs.

    advance (ordered, no functor): frontier 4 B + row bounds 8 B + per-row output offset
    8 B written and read per row, columns 4 B and outputs 4 B per edge.
    exact-unique and cull filters: 4 B read per input item, 4 B written per output item.
    multisplit: 4 B read per input item, 8 B key read per item, 4 B written per output item.
    """
    if op == "advance":
        return 4 * f + 8 * f + 16 * f + 8 * e
    if op == "multisplit":
        return 12 * e + 4 * u
    return 4 * e + 4 * u


def combine_e2e(e2e: dict, world: int) -> dict:
    """Whole-job e2e figure from one rank's: traversed edges summed over ranks over the
    longest rank's timed region; copied bytes per step summed over ranks.  With one rank
    the figure is the rank's own."""
    e2e = dict(e2e)
    ms, edges = e2e.pop("_ms"), e2e.pop("_edges")
    ms_max, edges_all = aggregate_ranks(ms, edges, world)
    e2e["value"] = edges_all / (ms_max / 1e3) / 1e9
    e2e["ms_per_step"] = ms_max / e2e["steps"]
    e2e["h2d_bytes_per_step"] *= world
    e2e["d2h_bytes_per_step"] *= world
    return e2e


# ------------------------------------------------ the other configurations ---

def _events_ms(fn, reps, warm=2):
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
    return ts


def run_other(args):
    """Non-default workloads: one JSON line each, same keys where they apply."""
    import torch

    import graphgen as gg
    import paper_1701_01170_gb300 as gr
    torch.cuda.set_device(0)
    gr.load()
    base = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "dtype": "int32",
            "data": "synthetic", "vs_baseline": None, "scaling": "weak"}
    if args.workload in ("s16", "grid"):
        if args.workload == "s16":
            g = gg.rmat(16, 16, 1)
            srcs, ops = [0], ["bfs"]
            desc = "rmat_s16_ef16_seed1: BFS from vertex 0 (int32 depth + pred)"
        else:
            g = gg.grid_weighted(4096, 0.1, 3)
            srcs = [0] + [int(x) for x in gg.sources(g, 4, seed=3)]
            ops = ["bfs", "sssp"]
            desc = "grid 4096x4096, 10% edges deleted (seed 3), weights U[1,1000]: BFS + SSSP"
        G = gr.Graph.from_csr(g)
        deg = g.degrees()
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        p = torch.empty_like(d)
        res = {}
        for op in ops:
            tot_ms, tot_e, levels = 0.0, 0, []
            for src in srcs:
                fn = (lambda: gr.gr_bfs(G.handle, src, d, p)) if op == "bfs" else \
                    (lambda: gr.gr_sssp(G.handle, src, d, p))
                ts = _events_ms(fn, max(1, args.steps // len(srcs)), warm=1)
                st = gr.gr_last_run_stats(G.handle)
                levels.append(st["levels"])
                reached = host_reached(d, op)
                tot_ms += statistics.mean(ts)
                tot_e += int(deg[reached].sum())
            res[op] = {"gteps": tot_e / (tot_ms / 1e3) / 1e9, "ms_per_query": tot_ms / len(srcs),
                       "levels_or_steps": levels,
                       "us_per_level": 1e3 * tot_ms / max(1, sum(levels))}
        assert G.sync_status() == 0
        val = sum(r["gteps"] for r in res.values()) / len(res)
        emit({"metric": "GTEPS", "value": val, "unit": "GTEPS", **base,
              "ms_per_step": sum(r["ms_per_query"] for r in res.values()),
              "higher_is_better": True, "config": {"workload": desc}, "per_op": res})
        return
    if args.workload == "ops":
        # the standalone operators on the BFS frontier after the first level from the hub of
        # R-MAT s22: advance (prefix-sum placement, ordered) and the two deduplicating filters
        g, srcs = workload(22)
        G = gr.Graph.from_csr(g)
        hub = srcs[0]
        deg = g.degrees()
        Fh = np.ascontiguousarray(g.C[g.R[hub]:g.R[hub + 1]])   # sorted, distinct rows
        E = int(deg[Fh].sum())
        in_f = np.zeros(g.n, bool)
        in_f[Fh] = True
        sel = np.repeat(in_f, deg)                              # edges of the frontier's rows
        want = g.C[sel]                                         # rows ascending = frontier order
        mark = np.zeros(g.n, bool)
        mark[want] = True
        U = int(mark.sum())
        F = torch.from_numpy(Fh).cuda()
        out = torch.empty(E, dtype=torch.int32, device="cuda")
        ol = torch.zeros(1, dtype=torch.int64, device="cuda")
        uo = torch.empty(g.n, dtype=torch.int32, device="cuda")
        ul = torch.zeros(1, dtype=torch.int64, device="cuda")
        reps = max(3, args.steps)
        res = {}
        t = _events_ms(lambda: gr.gr_advance(G.handle, F, len(Fh), out, ol), reps)
        if int(ol.item()) != E or not np.array_equal(out.cpu().numpy(), want):
            raise RuntimeError("advance output differs from the concatenated rows")
        res["advance"] = (t, ops_algorithmic_bytes("advance", len(Fh), E, E))
        for name, mode in (("filter_exact_unique", gr.GR_FILTER_EXACT_UNIQUE),
                           ("filter_cull", gr.GR_FILTER_CULL)):
            t = _events_ms(lambda: gr.gr_filter(G.handle, out, E, uo, ul, mode=mode), reps)
            got = uo[:int(ul.item())].cpu().numpy()
            if len(got) != U or not mark[got].all() or len(np.unique(got)) != U:
                raise RuntimeError(f"{name} output is not the {U} distinct neighbours")
            res[name] = (t, ops_algorithmic_bytes("filter", len(Fh), E, U))
        # multisplit of the advance output into 8 distance buckets (seeded distances)
        rng = np.random.default_rng(9)
        dist0 = rng.integers(0, 400, g.n).astype(np.uint64)
        keys = torch.from_numpy((dist0 << np.uint64(32)).view(np.int64)).cuda()
        mo = torch.empty(E, dtype=torch.int32, device="cuda")
        blen = torch.zeros(8, dtype=torch.int64, device="cuda")
        mst = gr.gr_multisplit_state(key=keys.data_ptr(), base=20, delta=40, buckets=8,
                                     bucket_len=blen.data_ptr())
        t = _events_ms(lambda: gr.gr_filter(G.handle, out, E, mo, ul,
                                            mode=gr.GR_FILTER_MULTISPLIT, state=mst), reps)
        bk = np.minimum(7, np.maximum(dist0[want].astype(np.int64) - 20, -1) // 40)
        bk[bk < 0] = 0
        got_len = blen.cpu().numpy()
        if not np.array_equal(got_len, np.bincount(bk, minlength=8)) or int(ul.item()) != E:
            raise RuntimeError("multisplit bucket sizes differ")
        res["filter_multisplit"] = (t, ops_algorithmic_bytes("multisplit", len(Fh), E, E))
        if G.sync_status() != 0:
            raise RuntimeError("operator status")
        hbm, peak_note = hbm_peak()
        per_op = {}
        for name, (t, b) in res.items():
            ms = statistics.median(t)
            per_op[name] = {"ms": ms, "algorithmic_bytes": b, "gbs": b / (ms / 1e3) / 1e9,
                            "frac": b / (ms / 1e3) / 1e9 / hbm}
        tot_b = sum(b for _, b in res.values())
        tot_ms = sum(p["ms"] for p in per_op.values())
        adv = per_op["advance"]
        emit({"metric": "operator GB/s", "value": tot_b / (tot_ms / 1e3) / 1e9, "unit": "GB/s",
              **base, "ms_per_step": tot_ms, "higher_is_better": True,
              "config": {"workload": "rmat_s22_ef16_seed2: advance of the hub's 162,948-row "
                                     "neighbourhood (84.7 M edges), then exact-unique and cull "
                                     "filters of its output and an 8-bucket multisplit of it "
                                     "(seeded distances U[0,400), base 20, width 40)",
                         "frontier_rows": len(Fh), "edges": E, "distinct": U,
                         "l2": "inputs larger than L2 (339 MB advance output)"},
              "roofline": {"bound": "hbm", "achieved": adv["gbs"], "peak": hbm, "unit": "GB/s",
                           "frac": adv["frac"], "traffic": None, "peak_kind": peak_note,
                           "kernel": "adv_expand (with adv_degree_tiles, scan_block_sums)"},
              "per_op": per_op})
        return
    if args.workload == "push":
        # the push-only BFS leg of the s22 line on its own (hub first), for profiler runs
        g, srcs = workload(22)
        G = gr.Graph.from_csr(g)
        hbm, peak_note = hbm_peak()
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        deg_t = torch.from_numpy(g.degrees().astype(np.int64)).cuda()
        r = measure_push_bfs(gr, G, g, srcs[:max(1, args.steps)], d, flush, hbm, peak_note,
                             profiled_traffic().get("push_bfs"), deg_t,
                             torch.cuda.current_stream())
        G.close()
        emit({"metric": "GB/s", "value": r["achieved"], "unit": "GB/s", **base,
              "ms_per_step": r["ms_mean"], "higher_is_better": True,
              "config": {"workload": "rmat_s22_ef16_seed2: push-only BFS from the highest-degree "
                                     "vertex, then the seeded random sources"},
              "roofline": r["first_source"], **r})
        return
    if args.workload == "static":
        # gr_bfs_static (no allocation, scratch in a static device array) beside gr_bfs on
        # the largest graph it accepts: R-MAT scale 20 (n = 2^20), edge factor 16
        g = gg.rmat(20, 16, 1)
        srcs = [gg.max_degree_vertex(g)] + [int(x) for x in gg.sources(g, 7, seed=1)]
        G = gr.Graph.from_csr(g)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        res = {}
        for name, fn in (("gr_bfs", lambda s_: gr.gr_bfs(G.handle, s_, d, None)),
                         ("gr_bfs_static", lambda s_: gr.gr_bfs_static(
                             g.n, g.m, G.R, G.C, s_, d, None, st, flags=gr.GR_SYMMETRIC))):
            fn(srcs[0])
            ts = [statistics.median(_timed(lambda: fn(s_), flush, 3)) for s_ in srcs]
            res[name] = {"ms_hub": ts[0], "ms_mean": statistics.mean(ts)}
        ok = G.sync_status() == gr.GR_OK and int(st.item()) == gr.GR_OK
        G.close()
        emit({"metric": "ms", "value": res["gr_bfs_static"]["ms_mean"], "unit": "ms", **base,
              "ms_per_step": res["gr_bfs_static"]["ms_mean"], "higher_is_better": False,
              "config": {"workload": "rmat_s20_ef16_seed1: BFS from the hub and 7 random "
                                     "sources, static-scratch entry point vs gr_bfs"},
              "per_entry": res, "status_ok": ok})
        return
    if args.workload in ("bc", "cc", "tc"):
        # one operator family on R-MAT s22 (the s22 line's bc / cc / tc legs on their own)
        g, srcs = workload(22)
        G = gr.Graph.from_csr(g)
        hbm, peak_note = hbm_peak()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
        deg_t = torch.from_numpy(g.degrees().astype(np.int64)).cuda()
        if args.workload == "bc":
            r = measure_bc(gr, G, g, srcs[:max(1, args.steps)], flush, deg_t, hbm, peak_note)
            val, unit, ms = r["gteps"], "GTEPS", r["ms_mean"]
        elif args.workload == "cc":
            r = measure_cc(gr, G, g, srcs[0], flush, hbm, peak_note)
            val, unit, ms = r["gteps"], "GTEPS", r["ms"]
        else:
            r = measure_tc(gr, G, g, flush, hbm, peak_note)
            val, unit, ms = r["triangles_per_s"], "triangles/s", r["ms"]
        G.close()
        emit({"metric": unit, "value": val, "unit": unit, **base, "ms_per_step": ms,
              "higher_is_better": True,
              "config": {"workload": f"rmat_s22_ef16_seed2: {args.workload}"}, **r})
        return
    if args.workload == "msbfs":
        r = measure_msbfs(gr, reps=args.steps)
        emit({"metric": "GTEPS", "value": r["gteps"], "unit": "GTEPS", **base,
              "ms_per_step": r["ms"], "higher_is_better": True,
              "config": {"workload": r["workload"]}, **r})
        return
    if args.workload == "batch":
        r = measure_batch(gr, reps=args.steps)
        emit({"metric": "jobs/s", "value": r["jobs_per_s"], "unit": "jobs/s", **base,
              "ms_per_step": r["ms"], "higher_is_better": True,
              "config": {"workload": r["workload"]}, **r})
        return
    if args.workload == "serve":
        r = measure_serve(gr, [float(x) for x in args.rates.split(",")], args.requests)
        best = max(r["per_rate"], key=lambda x: x["served"]["queries_per_s"])
        emit({"metric": "queries/s", "value": best["served"]["queries_per_s"],
              "unit": "queries/s", **base, "ms_per_step": best["served"]["p50_ms"],
              "higher_is_better": True, "config": {"workload": r["workload"]}, **r})
        return


def host_reached(d, op):
    a = d.cpu().numpy()
    return a >= 0 if op == "bfs" else a != -1


def measure_msbfs(gr, reps):
    """256-source bit-parallel BFS on R-MAT s20 against 256 plain gr_bfs calls on the same
    GPU; the depth matrices must be identical."""
    import torch

    import graphgen as gg
    g = gg.rmat(20, 16, 1)
    srcs = gg.sources(g, 256, seed=4)
    G = gr.Graph.from_csr(g)
    n = g.n
    D = torch.empty(256 * n, dtype=torch.int32, device="cuda")
    ts = _events_ms(lambda: gr.gr_bfs_multi(G.handle, srcs, D), reps)
    P = torch.empty_like(D)

    def plain():
        for i, s_ in enumerate(srcs):
            gr.gr_bfs(G.handle, int(s_), P[i * n:(i + 1) * n], None)
    tp = _events_ms(plain, max(1, reps // 2), warm=1)
    same = bool(torch.equal(D, P))
    deg_t = torch.from_numpy(g.degrees().astype(np.int64)).cuda()
    edges = int(((D.view(256, n) >= 0).to(torch.int64) * deg_t).sum().item())
    ok = G.sync_status() == gr.GR_OK
    G.close()
    ms, mp = statistics.median(ts), statistics.median(tp)
    return {"workload": "rmat_s20_ef16_seed1: 256-source bit-parallel BFS (sources: 256 "
                        "random non-isolated vertices, seed 4) vs 256 gr_bfs calls",
            "ms": ms, "gteps": edges / (ms / 1e3) / 1e9, "queries_per_s": 256 / ms * 1e3,
            "plain_path": {"ms_256_gr_bfs": mp, "gteps": edges / (mp / 1e3) / 1e9,
                           "queries_per_s": 256 / mp * 1e3},
            "speedup_vs_plain": mp / ms, "results_identical": same and ok}


def measure_batch(gr, reps):
    """512 BFS/SSSP jobs over 64 R-MAT graphs in one persistent launch under a CUDA graph
    (launch shape and per-level strategy from the batch autotuner) against the plain
    one-query-at-a-time loop; depths, distances and SSSP predecessors must be identical."""
    import torch

    from graphgen import workloads as wl
    from paper_1701_01170_gb300 import tune
    bgs = wl.batch_graphs(64, seed=5)
    triples = wl.batch_jobs(bgs, 512, seed=5)
    Gs = [gr.Graph.from_csr(b.csr) for b in bgs]
    jobs, outs, plain_outs = [], [], []
    for gi, op, src in triples:
        o = torch.empty(Gs[gi].n, dtype=torch.int32, device="cuda")
        pp = torch.empty_like(o)
        outs.append((o, pp))
        plain_outs.append((torch.empty_like(o), torch.empty_like(o)))
        jobs.append(gr.gr_job(g=Gs[gi].handle, op=op, src=src, out=o.data_ptr(),
                              pred=pp.data_ptr()))
    b0 = gr.gr_batch_create(jobs)                       # library defaults
    t0 = _events_ms(lambda: gr.gr_batch_run(b0), reps)
    ok = gr.gr_batch_status(b0)[0] == 0
    gr.gr_batch_destroy(b0)
    by_handle = {G.handle: G for G in Gs}
    best_opts, _, chosen = tune.tune_batch_strategy(jobs, by_handle, reps=2)
    b = gr.gr_batch_create(jobs, gr.batch_opts(**best_opts))
    ts = _events_ms(lambda: gr.gr_batch_run(b), reps)
    ok = ok and gr.gr_batch_status(b)[0] == 0
    info = gr.gr_batch_info(b)
    gr.gr_batch_destroy(b)

    def plain():
        for (gi, op, src), (o, pp) in zip(triples, plain_outs):
            if op == wl.OP_BFS:
                gr.gr_bfs(Gs[gi].handle, src, o, pp)
            else:
                gr.gr_sssp(Gs[gi].handle, src, o, pp)
    tp = _events_ms(plain, max(1, reps // 2), warm=1)
    same = ok
    for (gi, op, src), (o, pp), (o2, pp2) in zip(triples, outs, plain_outs):
        same = same and bool(torch.equal(o, o2))
        if op == wl.OP_SSSP:                # canonical predecessors (BFS trees may differ)
            same = same and bool(torch.equal(pp, pp2))
    same = same and all(G.sync_status() == gr.GR_OK for G in Gs)
    for G in Gs:
        G.close()
    ms, mp = statistics.median(ts), statistics.median(tp)
    return {"workload": "512 BFS/SSSP jobs (50/50) over 64 R-MAT graphs, scale U{10..18}, ef "
                        "U{8..32}, weights U[1,64]; one persistent launch replayed from a CUDA "
                        "graph; launch shape and per-level strategy from the batch autotuner",
            "ms": ms, "jobs_per_s": 512 / ms * 1e3, "batch_opts": best_opts, "tuned": chosen,
            "info": info,
            "library_defaults": {"ms": statistics.median(t0),
                                 "jobs_per_s": 512 / statistics.median(t0) * 1e3},
            "plain_path": {"ms": mp, "jobs_per_s": 512 / mp * 1e3},
            "speedup_vs_plain": mp / ms, "results_identical": same}


def measure_serve(gr, rates, requests):
    """Poisson BFS/SSSP requests over 8 resident graphs through the serving loop, and the same
    trace one query at a time on the plain path; every result must be identical."""
    import numpy as np

    from graphgen import workloads as wl
    from paper_1701_01170_gb300 import serve
    graphs = {name: gr.Graph.from_csr(g) for name, g in wl.serving_graphs()}
    cands = {name: np.flatnonzero(np.diff(G.R.cpu().numpy()) > 0) for name, G in graphs.items()}
    # BFS requests on the low-diameter R-MAT graphs are grouped into bit-parallel
    # multi-source units (a few levels, each O(n)); the grids' thousands of levels make
    # that O(n x levels), so their queries run alone on capped grids side by side
    multi = [n for n in graphs if n.startswith("rmat")]
    lanes = 4
    be = serve.GpuBackend(graphs, lanes, blocks_per_sm=1)
    be.prepare_multi(multi)
    caps = be.calibrate([n for n in graphs if not n.startswith("rmat")],
                        {n: int(cands[n][0]) for n in graphs})
    budget = 96 << 30     # per-lane workspaces; the graphs themselves take about 9 GB
    names = sorted(graphs)
    results = []
    for rate in rates:
        def src_of(name, rng):
            c = cands[name]
            return c[int(rng.integers(0, len(c)))]
        trace = serve.poisson_trace(names, rate, requests, 6, src_of)
        st = serve.serve_trace(be, trace, lanes, budget, multi_names=multi)
        trace2 = serve.poisson_trace(names, rate, requests, 6, src_of)
        st2 = serve.serve_serial(be, trace2)
        same = all(np.array_equal(a.result, b.result) for a, b in zip(
            sorted(trace, key=lambda r: r.rid), sorted(trace2, key=lambda r: r.rid)))
        results.append({"rate": rate, "served": st, "serial": st2, "results_identical": same,
                        "speedup_vs_serial": (st["queries_per_s"] or 0) /
                                             max(1e-9, st2["queries_per_s"] or 0)})
    be.close()
    for G in graphs.values():
        G.close()
    return {"workload": "serving: 8 resident graphs (R-MAT s18/20/22/24 ef16, grids "
                        "1024^2..8192^2), Poisson BFS/SSSP 50/50, random sources, "
                        f"{requests} requests per rate, {lanes} lanes, 96 GB workspace budget, "
                        "R-MAT BFS grouped into multi-source units; serial = the same trace "
                        "one query at a time on the plain path",
            "cta_caps": caps, "per_rate": results,
            "results_identical": all(r["results_identical"] for r in results)}


def main():
    args = parse_args()
    if args.workload != "s22":
        run_other(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
