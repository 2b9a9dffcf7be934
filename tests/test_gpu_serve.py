"""Serving on the GPU: every request's result is the same alone and in the mix.

A Poisson trace over eight small resident graphs (R-MAT and grids) runs
through the continuous-batching loop (several lanes overlapping, BFS
requests on the R-MAT graphs grouped into multi-source units, a memory
budget that forces evictions, released in each lane's stream order) and
through the serial plain path; each result must equal the CPU oracle's
answer for that request, and lanes must still overlap under evictions.
"""
import numpy as np
import pytest

import oracle
from graphgen import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_1701_01170_gb300 as gr
    from paper_1701_01170_gb300 import serve
    gr.load()
    csrs = dict(wl.serving_graphs(small=True))
    graphs = {name: gr.Graph.from_csr(g) for name, g in csrs.items()}
    return gr, serve, csrs, graphs


def expected(csr, op, src):
    if op == 1:
        return oracle.bfs(csr.R, csr.C, src)[0]
    return oracle.dijkstra(csr.R, csr.C, csr.W, src)[0].view(np.int32)


def test_served_results_equal_solo_results(setup):
    gr, serve, csrs, graphs = setup
    names = sorted(graphs)
    cands = {n: np.flatnonzero(np.diff(c.R) > 0) for n, c in csrs.items()}
    trace = serve.poisson_trace(names, 4000.0, 120, 6,
                                lambda name, rng: cands[name][int(rng.integers(0, len(cands[name])))])
    multi = [n for n in names if n.startswith("rmat")]
    be = serve.GpuBackend(graphs, lanes=3, blocks_per_sm=1)
    be.prepare_multi(multi)
    caps = be.calibrate([n for n in names if n not in multi],
                        {n: int(cands[n][0]) for n in names}, slack=1e9)
    assert all(c > 0 for c in caps.values())     # capped queries run side by side below
    infos = be.graph_infos(set(multi))
    # a budget below the sum of all workspaces: admission must evict and wait
    budget = sum(i.bytes_multi for i in infos.values() if i.multi_ok) + \
        2 * max(i.bytes_sssp for i in infos.values())
    stats = serve.serve_trace(be, trace, 3, budget, multi_names=multi)
    assert stats["completed"] == len(trace) and stats["errors"] == 0
    # the budget forced evictions (released in stream order), and lanes still overlapped:
    # some requests on different lanes ran at the same time
    assert stats["evictions"] > 0 and be.evicted > 0
    overlap = any(a.lane != b.lane and a.t_start < b.t_done and b.t_start < a.t_done
                  for a in trace for b in trace)
    assert overlap
    grouped = 0
    for r in trace:
        want = expected(csrs[r.graph], r.op, r.src)
        assert np.array_equal(r.result, want), (r.graph, r.op, r.src)
    serial = serve.poisson_trace(names, 4000.0, 40, 7,
                                 lambda name, rng: cands[name][int(rng.integers(0, len(cands[name])))])
    st2 = serve.serve_serial(be, serial)
    assert st2["completed"] == 40
    for r in serial:
        assert np.array_equal(r.result, expected(csrs[r.graph], r.op, r.src))
    be.close()
