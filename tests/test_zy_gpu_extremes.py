"""GPU parity on the adversarial extremes: a hub with 10^6 leaves and a path of 10^5 vertices.

The hub row is cut into thousands of edge chunks shared by the whole grid; the
path runs one frontier vertex per level for 10^5 levels (BFS) or steps (SSSP),
so every level pays the grid barrier.  Depths and distances must equal the
oracle's, predecessors the canonical ones (SSSP) or a valid tree (BFS).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import host, star_plus, undirected

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


def extremes():
    hub = star_plus(1_000_000)
    k = 100_000
    path = undirected(k, np.stack([np.arange(k - 1), np.arange(1, k)], 1))
    return [(hub, (0, 1, hub.n - 1)), (path, (0, k // 2))]


def test_bfs_extremes(gr):
    import torch
    for g, srcs in extremes():
        G = gr.Graph.from_csr(g)
        depth = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pred = torch.empty_like(depth)
        for src in srcs:
            want, _ = oracle.bfs(g.R, g.C, src)
            for direction in (0, 1):
                gr.gr_bfs(G.handle, src, depth, pred, gr.bfs_opts(direction=direction))
                assert G.sync_status() == gr.GR_OK
                d, p = host(depth), host(pred)
                assert np.array_equal(d, want)
                assert oracle.bfs_certificate(g.R, g.C, src, d, p) == 0
        G.close()


def test_sssp_extremes(gr):
    import torch
    for g, srcs in extremes():
        g.W = gg.weights(g, 1, 64, seed=9)
        G = gr.Graph.from_csr(g)
        dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
        pred = torch.empty_like(dist)
        for src in srcs:
            want, _, over = oracle.dijkstra(g.R, g.C, g.W, src)
            assert not over
            gr.gr_sssp(G.handle, src, dist, pred)
            assert G.sync_status() == gr.GR_OK
            d, p = host(dist, np.uint32), host(pred)
            assert np.array_equal(d, want)
            assert np.array_equal(p, oracle.sssp_min_parent(g.R, g.C, g.W, want, src))
        G.close()
