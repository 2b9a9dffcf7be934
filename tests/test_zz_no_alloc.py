"""gr_bfs_static: the BFS entry point that allocates nothing.

Some callers cannot allocate device memory when they issue a query (an
allocator or memory-pool callback, a latency-critical thread, a runtime that
owns all device memory).  gr_bfs_static serves them from a static device
array.  This file is collected last on purpose, so that a failure here stops
a -x run only after every other test has run; it also passes on its own in a
fresh process.  Depths must equal the oracle's (and gr_bfs's) bit for bit
(integers), and predecessors must pass the BFS certificate, on consecutive
calls that reuse the shared scratch.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import host, star_plus

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


def static_bfs(gr, G, g, src, flags):
    import torch
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    depth = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    pred = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    gr.gr_bfs_static(g.n, g.m, G.R, G.C, src, depth, pred, status, flags=flags)
    torch.cuda.synchronize()
    assert int(status.item()) == gr.GR_OK
    return host(depth), host(pred)


def test_static_bfs_matches_the_oracle_on_consecutive_calls(gr):
    import torch
    g = gg.rmat(16, 16, seed=1)
    G = gr.Graph.from_csr(g)
    hub = gg.max_degree_vertex(g)
    for flags in (gr.GR_SYMMETRIC, 0):
        for src in (hub, 4321, hub):           # consecutive calls reuse the scratch
            ref = torch.empty(g.n, dtype=torch.int32, device="cuda")
            gr.gr_bfs(G.handle, src, ref, None)
            assert G.sync_status() == gr.GR_OK
            depth, pred = static_bfs(gr, G, g, src, flags)
            want, _ = oracle.bfs(g.R, g.C, src)
            assert np.array_equal(depth, want)
            assert np.array_equal(depth, host(ref))
            assert oracle.bfs_certificate(g.R, g.C, src, depth, pred) == 0
    G.close()


def test_static_bfs_shares_long_pull_rows(gr):
    # from the second hub, the first hub's 300,000-entry row has no frontier
    # neighbour on the first pull level: the static scratch's deferred list
    # spreads it over the grid, and its later match must still be exact
    g = star_plus(300_000)
    G = gr.Graph.from_csr(g)
    for src in (g.n - 1, 0, 1, g.n - 1):
        depth, pred = static_bfs(gr, G, g, src, gr.GR_SYMMETRIC)
        want, _ = oracle.bfs(g.R, g.C, src)
        assert np.array_equal(depth, want)
        assert oracle.bfs_certificate(g.R, g.C, src, depth, pred) == 0
    G.close()


@pytest.mark.slow
def test_static_bfs_near_its_limits(gr):
    # n = 2^20 (the vertex limit), m = 31.4 M (below the 2^25 edge limit), and the
    # hub's row of tens of thousands of edges goes through the chunk lists
    g = gg.rmat(20, 16, seed=1)
    assert g.n == gr.GR_STATIC_MAX_VERTICES and g.m <= gr.GR_STATIC_MAX_EDGES
    assert int(g.degrees().max()) >= 1024
    G = gr.Graph.from_csr(g)
    hub = gg.max_degree_vertex(g)
    for flags, src in ((gr.GR_SYMMETRIC, hub), (0, hub), (gr.GR_SYMMETRIC, 12345)):
        depth, pred = static_bfs(gr, G, g, src, flags)
        want, _ = oracle.bfs(g.R, g.C, src)
        assert np.array_equal(depth, want)
        assert oracle.bfs_certificate(g.R, g.C, src, depth, pred) == 0
    G.close()


def test_static_bfs_rejects_inputs_beyond_its_limits(gr):
    import torch
    R = torch.zeros(2, dtype=torch.int32, device="cuda")
    C = torch.zeros(1, dtype=torch.int32, device="cuda")
    d = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gr.GrError) as e:
        gr.gr_bfs_static(gr.GR_STATIC_MAX_VERTICES + 1, 0, R, C, 0, d)
    assert e.value.status == gr.GR_ERR_CAPACITY
    with pytest.raises(gr.GrError) as e:
        gr.gr_bfs_static(1, gr.GR_STATIC_MAX_EDGES + 1, R, C, 0, d)
    assert e.value.status == gr.GR_ERR_CAPACITY
