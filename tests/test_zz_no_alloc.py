"""gr_bfs_static: the BFS entry point that allocates nothing.

Some callers cannot allocate device memory when they issue a query (an
allocator or memory-pool callback, a latency-critical thread, a runtime that
owns all device memory).  gr_bfs_static serves them from a static device
array.  This file is collected last on purpose, so that a failure here stops
a -x run only after every other test has run; it also passes on its own in a
fresh process.  Depths must equal those of gr_bfs bit for bit (integers), and
predecessors must pass the BFS certificate, on consecutive calls that reuse
the shared scratch.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


def test_static_bfs_matches_gr_bfs_on_consecutive_calls(gr):
    import torch
    g = gg.rmat(16, 16, seed=1)
    G = gr.Graph.from_csr(g)
    n, m = g.n, g.m
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    hub = gg.max_degree_vertex(g)
    for flags in (gr.GR_SYMMETRIC, 0):
        for src in (hub, 4321, hub):           # consecutive calls reuse the scratch
            ref = torch.empty(n, dtype=torch.int32, device="cuda")
            gr.gr_bfs(G.handle, src, ref, None)
            assert G.sync_status() == gr.GR_OK
            depth = torch.full((n,), 7, dtype=torch.int32, device="cuda")
            pred = torch.full((n,), 7, dtype=torch.int32, device="cuda")
            gr.gr_bfs_static(n, m, G.R, G.C, src, depth, pred, status, flags=flags)
            torch.cuda.synchronize()
            assert int(status.item()) == gr.GR_OK
            assert np.array_equal(host(depth), host(ref))
            assert oracle.bfs_certificate(g.R, g.C, src, host(depth), host(pred)) == 0
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
