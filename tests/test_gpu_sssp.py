"""GPU parity of gr_sssp (persistent SSSP with a multi-level or near/far priority queue)
against the CPU oracle.

Distances must equal Dijkstra's bit for bit.  Predecessors are the
smallest-id tight predecessor (the packed 64-bit atomicMin makes them
unique), so they are compared element-wise with the oracle's canonical
parents, and must also pass the SSSP certificate.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import host, star_plus, undirected

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


def run_sssp(gr, G, src, expect=0, **opts):
    import torch
    dist = torch.empty(G.n, dtype=torch.int32, device="cuda")
    pred = torch.empty_like(dist)
    o = gr.sssp_opts(**opts) if opts else None
    gr.gr_sssp(G.handle, src, dist, pred, o)
    st = G.sync_status()
    assert st == expect, gr.status_str(st)
    return host(dist, np.uint32), host(pred)


def check(g, src, dist, pred):
    want, _, over = oracle.dijkstra(g.R, g.C, g.W, src)
    assert not over
    assert np.array_equal(dist, want)
    assert np.array_equal(pred, oracle.sssp_min_parent(g.R, g.C, g.W, want, src))
    assert oracle.sssp_certificate(g.R, g.C, g.W, src, dist, pred) == 0


@pytest.fixture(scope="module")
def s16w(gr):
    g = gg.rmat_weighted(16, 16, seed=1)
    return g, gr.Graph.from_csr(g)


@pytest.mark.parametrize("delta", [0, 1, 2, 4, 7, 64, 1 << 30])
@pytest.mark.parametrize("levels", [0, 2])
def test_rmat_s16_deltas_agree(gr, s16w, delta, levels):
    # levels 0: multi-level queue (8 buckets); 2: near/far
    g, G = s16w
    for src in (gg.max_degree_vertex(g), 4321):
        d, p = run_sssp(gr, G, src, delta=delta, levels=levels)
        check(g, src, d, p)


def test_step_stats(gr, s16w):
    import torch
    g, G = s16w
    cap = 4096
    stats = torch.full((4 * cap,), -7, dtype=torch.int32, device="cuda")
    src = gg.max_degree_vertex(g)
    for delta, levels in ((7, 2), (64, 2), (7, 0), (64, 0)):
        stats.fill_(-7)
        d, p = run_sssp(gr, G, src, delta=delta, level_stats=stats.data_ptr(), max_levels=cap,
                        levels=levels)
        check(g, src, d, p)
        steps = gr.gr_last_run_stats(G.handle)["levels"]
        assert 0 < steps < cap
        s = host(stats).reshape(cap, 4)[:steps]
        assert s[0, 0] == 1 and s[0, 1] == 0 and s[0, 2] == 0    # the source alone
        split = s[:, 1] == 1
        assert (s[split, 0] == 0).all()
        if levels == 2:
            assert (s[split, 2] > 0).all()    # near/far splits drain the far pile
        assert (s[~split, 0] > 0).all()
        assert (np.diff(s[:, 3]) >= 0).all()
        end = host(stats).reshape(cap, 4)[steps]            # the loop's end row
        assert end[0] == 0 and end[1] == 0 and end[2] == 0 and end[3] >= s[-1, 3]
        assert (host(stats).reshape(cap, 4)[steps + 1:] == -7).all()


@pytest.mark.parametrize("bulk", [-1, 1, 4096])
@pytest.mark.parametrize("delta", [0, 3, 7, 1 << 30])
@pytest.mark.parametrize("levels", [0, 2])
def test_bulk_and_per_edge_steps_agree(gr, s16w, bulk, delta, levels):
    # bulk = 1: every relax step runs in bulk; -1: none does; 4096: mixed
    g, G = s16w
    for src in (gg.max_degree_vertex(g), 4321):
        d, p = run_sssp(gr, G, src, delta=delta, bulk_rows=bulk, levels=levels)
        check(g, src, d, p)


def test_queue_levels_validated(gr, s16w):
    g, G = s16w
    with pytest.raises(gr.GrError):
        run_sssp(gr, G, 0, levels=3)


@pytest.mark.parametrize("cap", [1, 7, 38])
def test_cta_cap_does_not_change_distances(gr, s16w, cap):
    g, G = s16w
    for src in (gg.max_degree_vertex(g), 4321):
        d, p = run_sssp(gr, G, src, max_blocks=cap)
        check(g, src, d, p)


@pytest.mark.parametrize("big", [32, 1 << 30])
def test_split_thresholds_agree(gr, s16w, big):
    g, G = s16w
    d, p = run_sssp(gr, G, 0, big_degree=big)
    check(g, 0, d, p)


def test_grid_small_wide_weights(gr):
    g = gg.grid_weighted(200, 0.1, seed=3)
    G = gr.Graph.from_csr(g)
    for delta in (0, 30, 100, 5000):
        for bulk in (0, 1):
            for levels in (0, 2):
                d, p = run_sssp(gr, G, 0, delta=delta, bulk_rows=bulk, levels=levels)
                check(g, 0, d, p)


def test_constant_weight_is_scaled_bfs(gr):
    g = gg.rmat(12, 8, seed=5)
    g.W = np.full(g.m, 3, np.uint32)
    G = gr.Graph.from_csr(g)
    d, p = run_sssp(gr, G, 0)
    depth, _ = oracle.bfs(g.R, g.C, 0)
    want = np.where(depth < 0, np.int64(oracle.INF32), 3 * depth.astype(np.int64))
    assert np.array_equal(d.astype(np.int64), want)
    check(g, 0, d, p)


def test_degenerate_graphs(gr):
    cases = [undirected(1, np.zeros((0, 2))), undirected(6, [(0, 1), (2, 3)])]
    for deg in (31, 33, 1023, 1025, 4000):
        cases.append(star_plus(deg))
    for g in cases:
        g.W = gg.weights(g, 1, 64, seed=4)
        G = gr.Graph.from_csr(g)
        for src in {0, g.n - 1}:
            for big in (32, 1024):
                for bulk in (-1, 1):
                    for delta in (0, 2):
                        d, p = run_sssp(gr, G, src, big_degree=big, bulk_rows=bulk, delta=delta)
                        check(g, src, d, p)
        G.close()


def test_overflow_detected(gr):
    g = undirected(4, [(0, 1), (1, 2), (2, 3)])
    g.W = np.full(g.m, 2**31, np.uint32)
    G = gr.Graph.from_csr(g)
    for bulk in (-1, 1):
        for delta in (0, 1):
            run_sssp(gr, G, 0, expect=gr.GR_ERR_OVERFLOW, bulk_rows=bulk, delta=delta)
    g.W = np.full(g.m, 2**30, np.uint32)
    G2 = gr.Graph.from_csr(g)
    for bulk in (-1, 1):
        for delta in (0, 1, 2**29):
            d, p = run_sssp(gr, G2, 0, bulk_rows=bulk, delta=delta)
            check(g, 0, d, p)


def test_sssp_needs_weights(gr):
    import torch
    g = gg.rmat(8, 4, seed=1)
    G = gr.Graph.from_csr(g)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(gr.GrError) as e:
        gr.gr_sssp(G.handle, 0, dist)
    assert e.value.status == gr.GR_ERR_UNSUPPORTED


@pytest.mark.slow
def test_config_s22_full_size(gr):
    g = gg.rmat_weighted(22, 16, seed=2)
    G = gr.Graph.from_csr(g)
    hub = gg.max_degree_vertex(g)
    d, p = run_sssp(gr, G, hub)
    check(g, hub, d, p)
    src = int(gg.sources(g, 1, seed=2)[0])
    d, p = run_sssp(gr, G, src)
    check(g, src, d, p)
    G.close()


@pytest.mark.slow
def test_config_grid4096_full_size(gr):
    g = gg.grid_weighted(4096, 0.1, seed=3)
    G = gr.Graph.from_csr(g)
    d, p = run_sssp(gr, G, 0)
    check(g, 0, d, p)
    G.close()
