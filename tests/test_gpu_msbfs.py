"""GPU parity of gr_bfs_multi (bit-parallel multi-source BFS) against k oracle BFS runs.

Every depth row must equal the oracle's queue BFS from that source, bit for
bit.  Cases cover word boundaries of the bit masks (64, 65, 128, 256, 257
sources), duplicate sources, push-only and pull-only schedules, a directed
graph, and a high-diameter grid whose level count forces the snapshot
buffer to grow; concurrent calls on one graph from several threads.
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


def run_multi(gr, G, srcs, **opts):
    import torch
    depth = torch.full((len(srcs) * G.n,), -7, dtype=torch.int32, device="cuda")
    o = gr.msbfs_opts(**opts) if opts else None
    gr.gr_bfs_multi(G.handle, srcs, depth, o)
    torch.cuda.synchronize()
    return host(depth).reshape(len(srcs), G.n)


@pytest.fixture(scope="module")
def s13(gr):
    g = gg.rmat(13, 16, seed=3)
    return g, gr.Graph.from_csr(g)


@pytest.mark.parametrize("k", [1, 3, 64, 65, 128, 129, 256, 257])
def test_matches_independent_bfs(gr, s13, k):
    g, G = s13
    srcs = gg.sources(g, min(k, 300), seed=k)
    srcs = np.resize(srcs, k)
    got = run_multi(gr, G, srcs)
    assert np.array_equal(got, oracle.bfs_multi(g.R, g.C, srcs))


@pytest.mark.parametrize("direction", [1, 2])
def test_push_only_and_pull_only(gr, s13, direction):
    g, G = s13
    srcs = np.concatenate([[0, 0], gg.sources(g, 70, seed=7)])   # includes a duplicate
    got = run_multi(gr, G, srcs, direction=direction)
    assert np.array_equal(got, oracle.bfs_multi(g.R, g.C, srcs))


@pytest.mark.parametrize("ratio", [0.0, 1e-4, 1.0, 1e9])
def test_switch_ratio_does_not_change_results(gr, s13, ratio):
    g, G = s13
    srcs = gg.sources(g, 40, seed=9)
    assert np.array_equal(run_multi(gr, G, srcs, push_ratio=ratio),
                          oracle.bfs_multi(g.R, g.C, srcs))


@pytest.mark.parametrize("keep", [2, 3, 5])
def test_deep_mode_writes_depths_directly(gr, s13, keep):
    # after `keep` snapshot levels the depths of later levels are written as
    # their bits appear; the matrix must not change
    g, G = s13
    srcs = np.concatenate([[0, 0], gg.sources(g, 90, seed=11)])
    got = run_multi(gr, G, srcs, snapshot_levels=keep)
    assert np.array_equal(got, oracle.bfs_multi(g.R, g.C, srcs))
    m = gg.grid(48, 0.1, seed=3)
    M = gr.Graph.from_csr(m)
    msrcs = np.array([0, m.n - 1, m.n // 2, 17, 17], np.int32)
    for direction in (0, 1):
        got = run_multi(gr, M, msrcs, snapshot_levels=keep, direction=direction)
        assert np.array_equal(got, oracle.bfs_multi(m.R, m.C, msrcs))
    M.close()


def test_high_diameter_grid_grows_snapshots(gr):
    g = gg.grid(48, 0.1, seed=3)
    G = gr.Graph.from_csr(g)
    srcs = np.array([0, g.n - 1, g.n // 2, 17], np.int32)
    got = run_multi(gr, G, srcs)
    want = oracle.bfs_multi(g.R, g.C, srcs)
    assert want.max() > 40
    assert np.array_equal(got, want)


def test_directed_graph_uses_push(gr):
    rng = np.random.default_rng(11)
    n = 2000
    s, t = rng.integers(0, n, 9000), rng.integers(0, n, 9000)
    keep = s != t
    pairs = np.unique(np.stack([s[keep], t[keep]], 1), axis=0)
    g = gg.directed(n, pairs[:, 0], pairs[:, 1])
    G = gr.Graph.from_csr(g, symmetric=False)
    srcs = np.arange(0, 100, 3, dtype=np.int32)
    assert np.array_equal(run_multi(gr, G, srcs), oracle.bfs_multi(g.R, g.C, srcs))


def test_concurrent_calls_on_one_graph(gr, s13):
    # the multi-source scratch is per graph: calls from several host threads
    # on their own streams must be serialised by the library, each one
    # returning its own sources' depths
    import threading

    import torch
    g, G = s13
    sets = [gg.sources(g, k, seed=40 + i) for i, k in enumerate((5, 64, 70, 200))]
    want = [oracle.bfs_multi(g.R, g.C, srcs) for srcs in sets]
    got = [None] * len(sets)
    errors = []

    def worker(i):
        try:
            stream = torch.cuda.Stream()
            ok = True
            with torch.cuda.stream(stream):
                depth = torch.empty(len(sets[i]) * G.n, dtype=torch.int32, device="cuda")
                for _ in range(3):
                    depth.fill_(-7)
                    gr.gr_bfs_multi(G.handle, sets[i], depth, None, stream)
                    h = host(depth).reshape(len(sets[i]), G.n)
                    ok = ok and np.array_equal(h, want[i])
            got[i] = ok
        except Exception as e:  # reported below, on the test's thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(sets))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert got == [True] * len(sets)


def test_rejects_bad_sources(gr, s13):
    import torch
    g, G = s13
    d = torch.empty(2 * g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(gr.GrError):
        gr.gr_bfs_multi(G.handle, [0, g.n], d)


@pytest.mark.slow
def test_config_s20_256_sources(gr):
    g = gg.rmat(20, 16, seed=1)
    G = gr.Graph.from_csr(g)
    srcs = gg.sources(g, 256, seed=4)
    got = run_multi(gr, G, srcs)
    for i in list(range(0, 256, 17)) + [255]:        # sampled rows, each a full oracle BFS
        want, _ = oracle.bfs(g.R, g.C, int(srcs[i]))
        assert np.array_equal(got[i], want)
    # every row: the source at depth 0, and on an undirected graph the
    # distance matrix between the sources is symmetric
    assert (got[np.arange(256), srcs] == 0).all()
    between = got[:, srcs]
    assert np.array_equal(between, between.T)
    G.close()
