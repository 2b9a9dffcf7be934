"""GPU parity of batched jobs (gr_batch_*): many BFS/SSSP jobs over many graphs in
one persistent launch must give, job by job, exactly the single-query results.

Depths and distances are compared with the oracle bit for bit; BFS
predecessors must pass the certificate and SSSP predecessors must equal the
oracle's smallest-id tight predecessors.  Every cluster size and both the
direct launch and the CUDA-graph replay are exercised, and replays must
reproduce the first run.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import host
from graphgen import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


def make_jobs(gr, graphs, triples):
    import torch
    handles = [gr.Graph.from_csr(g, symmetric=sym) for g, sym in graphs]
    jobs, outs = [], []
    for gi, op, src in triples:
        n = graphs[gi][0].n
        out = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        pred = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        jobs.append(gr.gr_job(g=handles[gi].handle, op=op, src=src, out=out.data_ptr(),
                              pred=pred.data_ptr()))
        outs.append((out, pred))
    return handles, jobs, outs


def check(graphs, triples, outs):
    for (gi, op, src), (out, pred) in zip(triples, outs):
        g = graphs[gi][0]
        o, p = host(out), host(pred)
        if op == wl.OP_BFS:
            want, _ = oracle.bfs(g.R, g.C, src)
            assert np.array_equal(o, want)
            assert oracle.bfs_certificate(g.R, g.C, src, o, p) == 0
        else:
            want, _, _ = oracle.dijkstra(g.R, g.C, g.W, src)
            d = o.view(np.uint32)
            assert np.array_equal(d, want)
            assert np.array_equal(p, oracle.sssp_min_parent(g.R, g.C, g.W, want, src))


def small_mix():
    graphs = []
    for i, (s, ef) in enumerate([(8, 8), (10, 16), (11, 4), (12, 24)]):
        graphs.append((gg.rmat_weighted(s, ef, seed=50 + i), True))
    graphs.append((gg.grid_weighted(40, 0.1, seed=3), True))
    rng = np.random.default_rng(2)
    n = 1500
    s_, t_ = rng.integers(0, n, 7000), rng.integers(0, n, 7000)
    keep = s_ != t_
    pairs = np.unique(np.stack([s_[keep], t_[keep]], 1), axis=0)
    d = gg.directed(n, pairs[:, 0], pairs[:, 1])
    d.W = rng.integers(1, 50, d.m).astype(np.uint32)
    graphs.append((d, False))
    triples = []
    for j in range(30):
        gi = j % len(graphs)
        g = graphs[gi][0]
        src = int(gg.sources(g, 8, seed=j)[j % 8])
        triples.append((gi, wl.OP_BFS if (j // len(graphs)) % 2 == 0 else wl.OP_SSSP, src))
    return graphs, triples


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_matches_single_queries(gr, cluster, use_graph):
    graphs, triples = small_mix()
    handles, jobs, outs = make_jobs(gr, graphs, triples)
    b = gr.gr_batch_create(jobs, gr.batch_opts(cluster_size=cluster, use_graph=use_graph))
    gr.gr_batch_run(b)
    st, per_job = gr.gr_batch_status(b, len(jobs))
    assert st == 0 and all(x == 0 for x in per_job)
    check(graphs, triples, outs)
    first = [(host(o).copy(), host(p).copy()) for o, p in outs]
    for o, p in outs:
        o.fill_(-9)
        p.fill_(-9)
    gr.gr_batch_run(b)                   # replay
    assert gr.gr_batch_status(b)[0] == 0
    for (o, p), (o0, p0) in zip(outs, first):
        assert np.array_equal(host(o), o0)
    gr.gr_batch_destroy(b)
    for h in handles:
        h.close()


def test_tuned_batch_matches_single_queries(gr):
    # the strategy tuner rewrites the jobs' knobs and the launch shape; the
    # results must not move
    from paper_1701_01170_gb300 import tune
    graphs, triples = small_mix()
    handles, jobs, outs = make_jobs(gr, graphs, triples)
    by_handle = {h.handle: h for h in handles}
    opts, ms, chosen = tune.tune_batch_strategy(jobs, by_handle, reps=1)
    assert ms > 0 and chosen["cluster_size"] in tune.BATCH_CLUSTERS
    for o, p in outs:
        o.fill_(-5)
        p.fill_(-5)
    b = gr.gr_batch_create(jobs, gr.batch_opts(**opts))
    gr.gr_batch_run(b)
    st, _ = gr.gr_batch_status(b, len(jobs))
    assert st == 0
    check(graphs, triples, outs)
    gr.gr_batch_destroy(b)
    for h in handles:
        h.close()


def test_batch_rejects_bad_jobs(gr):
    import torch
    g = gg.rmat(8, 4, seed=1)
    G = gr.Graph.from_csr(g)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    bad = [gr.gr_job(g=G.handle, op=gr.GR_OP_BFS, src=g.n, out=out.data_ptr())]
    with pytest.raises(gr.GrError):
        gr.gr_batch_create(bad)
    unweighted = [gr.gr_job(g=G.handle, op=gr.GR_OP_SSSP, src=0, out=out.data_ptr())]
    with pytest.raises(gr.GrError):
        gr.gr_batch_create(unweighted)


@pytest.mark.slow
def test_config_512_jobs_64_graphs(gr):
    bgs = wl.batch_graphs(64, seed=5)
    graphs = [(b.csr, True) for b in bgs]
    triples = wl.batch_jobs(bgs, 512, seed=5)
    handles, jobs, outs = make_jobs(gr, graphs, triples)
    b = gr.gr_batch_create(jobs, gr.batch_opts(cluster_size=2))
    gr.gr_batch_run(b)
    st, per_job = gr.gr_batch_status(b, len(jobs))
    assert st == 0
    # complete certificates for every job, exact oracle comparison for a sample
    for k, ((gi, op, src), (out, pred)) in enumerate(zip(triples, outs)):
        g = graphs[gi][0]
        o, p = host(out), host(pred)
        if op == wl.OP_BFS:
            assert oracle.bfs_certificate(g.R, g.C, src, o, p) == 0
        else:
            assert oracle.sssp_certificate(g.R, g.C, g.W, src, o.view(np.uint32), p) == 0
    sample = list(range(0, 512, 37))
    check(graphs, [triples[i] for i in sample], [outs[i] for i in sample])
    gr.gr_batch_destroy(b)
    for h in handles:
        h.close()
