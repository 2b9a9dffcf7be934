"""GPU parity of the standalone operators (gr_advance, gr_filter) against the CPU oracle.

Sizes span several scan tiles (4096 items) and warps with ragged tails; the
frontiers include the highest-degree vertex so that output-balanced
partitioning crosses row boundaries inside a warp.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import dev, empty_i32, host, len_tensor, pack_keys, undirected, unpack_keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def rmat14(gr):
    g = gg.rmat_weighted(14, 16, seed=1)
    return g, gr.Graph.from_csr(g)


def frontier(g, k, seed, dup=True):
    rng = np.random.default_rng(seed)
    f = rng.integers(0, g.n, k).astype(np.int32)
    if dup:
        f[::7] = f[0]
    f[k // 2] = gg.max_degree_vertex(g)
    return f


@pytest.mark.parametrize("k", [1, 31, 33, 4095, 4097, 20000])
@pytest.mark.parametrize("edges", [False, True])
def test_advance_ordered_exact(gr, rmat14, k, edges):
    g, G = rmat14
    F = frontier(g, k, seed=k)
    want = oracle.advance(g.R, g.C, F, edge_ids=edges)
    out = empty_i32(len(want))
    ol = len_tensor()
    gr.gr_advance(G.handle, dev(F), len(F), out, ol, mode=gr.GR_V2E if edges else gr.GR_V2V)
    assert G.sync_status() == 0
    assert int(ol.item()) == len(want)
    assert np.array_equal(host(out)[:len(want)], want)


def test_advance_device_length_and_capacity(gr, rmat14):
    g, G = rmat14
    F = frontier(g, 5000, seed=3)
    used = 3000
    want = oracle.advance(g.R, g.C, F[:used])
    out = empty_i32(len(want))
    ol = len_tensor()
    ld = dev(np.array([used], np.int64))
    gr.gr_advance(G.handle, dev(F), len(F), out, ol, in_len_dev=ld)
    assert G.sync_status() == 0
    assert int(ol.item()) == len(want) and np.array_equal(host(out)[:len(want)], want)
    # too small an output: the first cap items are written, the full count reported
    cap = len(want) // 3
    out2 = empty_i32(cap)
    gr.gr_advance(G.handle, dev(F), len(F), out2, ol, in_len_dev=ld, out_cap=cap)
    assert G.sync_status() == gr.GR_ERR_CAPACITY
    assert int(ol.item()) == len(want)
    assert np.array_equal(host(out2)[:cap], want[:cap])


def test_advance_empty_input(gr, rmat14):
    _, G = rmat14
    ol = len_tensor() + 5
    gr.gr_advance(G.handle, None, 0, empty_i32(1), ol)
    assert int(ol.item()) == 0


@pytest.mark.parametrize("idempotent", [False, True])
def test_advance_bfs_visit(gr, rmat14, idempotent):
    g, G = rmat14
    src = gg.max_degree_vertex(g)
    d_ref, _ = oracle.bfs(g.R, g.C, src)
    level = 1
    # state after level 1: vertices at depth <= 1 visited
    depth0 = np.where((d_ref >= 0) & (d_ref <= level), d_ref, -1).astype(np.int32)
    pred0 = np.full(g.n, -1, np.int32)
    F = np.flatnonzero(d_ref == level).astype(np.int32)
    want, want_depth, _ = oracle.advance_bfs(g.R, g.C, F, level, depth0, pred0)
    depth, pred = dev(depth0), dev(pred0)
    st = gr.gr_bfs_state(depth=depth.data_ptr(), pred=pred.data_ptr(), level=level)
    out = empty_i32(g.m)
    ol = len_tensor()
    mode = gr.GR_IDEMPOTENT if idempotent else 0
    gr.gr_advance(G.handle, dev(F), len(F), out, ol, mode=mode, functor=gr.GR_FN_BFS_VISIT,
                  state=st)
    assert G.sync_status() == 0
    got = host(out)[:int(ol.item())]
    if idempotent:
        assert np.array_equal(np.unique(got), np.sort(want))
    else:
        assert np.array_equal(np.sort(got), np.sort(want))  # each vertex exactly once
    assert np.array_equal(host(depth), want_depth)
    p = host(pred)
    for v in np.sort(want)[:: max(1, len(want) // 500)]:   # parent is a frontier neighbour
        assert d_ref[p[v]] == level and v in g.C[g.R[p[v]]:g.R[p[v] + 1]]


def test_advance_pull_exact(gr, rmat14):
    g, G = rmat14
    src = 0
    d_ref, _ = oracle.bfs(g.R, g.C, src)
    for level in range(0, int(d_ref.max())):
        depth0 = np.where((d_ref >= 0) & (d_ref <= level), d_ref, -1).astype(np.int32)
        pred0 = np.full(g.n, -1, np.int32)
        cand = oracle.filter_unvisited(depth0)
        act, _, want_depth, want_pred = oracle.pull(g.R, g.C, cand, level, depth0, pred0)
        depth, pred = dev(depth0), dev(pred0)
        st = gr.gr_bfs_state(depth=depth.data_ptr(), pred=pred.data_ptr(), level=level)
        out = empty_i32(len(cand))
        ol = len_tensor()
        gr.gr_advance(G.handle, dev(cand), len(cand), out, ol, mode=gr.GR_PULL,
                      functor=gr.GR_FN_BFS_VISIT, state=st)
        assert G.sync_status() == 0
        assert np.array_equal(host(out)[:int(ol.item())], act)
        assert np.array_equal(host(depth), want_depth)
        assert np.array_equal(host(pred), want_pred)


def test_advance_relax(gr, rmat14):
    g, G = rmat14
    src = gg.max_degree_vertex(g)
    final, _, _ = oracle.dijkstra(g.R, g.C, g.W, src)
    canon = oracle.sssp_min_parent(g.R, g.C, g.W, final, src)
    fin = final.astype(np.int64)
    for lo, hi in [(0, 1), (1, 20), (20, 40), (40, 80)]:
        settled = fin < hi
        dist0 = np.where(settled, final, oracle.INF32).astype(np.uint32)
        pred0 = np.where(settled, canon, -1).astype(np.int32)
        F = np.flatnonzero((fin >= lo) & (fin < hi)).astype(np.int32)
        want, wd, wp = oracle.advance_relax(g.R, g.C, g.W, F, dist0, pred0)
        keys = dev(pack_keys(dist0, pred0))
        st = gr.gr_sssp_state(key=keys.data_ptr(), threshold=0)
        out = empty_i32(g.m)
        ol = len_tensor()
        gr.gr_advance(G.handle, dev(F), len(F), out, ol, functor=gr.GR_FN_SSSP_RELAX, state=st)
        assert G.sync_status() == 0
        got = host(out)[:int(ol.item())]
        assert np.array_equal(np.unique(got), want)
        d, p = unpack_keys(host(keys))
        assert np.array_equal(d, wd) and np.array_equal(p, wp)


def test_relax_overflow_is_reported(gr):
    g = undirected(3, [(0, 1), (1, 2)])
    g.W = np.full(g.m, 2**31 + 5, np.uint32)
    G = gr.Graph.from_csr(g)
    keys = dev(pack_keys(np.array([0, 2**31 + 5, 2**32 - 1], np.uint64), [-1, 0, -1]))
    st = gr.gr_sssp_state(key=keys.data_ptr(), threshold=0)
    ol = len_tensor()
    gr.gr_advance(G.handle, dev(np.array([1], np.int32)), 1, empty_i32(4), ol,
                  functor=gr.GR_FN_SSSP_RELAX, state=st)
    assert G.sync_status() == gr.GR_ERR_OVERFLOW


@pytest.mark.parametrize("k", [1, 4095, 4096, 4097, 30000])
def test_filter_exact_unique(gr, rmat14, k):
    g, G = rmat14
    rng = np.random.default_rng(k)
    items = rng.integers(-5, g.n + 5, k).astype(np.int32)
    items[::3] = items[0]
    want = oracle.filter_unique(g.n, items)
    out = empty_i32(k)
    ol = len_tensor()
    for _ in range(2):  # the second call checks the scratch was left clean
        gr.gr_filter(G.handle, dev(items), k, out, ol, mode=gr.GR_FILTER_EXACT_UNIQUE)
        assert G.sync_status() == 0
        assert np.array_equal(host(out)[:int(ol.item())], want)


def test_filter_cull_contract(gr, rmat14):
    g, G = rmat14
    rng = np.random.default_rng(7)
    items = rng.integers(-3, g.n + 3, 50000).astype(np.int32)
    items[::2] = rng.integers(0, 100, 25000)
    out = empty_i32(len(items))
    ol = len_tensor()
    for _ in range(2):
        gr.gr_filter(G.handle, dev(items), len(items), out, ol, mode=gr.GR_FILTER_CULL)
        assert G.sync_status() == 0
        got = host(out)[:int(ol.item())]
        valid = items[(items >= 0) & (items < g.n)]
        assert set(got.tolist()) == set(valid.tolist())
        cg = np.bincount(got, minlength=g.n)
        ci = np.bincount(valid, minlength=g.n)
        assert (cg <= ci).all()


def test_filter_unvisited(gr, rmat14):
    g, G = rmat14
    rng = np.random.default_rng(9)
    depth0 = rng.integers(-1, 3, g.n).astype(np.int32)
    depth = dev(depth0)
    st = gr.gr_bfs_state(depth=depth.data_ptr(), pred=0, level=0)
    out = empty_i32(g.n)
    ol = len_tensor()
    gr.gr_filter(G.handle, None, 0, out, ol, mode=gr.GR_FILTER_UNVISITED, state=st)
    assert G.sync_status() == 0
    assert np.array_equal(host(out)[:int(ol.item())], oracle.filter_unvisited(depth0))


@pytest.mark.parametrize("k", [1, 4097, 40000])
def test_filter_near_far(gr, rmat14, k):
    g, G = rmat14
    rng = np.random.default_rng(k + 1)
    dist0 = rng.integers(0, 200, g.n).astype(np.uint32)
    dist0[::11] = oracle.INF32
    keys = dev(pack_keys(dist0, np.full(g.n, -1)))
    items = rng.integers(-2, g.n + 2, k).astype(np.int32)
    near_w, far_w = oracle.filter_near_far(g.n, items, dist0, 100)
    st = gr.gr_sssp_state(key=keys.data_ptr(), threshold=100)
    near, far = empty_i32(k), empty_i32(k)
    nl, fl = len_tensor(), len_tensor()
    gr.gr_filter(G.handle, dev(items), k, near, nl, mode=gr.GR_FILTER_NEAR_FAR, state=st,
                 far=far, far_len=fl)
    assert G.sync_status() == 0
    assert np.array_equal(host(near)[:int(nl.item())], near_w)
    assert np.array_equal(host(far)[:int(fl.item())], far_w)


@pytest.mark.parametrize("k", [1, 4097, 40000])
@pytest.mark.parametrize("buckets,base,delta", [(2, 0, 100), (8, 30, 17), (5, 250, 1),
                                                (8, 0, 1 << 31)])
def test_filter_multisplit(gr, rmat14, k, buckets, base, delta):
    import torch
    g, G = rmat14
    rng = np.random.default_rng(k + buckets)
    dist0 = rng.integers(0, 400, g.n).astype(np.uint32)
    dist0[::13] = oracle.INF32
    keys = dev(pack_keys(dist0, np.full(g.n, -1)))
    items = rng.integers(-2, g.n + 2, k).astype(np.int32)
    want, want_len = oracle.multisplit(g.n, items, dist0, base, delta, buckets)
    blen = torch.full((buckets,), -7, dtype=torch.int64, device="cuda")
    st = gr.gr_multisplit_state(key=keys.data_ptr(), base=base, delta=delta, buckets=buckets,
                                bucket_len=blen.data_ptr())
    out, ol = empty_i32(k), len_tensor()
    gr.gr_filter(G.handle, dev(items), k, out, ol, mode=gr.GR_FILTER_MULTISPLIT, state=st)
    assert G.sync_status() == 0
    assert int(ol.item()) == len(want)
    assert np.array_equal(host(out)[:len(want)], want)
    assert np.array_equal(host(blen), want_len)
    if buckets == 2 and base == 0:               # two buckets: the near/far split
        near, far = oracle.filter_near_far(g.n, items, dist0, delta)
        assert np.array_equal(want, np.concatenate([near, far]))


def test_filter_multisplit_rejects_bad_states(gr, rmat14):
    import torch
    g, G = rmat14
    keys = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    blen = torch.zeros(9, dtype=torch.int64, device="cuda")
    out, ol = empty_i32(4), len_tensor()
    items = dev(np.arange(4, dtype=np.int32))
    for buckets, delta in ((1, 5), (9, 5), (4, 0)):
        st = gr.gr_multisplit_state(key=keys.data_ptr(), base=0, delta=delta, buckets=buckets,
                                    bucket_len=blen.data_ptr())
        with pytest.raises(gr.GrError):
            gr.gr_filter(G.handle, items, 4, out, ol, mode=gr.GR_FILTER_MULTISPLIT, state=st)


def test_operators_compose_into_bfs(gr, rmat14):
    """advance(BFS_VISIT, idempotent) + filter(EXACT_UNIQUE) per level == queue BFS."""
    g, G = rmat14
    import torch
    src = 5
    depth = dev(np.where(np.arange(g.n) == src, 0, -1).astype(np.int32))
    pred = dev(np.full(g.n, -1, np.int32))
    F = dev(np.array([src], np.int32))
    flen = 1
    level = 0
    buf = empty_i32(g.m)
    ol = len_tensor()
    while flen:
        st = gr.gr_bfs_state(depth=depth.data_ptr(), pred=pred.data_ptr(), level=level)
        gr.gr_advance(G.handle, F, flen, buf, ol, mode=gr.GR_IDEMPOTENT,
                      functor=gr.GR_FN_BFS_VISIT, state=st)
        n_adv = int(ol.item())
        nxt = empty_i32(n_adv)
        gr.gr_filter(G.handle, buf, n_adv, nxt, ol, mode=gr.GR_FILTER_EXACT_UNIQUE)
        flen = int(ol.item())
        F = nxt
        level += 1
    assert G.sync_status() == 0
    want, _ = oracle.bfs(g.R, g.C, src)
    assert np.array_equal(host(depth), want)
    assert oracle.bfs_certificate(g.R, g.C, src, want, host(pred)) == 0
    torch.cuda.synchronize()


@pytest.mark.slow
def test_config_s22_hub_neighbourhood(gr):
    # the operator workload the benchmark times: advance of the hub's 162,948 rows of
    # R-MAT s22 (84.7 M edges), then both deduplicating filters of that output
    g = gg.rmat_weighted(22, 16, 2, 1, 64)
    G = gr.Graph.from_csr(g)
    hub = gg.max_degree_vertex(g)
    F = np.ascontiguousarray(g.C[g.R[hub]:g.R[hub + 1]])
    want = oracle.advance(g.R, g.C, F)
    out = empty_i32(len(want))
    ol = len_tensor()
    gr.gr_advance(G.handle, dev(F), len(F), out, ol)
    assert G.sync_status() == 0
    assert int(ol.item()) == len(want)
    assert np.array_equal(host(out), want)
    uniq = oracle.filter_unique(g.n, want)
    uo = empty_i32(g.n)
    gr.gr_filter(G.handle, out, len(want), uo, ol, mode=gr.GR_FILTER_EXACT_UNIQUE)
    assert G.sync_status() == 0
    assert np.array_equal(host(uo)[:int(ol.item())], uniq)
    gr.gr_filter(G.handle, out, len(want), uo, ol, mode=gr.GR_FILTER_CULL)
    assert G.sync_status() == 0
    got = host(uo)[:int(ol.item())]
    assert len(got) == len(uniq) and np.array_equal(np.sort(got), np.sort(uniq))
    G.close()
