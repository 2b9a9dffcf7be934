"""GPU parity of the segmented-intersection operator (Sec. 4.3) and of triangle
counting (Sec. 6.6) against the CPU oracle.  Everything here is integer work:
counts, items and triangle totals must equal the oracle's exactly."""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import dev, host, star_plus, undirected

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


def intersect(gr, G, a, b, items=True, cap=0):
    import torch
    n = len(a)
    counts = torch.full((max(n, 1),), -7, dtype=torch.int64, device="cuda")
    total = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    out = out_len = None
    if items:
        out = torch.full((max(1, cap),), -7, dtype=torch.int32, device="cuda")
        out_len = torch.zeros(1, dtype=torch.int64, device="cuda")
    gr.gr_segmented_intersect(G.handle, dev(np.asarray(a, np.int32)), dev(np.asarray(b, np.int32)),
                              n, counts, total, out, out_len)
    st = G.sync_status()
    assert st == gr.GR_OK, gr.status_str(st)
    res = host(counts)[:n], int(total.item())
    if items:
        k = int(out_len.item())
        return res + (host(out)[:min(k, out.numel())], k)
    return res


@pytest.mark.parametrize("seed", [1, 2])
def test_intersect_pairs_against_the_oracle(gr, seed):
    g = gg.rmat(14, 16, seed)
    G = gr.Graph.from_csr(g)
    rng = np.random.default_rng(seed)
    a = rng.integers(0, g.n, 5000)
    b = rng.integers(0, g.n, 5000)
    hub = gg.max_degree_vertex(g)
    a[:64] = hub                                   # long against short lists
    b[64:128] = hub
    a[128:160] = b[128:160] = hub                  # long against long
    counts, items, total = oracle.segmented_intersect(g.R, g.C, a, b)
    c, t, it, k = intersect(gr, G, a, b, cap=total)
    assert np.array_equal(c, counts) and t == total and k == total
    assert np.array_equal(it, items)
    c2, t2 = intersect(gr, G, a, b, items=False)  # counts only
    assert np.array_equal(c2, counts) and t2 == total
    G.close()


def test_intersect_small_capacity_and_empty(gr):
    import torch
    g = gg.rmat(12, 16, 3)
    G = gr.Graph.from_csr(g)
    a = np.arange(100) % g.n
    b = (np.arange(100) * 7) % g.n
    counts, items, total = oracle.segmented_intersect(g.R, g.C, a, b)
    out = torch.full((5,), -7, dtype=torch.int32, device="cuda")
    out_len = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt = torch.empty(100, dtype=torch.int64, device="cuda")
    gr.gr_segmented_intersect(G.handle, dev(a.astype(np.int32)), dev(b.astype(np.int32)), 100,
                              cnt, None, out, out_len)
    assert G.sync_status() == gr.GR_OK
    assert int(out_len.item()) == total and np.array_equal(host(out), items[:5])
    t = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    gr.gr_segmented_intersect(G.handle, dev(a[:1].astype(np.int32)), dev(b[:1].astype(np.int32)),
                              0, None, t)
    assert int(t.item()) == 0
    G.close()


def triangles(gr, G, per=True):
    import torch
    total = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    pv = torch.full((G.n,), -7, dtype=torch.int64, device="cuda") if per else None
    gr.gr_triangle_count(G.handle, total, pv)
    st = G.sync_status()
    assert st == gr.GR_OK, gr.status_str(st)
    return int(total.item()), (host(pv) if per else None)


@pytest.mark.parametrize("scale,ef", [(12, 16), (16, 16), (14, 4)])
def test_triangles_rmat(gr, scale, ef):
    g = gg.rmat(scale, ef, 1)
    G = gr.Graph.from_csr(g)
    t, per = oracle.triangles(g.R, g.C)
    gt, gper = triangles(gr, G)
    assert gt == t and np.array_equal(gper, per)
    assert triangles(gr, G, per=False)[0] == t      # total alone, same workspace again
    G.close()


def test_triangles_closed_forms(gr):
    for n in (3, 4, 10, 70):
        g = undirected(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
        G = gr.Graph.from_csr(g)
        t, per = triangles(gr, G)
        assert t == math.comb(n, 3) and (per == math.comb(n - 1, 2)).all()
        G.close()
    for g in (gg.grid(64, 0.0, 1), undirected(1, np.zeros((0, 2))), star_plus(3000),
              undirected(500, [(i, (i + 1) % 500) for i in range(500)])):
        G = gr.Graph.from_csr(g)
        t, per = oracle.triangles(g.R, g.C)
        gt, gper = triangles(gr, G)
        assert gt == t and np.array_equal(gper, per)
        G.close()


@pytest.mark.slow
def test_triangles_s20_total(gr):
    g = gg.rmat(20, 16, 1)
    G = gr.Graph.from_csr(g)
    t, _ = oracle.triangles(g.R, g.C)
    assert triangles(gr, G, per=False)[0] == t
    G.close()


def test_directed_graph_is_refused(gr):
    import torch
    g = gg.directed(4, np.array([0, 1]), np.array([1, 2]))
    G = gr.Graph.from_csr(g, symmetric=False)
    with pytest.raises(gr.GrError) as e:
        gr.gr_triangle_count(G.handle, torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert e.value.status == gr.GR_ERR_UNSUPPORTED
    G.close()
