"""GPU parity of gr_cc (hooking + pointer jumping, Sec. 6.4) against the CPU oracle.

The labelling is canonical (every vertex gets the smallest vertex id of its
component), so labels and the component count must equal the oracle's bit for
bit.
"""
import itertools

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


def run_cc(gr, G, **opts):
    import torch
    comp = torch.full((G.n,), -7, dtype=torch.int32, device="cuda")
    k = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    gr.gr_cc(G.handle, comp, k, gr.cc_opts(**opts) if opts else None)
    st = G.sync_status()
    assert st == gr.GR_OK, gr.status_str(st)
    return host(comp), int(k.item())


def check(gr, g, **opts):
    G = gr.Graph.from_csr(g)
    comp, k = run_cc(gr, G, **opts)
    want, kw = oracle.cc(g.R, g.C)
    assert k == kw
    assert np.array_equal(comp, want)
    G.close()


@pytest.mark.parametrize("big", [32, 1024, 1 << 30])
def test_rmat_s16(gr, big):
    check(gr, gg.rmat(16, 16, seed=1), big_degree=big)


def test_sparse_rmat_many_components(gr):
    check(gr, gg.rmat(16, 1, seed=2))          # a thin graph: thousands of components


def test_cut_grid(gr):
    check(gr, gg.grid(300, 0.45, seed=3))      # near the percolation threshold


@pytest.mark.slow
def test_rmat_s20(gr):
    check(gr, gg.rmat(20, 16, seed=1))


def test_long_path_and_shapes(gr):
    n = 100_000
    rng = np.random.default_rng(5)
    perm = rng.permutation(n)                   # a path through scrambled ids
    check(gr, undirected(n, np.stack([perm[:-1], perm[1:]], 1)))
    check(gr, undirected(n, [(i, i + 1) for i in range(n - 1)]))
    groups = [[0, 3, 6, 9], [1], [2, 4, 5, 7, 8]]
    check(gr, undirected(12, [p for grp in groups for p in itertools.combinations(grp, 2)]))
    check(gr, undirected(1, np.zeros((0, 2))))
    check(gr, undirected(7, np.zeros((0, 2))))
    for deg in (31, 1023, 1024, 5000):
        check(gr, star_plus(deg), big_degree=1024)


def test_directed_graph_is_refused(gr):
    import torch
    g = gg.directed(4, np.array([0, 1]), np.array([1, 2]))
    G = gr.Graph.from_csr(g, symmetric=False)
    with pytest.raises(gr.GrError) as e:
        gr.gr_cc(G.handle, torch.empty(4, dtype=torch.int32, device="cuda"))
    assert e.value.status == gr.GR_ERR_UNSUPPORTED
    G.close()
