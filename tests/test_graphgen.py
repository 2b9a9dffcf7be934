"""Input generators: determinism, structure and loose sanity against the paper's dataset stats.

The generators are not pinned against Graph500's own generator (its code is
not available here); they are pinned by determinism and by the structural
rules of the paper's datasets (Sec. 7: undirected, no self-loops, no
duplicate edges) plus the scale-free shape it reports for R-MAT.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle


def check_structure(g):
    R, C = g.R.astype(np.int64), g.C.astype(np.int64)
    assert R[0] == 0 and R[-1] == g.m and (np.diff(R) >= 0).all()
    assert ((C >= 0) & (C < g.n)).all()
    u = np.repeat(np.arange(g.n), np.diff(R))
    assert (u != C).all(), "self-loop"
    for a in range(g.n):                               # rows sorted, no duplicates
        row = C[R[a]:R[a + 1]]
        assert (np.diff(row) > 0).all()
    key = u * g.n + C                                  # symmetric
    rkey = np.sort(C * g.n + u)
    assert (np.sort(key) == rkey).all()


def test_rmat_structure_and_determinism():
    a = gg.rmat(10, 16, seed=1)
    b = gg.rmat(10, 16, seed=1)
    c = gg.rmat(10, 16, seed=2)
    check_structure(a)
    assert gg.csr_digest(a) == gg.csr_digest(b)
    assert gg.csr_digest(a) != gg.csr_digest(c)
    assert a.m <= 2 * 16 * a.n


def test_rmat_scale_free_shape():
    g = gg.rmat(14, 16, seed=1)
    deg = g.degrees()
    # heavy tail: the hub sits at vertex 0 (no permutation) and dwarfs the mean
    assert gg.max_degree_vertex(g) == 0
    assert deg.max() > 50 * deg[deg > 0].mean()
    # "80% of nodes have degree less than 64" (Sec. 7 dataset notes)
    assert (deg < 64).mean() >= 0.8
    # small diameter from the hub (the paper's R-MAT diameters are 5-6)
    d, _ = oracle.bfs(g.R, g.C, 0)
    assert 3 <= d.max() <= 9


def test_grid_structure_and_deletion_rate():
    g = gg.grid(64, 0.1, seed=3)
    check_structure(g)
    full = 2 * 64 * 63
    kept = g.m // 2
    assert abs((full - kept) / full - 0.1) < 0.02
    assert gg.csr_digest(g) == gg.csr_digest(gg.grid(64, 0.1, seed=3))
    full_g = gg.grid(8, 0.0)
    assert full_g.m == 2 * 2 * 8 * 7


def test_weights_symmetric_and_in_range():
    g = gg.rmat(10, 8, seed=5)
    W = gg.weights(g, 1, 64, seed=2)
    assert W.min() >= 1 and W.max() <= 64
    u = np.repeat(np.arange(g.n), g.degrees())
    wmap = dict(zip(zip(u.tolist(), g.C.tolist()), W.tolist()))
    assert all(wmap[(b, a)] == w for (a, b), w in wmap.items())
    assert len(np.unique(W)) == 64


def test_sources_distinct_nonisolated_deterministic():
    g = gg.rmat(12, 16, seed=1)
    s = gg.sources(g, 64, seed=4)
    assert len(s) == 64 and len(np.unique(s)) == 64
    assert (g.degrees()[s] >= 1).all()
    assert (s == gg.sources(g, 64, seed=4)).all()


def test_from_edges_rejects_out_of_range():
    with pytest.raises(ValueError):
        gg.from_edges(3, [0, 5], [1, 1])
