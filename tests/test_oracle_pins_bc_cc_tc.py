"""Pins of the oracle functions for betweenness centrality (Sec. 6.3), connected
components (Sec. 6.4), segmented intersection and triangle counting (Sec. 4.3,
Sec. 6.6) and the K-way multisplit of the priority queue (Sec. 5.1.5).

Every oracle function is checked against something other than itself: closed
forms, brute force over all-pairs distances, and independent library routines
(scipy's csgraph and sparse products, numpy's set intersection, networkx's
Brandes and triangle routines).  A few planted mistakes show that the checks
would catch a dropped term or a wrong index.
"""
import itertools
import math

import numpy as np
import pytest

import graphgen as gg
import oracle


def undirected(n, pairs):
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return gg.from_edges(n, pairs[:, 0], pairs[:, 1])


def path(n):
    return undirected(n, [(i, i + 1) for i in range(n - 1)])


def star(n):
    return undirected(n, [(0, i) for i in range(1, n)])


def complete(n):
    return undirected(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def cycle(n):
    return undirected(n, [(i, (i + 1) % n) for i in range(n)])


def full_grid(w):
    pairs = []
    for r in range(w):
        for c in range(w):
            v = r * w + c
            if c + 1 < w:
                pairs.append((v, v + 1))
            if r + 1 < w:
                pairs.append((v, v + w))
    return undirected(w * w, pairs)


def diamonds(k):
    """A chain of k diamonds: every diamond doubles the number of shortest paths."""
    pairs, top = [], 0
    for i in range(k):
        a, b, bot = 3 * i + 1, 3 * i + 2, 3 * i + 3
        pairs += [(top, a), (top, b), (a, bot), (b, bot)]
        top = bot
    return undirected(3 * k + 1, pairs), top


def random_graph(n, m, seed):
    rng = np.random.default_rng(seed)
    s, t = rng.integers(0, n, m), rng.integers(0, n, m)
    keep = s != t
    return undirected(n, np.stack([s[keep], t[keep]], 1))


def brute_sigma(g, src):
    """Shortest-path counts by dynamic programming over all-pairs distances."""
    D = oracle.floyd_warshall(g.R, g.C).astype(np.float64)
    D[D > 1e18] = np.inf
    d = D[src]
    order = np.argsort(d, kind="stable")
    sigma = np.zeros(g.n, dtype=object)
    sigma[src] = 1
    for v in order:
        if v == src or not np.isfinite(d[v]):
            continue
        for u in range(g.n):
            if d[u] + 1 == d[v] and v in g.C[g.R[u]:g.R[u + 1]]:
                sigma[v] += sigma[u]
    return sigma


# ---------------------------------------------------------------- BC -----

def test_sigma_on_a_full_grid_is_binomial():
    # from the corner, the shortest paths to (r, c) are the C(r + c, r) lattice paths
    w = 9
    g = full_grid(w)
    depth, sigma, _, ovf = oracle.bc_source(g.R, g.C, 0)
    assert not ovf
    for r in range(w):
        for c in range(w):
            assert depth[r * w + c] == r + c
            assert sigma[r * w + c] == math.comb(r + c, r)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sigma_matches_brute_force_counting(seed):
    g = random_graph(40, 90, seed)
    for src in (0, 7, 39):
        depth, sigma, _, _ = oracle.bc_source(g.R, g.C, src)
        want = brute_sigma(g, src)
        assert [int(x) for x in sigma] == [int(x) for x in want]
        bd, _ = oracle.bfs(g.R, g.C, src)
        assert np.array_equal(depth, bd)


def test_sigma_overflow_is_reported_exactly_at_int64():
    g, end = diamonds(62)
    _, sigma, _, ovf = oracle.bc_source(g.R, g.C, 0)
    assert not ovf and int(sigma[end]) == 2 ** 62
    g, end = diamonds(63)                     # 2^63 paths: one more than INT64_MAX
    _, _, _, ovf = oracle.bc_source(g.R, g.C, 0)
    assert ovf
    with pytest.raises(OverflowError):
        oracle.bc(g.R, g.C, [0])


@pytest.mark.parametrize("n", [2, 3, 7, 30])
def test_bc_closed_forms(n):
    all_src = list(range(n))
    # path: vertex i lies on every path between a vertex on its left and one on its right
    got = oracle.bc(path(n).R, path(n).C, all_src)
    assert np.array_equal(got, [2.0 * i * (n - 1 - i) for i in range(n)])
    # star: the centre on every leaf-to-leaf path, leaves on none
    got = oracle.bc(star(n).R, star(n).C, all_src)
    assert got[0] == (n - 1) * (n - 2) and not got[1:].any()
    # complete graph: every pair adjacent
    assert not oracle.bc(complete(n).R, complete(n).C, all_src).any()


@pytest.mark.parametrize("n", [5, 8, 11])
def test_bc_cycle_is_uniform_and_matches_networkx(n):
    nx = pytest.importorskip("networkx")
    g = cycle(n)
    got = oracle.bc(g.R, g.C, list(range(n)))
    assert np.allclose(got, got[0])                    # vertex-transitive
    ref = nx.betweenness_centrality(nx.cycle_graph(n), normalized=False)
    assert np.allclose(got, 2 * np.array([ref[i] for i in range(n)]))


@pytest.mark.parametrize("seed", [4, 5])
def test_bc_matches_networkx_brandes(seed):
    nx = pytest.importorskip("networkx")
    g = gg.rmat(9, 8, seed)
    srcs = list(range(g.n))
    got = oracle.bc(g.R, g.C, srcs)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        G.add_edges_from((u, int(v)) for v in g.C[g.R[u]:g.R[u + 1]])
    ref = nx.betweenness_centrality(G, normalized=False)
    # networkx counts each unordered pair once on an undirected graph
    assert np.allclose(got, 2 * np.array([ref[i] for i in range(g.n)]), rtol=1e-10, atol=1e-9)


def test_bc_planted_mistake_is_caught():
    # dropping the "1 +" of the dependency recursion breaks the path closed form
    g = path(6)
    _, sigma, _, _ = oracle.bc_source(g.R, g.C, 0)
    depth = np.arange(6)
    delta = np.zeros(6)
    for u in range(5, -1, -1):
        delta[u] = sum(sigma[u] / sigma[v] * delta[v] for v in g.C[g.R[u]:g.R[u + 1]]
                       if depth[v] == depth[u] + 1)
    assert not np.array_equal(delta[1:], [4.0, 3.0, 2.0, 1.0, 0.0])
    _, _, good, _ = oracle.bc_source(g.R, g.C, 0)
    assert np.array_equal(good[1:], [4.0, 3.0, 2.0, 1.0, 0.0])


# ---------------------------------------------------------------- CC -----

def canonical(labels):
    """Relabel a partition by the smallest member of each class."""
    first = {}
    out = np.empty(len(labels), np.int64)
    for v, l in enumerate(labels):
        first.setdefault(l, v)
        out[v] = first[l]
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cc_matches_scipy(seed):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    for g in (random_graph(500, 300, seed), gg.rmat(12, 2, seed), gg.grid(40, 0.45, seed)):
        label, k = oracle.cc(g.R, g.C)
        A = csr_matrix((np.ones(g.m), g.C, g.R), shape=(g.n, g.n))
        k_ref, lab_ref = connected_components(A, directed=False)
        assert k == k_ref
        assert np.array_equal(label, canonical(lab_ref))


def test_cc_closed_forms():
    # three cliques of sizes 4, 1, 5 with ids interleaved, and isolated vertices
    groups = [[0, 3, 6, 9], [1], [2, 4, 5, 7, 8]]
    pairs = [(a, b) for gr in groups for a, b in itertools.combinations(gr, 2)]
    g = undirected(12, pairs)                   # 10 and 11 isolated
    label, k = oracle.cc(g.R, g.C)
    assert k == 5
    want = {v: min(gr) for gr in groups for v in gr}
    want.update({10: 10, 11: 11})
    assert label.tolist() == [want[v] for v in range(12)]
    label, k = oracle.cc(path(50).R, path(50).C)
    assert k == 1 and not label.any()


# ------------------------------------------------- segmented intersection -

@pytest.mark.parametrize("seed", [1, 2])
def test_segmented_intersect_matches_numpy(seed):
    g = gg.rmat(11, 8, seed)
    rng = np.random.default_rng(seed)
    a = rng.integers(0, g.n, 400)
    b = rng.integers(0, g.n, 400)
    hub = int(np.argmax(g.degrees()))
    a[:5] = hub                                  # a long list against short ones
    counts, items, total = oracle.segmented_intersect(g.R, g.C, a, b)
    parts = [np.intersect1d(g.C[g.R[x]:g.R[x + 1]], g.C[g.R[y]:g.R[y + 1]]) for x, y in zip(a, b)]
    assert counts.tolist() == [len(p) for p in parts]
    assert total == sum(len(p) for p in parts)
    assert np.array_equal(items, np.concatenate(parts) if parts else [])


# ---------------------------------------------------------------- TC -----

@pytest.mark.parametrize("n", [3, 4, 6, 10])
def test_triangles_closed_forms(n):
    t, per = oracle.triangles(complete(n).R, complete(n).C)
    assert t == math.comb(n, 3) and (per == math.comb(n - 1, 2)).all()
    assert oracle.triangles(cycle(n + 1).R, cycle(n + 1).C)[0] == (1 if n + 1 == 3 else 0)
    assert oracle.triangles(full_grid(n).R, full_grid(n).C)[0] == 0   # bipartite


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_triangles_match_trace_of_a_cubed_and_networkx(seed):
    from scipy.sparse import csr_matrix
    g = gg.rmat(10, 8, seed)
    t, per = oracle.triangles(g.R, g.C)
    A = csr_matrix((np.ones(g.m, np.int64), g.C, g.R), shape=(g.n, g.n))
    A3 = A @ A @ A
    assert t * 6 == int(A3.diagonal().sum())
    assert np.array_equal(per * 2, A3.diagonal())          # (A^3)_vv = 2 x triangles at v
    nx = pytest.importorskip("networkx")
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        G.add_edges_from((u, int(v)) for v in g.C[g.R[u]:g.R[u + 1]])
    tri = nx.triangles(G)
    assert per.tolist() == [tri[i] for i in range(g.n)]


def test_triangles_planted_edge_adds_one():
    g = path(3)
    assert oracle.triangles(g.R, g.C)[0] == 0
    g = undirected(3, [(0, 1), (1, 2), (0, 2)])
    assert oracle.triangles(g.R, g.C)[0] == 1


# -------------------------------------------------------------- multisplit -

def test_multisplit_with_two_buckets_is_the_near_far_split():
    rng = np.random.default_rng(7)
    n = 300
    dist = rng.integers(0, 1000, n).astype(np.uint32)
    items = rng.integers(-5, n + 5, 2000)
    for T in (1, 250, 999, 1000):
        out, bl = oracle.multisplit(n, items, dist, 0, T, 2)
        near, far = oracle.filter_near_far(n, items, dist, T)
        assert bl.tolist() == [len(near), len(far)]
        assert np.array_equal(out, np.concatenate([near, far]))


def test_multisplit_invariants_and_identity_distances():
    rng = np.random.default_rng(8)
    n = 1000
    dist = rng.integers(0, 5000, n).astype(np.uint32)
    items = rng.integers(0, n, 4000)
    base, delta, K = 1200, 300, 9
    out, bl = oracle.multisplit(n, items, dist, base, delta, K)
    assert bl.sum() == len(items) and len(out) == len(items)
    assert sorted(out.tolist()) == sorted(items.tolist())           # a permutation
    start = 0
    for j in range(K):
        # bucket j holds, in input order, the items whose distance lies in its range
        lo = base + j * delta if j else -1
        hi = base + (j + 1) * delta if j < K - 1 else 1 << 40
        want = [v for v in items.tolist() if lo <= int(dist[v]) < hi]
        assert out[start:start + bl[j]].tolist() == want
        start += bl[j]
    # distances equal to the ids, sorted input: buckets of consecutive ids, order unchanged
    ident = np.arange(n, dtype=np.uint32)
    out, bl = oracle.multisplit(n, np.arange(n), ident, 0, 64, 64)
    assert np.array_equal(out, np.arange(n)) and bl[:15].tolist() == [64] * 15
