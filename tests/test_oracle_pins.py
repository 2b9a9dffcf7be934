"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each pin is a closed form, a hand-worked golden file, an independent library
routine (scipy.sparse.csgraph), a brute-force method, or a structural
invariant — chosen so that a dropped term, a wrong sign, an off-by-one level
or a transposed edge direction in the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF64 = np.uint64(2**64 - 1)


# ---------------------------------------------------------------- helpers ---

def undirected(n, pairs):
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return gg.from_edges(n, pairs[:, 0], pairs[:, 1])


def path_graph(n):
    return undirected(n, [(i, i + 1) for i in range(n - 1)])


def cycle_graph(n):
    return undirected(n, [(i, (i + 1) % n) for i in range(n)])


def star_graph(n):
    return undirected(n, [(0, i) for i in range(1, n)])


def complete_graph(n):
    return undirected(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def binary_tree(n):
    return undirected(n, [((i - 1) // 2, i) for i in range(1, n)])


def scipy_csr(g, W=None):
    sp = pytest.importorskip("scipy.sparse")
    data = np.ones(g.m) if W is None else W.astype(np.float64)
    return sp.csr_matrix((data, g.C.astype(np.int64), g.R.astype(np.int64)), shape=(g.n, g.n))


def scipy_dist(g, src, W=None):
    cs = pytest.importorskip("scipy.sparse.csgraph")
    d = cs.dijkstra(scipy_csr(g, W), directed=True, indices=src, unweighted=W is None)
    return d


def read_golden(name):
    out = {"e": [], "arc": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k, *vals = line.split()
            if k in ("e", "arc"):
                out[k].append([int(v) for v in vals])
            else:
                out[k] = [int(v) for v in vals] if len(vals) > 1 else int(vals[0])
    return out


# ------------------------------------------------------- closed forms: BFS ---

@pytest.mark.parametrize("n", [1, 2, 7, 100])
def test_bfs_path(n):
    g = path_graph(n)
    d, p = oracle.bfs(g.R, g.C, 0)
    assert list(d) == list(range(n))
    assert list(p) == [-1] + list(range(n - 1))


@pytest.mark.parametrize("n", [3, 8, 9, 101])
def test_bfs_cycle(n):
    g = cycle_graph(n)
    d, _ = oracle.bfs(g.R, g.C, 0)
    assert list(d) == [min(i, n - i) for i in range(n)]


def test_bfs_star_center_and_leaf():
    g = star_graph(50)
    d, _ = oracle.bfs(g.R, g.C, 0)
    assert d[0] == 0 and (d[1:] == 1).all()
    d, p = oracle.bfs(g.R, g.C, 7)
    assert d[7] == 0 and d[0] == 1 and p[0] == 7
    assert all(d[i] == 2 and p[i] == 0 for i in range(1, 50) if i != 7)


def test_bfs_complete_graph():
    g = complete_graph(33)
    d, _ = oracle.bfs(g.R, g.C, 5)
    assert d[5] == 0 and (np.delete(d, 5) == 1).all()


def test_bfs_binary_tree():
    n = 1000
    g = binary_tree(n)
    d, p = oracle.bfs(g.R, g.C, 0)
    assert list(d) == [int(np.floor(np.log2(i + 1))) for i in range(n)]
    assert list(p[1:]) == [(i - 1) // 2 for i in range(1, n)]


@pytest.mark.parametrize("src_rc", [(0, 0), (3, 5), (9, 9)])
def test_bfs_full_grid_manhattan(src_rc):
    Wd = 10
    g = gg.grid(Wd, 0.0)
    r0, c0 = src_rc
    d, _ = oracle.bfs(g.R, g.C, r0 * Wd + c0)
    want = [abs(v // Wd - r0) + abs(v % Wd - c0) for v in range(Wd * Wd)]
    assert list(d) == want


def test_bfs_disconnected_and_isolated():
    g = undirected(6, [(0, 1), (1, 2), (4, 5)])
    d, p = oracle.bfs(g.R, g.C, 1)
    assert list(d) == [1, 0, 1, -1, -1, -1]
    assert list(p) == [1, -1, 1, -1, -1, -1]
    d, p = oracle.bfs(g.R, g.C, 3)  # isolated source
    assert list(d) == [-1, -1, -1, 0, -1, -1] and (p == -1).all()


# ------------------------------------------------------ closed forms: SSSP ---

def test_sssp_path_prefix_sums():
    rng = np.random.default_rng(0)
    n = 200
    g = path_graph(n)
    w_edge = rng.integers(1, 1000, n - 1)
    # weight of CSR entry (u, v) on a path is the weight of edge min(u, v)
    W = np.empty(g.m, np.uint32)
    for u in range(n):
        for e in range(g.R[u], g.R[u + 1]):
            W[e] = w_edge[min(u, g.C[e])]
    dist, pred, over = oracle.dijkstra(g.R, g.C, W, 0)
    assert not over
    assert list(dist) == [0] + list(np.cumsum(w_edge))
    assert list(pred) == [-1] + list(range(n - 1))


@pytest.mark.parametrize("c", [1, 5, 64])
def test_sssp_constant_weights_is_scaled_bfs(c):
    g = gg.rmat(10, 8, seed=11)
    W = np.full(g.m, c, np.uint32)
    src = gg.max_degree_vertex(g)
    dist, _, _ = oracle.dijkstra(g.R, g.C, W, src)
    depth, _ = oracle.bfs(g.R, g.C, src)
    want = np.where(depth < 0, oracle.INF32, depth.astype(np.int64) * c)
    assert (dist.astype(np.int64) == want).all()


def test_sssp_full_grid_unit_manhattan():
    Wd = 12
    g = gg.grid(Wd, 0.0)
    W = np.ones(g.m, np.uint32)
    dist, _, _ = oracle.dijkstra(g.R, g.C, W, 0)
    assert list(dist) == [v // Wd + v % Wd for v in range(Wd * Wd)]


def test_sssp_overflow_flag():
    g = path_graph(4)
    W = np.full(g.m, 2**31, np.uint32)
    dist, _, over = oracle.dijkstra(g.R, g.C, W, 0)
    assert over                       # 3 * 2^31 does not fit below UINT32_MAX
    assert dist[1] == 2**31 and dist[0] == 0
    W = np.full(g.m, 2**30, np.uint32)
    _, _, over = oracle.dijkstra(g.R, g.C, W, 0)
    assert not over                   # 3 * 2^30 fits


# --------------------------------------------------------- golden files ---

def test_golden_dijkstra_6v():
    gd = read_golden("dijkstra_6v.txt")
    e = np.array(gd["e"])
    g = gg.from_edges(gd["n"], e[:, 0], e[:, 1])
    wmap = {(min(a, b), max(a, b)): w for a, b, w in gd["e"]}
    W = np.array([wmap[(min(u, v), max(u, v))] for u in range(g.n)
                  for v in g.C[g.R[u]:g.R[u + 1]]], np.uint32)
    dist, pred, _ = oracle.dijkstra(g.R, g.C, W, gd["src"])
    assert list(dist) == gd["dist"]
    assert list(pred) == gd["sssp_pred"]
    assert list(oracle.sssp_min_parent(g.R, g.C, W, dist, gd["src"])) == gd["sssp_pred"]
    depth, _ = oracle.bfs(g.R, g.C, gd["src"])
    assert list(depth) == gd["depth"]
    assert list(oracle.bfs_min_parent(g.R, g.C, depth)) == gd["bfs_min_parent"]


def test_golden_directed_5v():
    gd = read_golden("directed_5v.txt")
    a = np.array(gd["arc"])
    g = gg.directed(gd["n"], a[:, 0], a[:, 1])
    d, p = oracle.bfs(g.R, g.C, 0)
    assert list(d) == gd["depth_from_0"] and list(p) == gd["pred_from_0"]
    d, _ = oracle.bfs(g.R, g.C, 3)
    assert list(d) == gd["depth_from_3"]


# ------------------------------------------- independent library: scipy ---

GRAPHS = [
    ("rmat10", lambda: gg.rmat(10, 16, seed=1)),
    ("rmat12e4", lambda: gg.rmat(12, 4, seed=7)),
    ("grid30del", lambda: gg.grid(30, 0.3, seed=3)),
    ("er", lambda: undirected(500, np.random.default_rng(5).integers(0, 500, (900, 2)))),
]


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_bfs_matches_scipy(name, make):
    g = make()
    for src in [gg.max_degree_vertex(g), 0, g.n - 1]:
        d, p = oracle.bfs(g.R, g.C, src)
        ref = scipy_dist(g, src)
        want = np.where(np.isinf(ref), -1, ref).astype(np.int64)
        assert (d == want).all()
        assert oracle.bfs_certificate(g.R, g.C, src, d, p) == 0


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_dijkstra_matches_scipy(name, make):
    g = make()
    W = gg.weights(g, 1, 64, seed=2)
    for src in [gg.max_degree_vertex(g), g.n // 2]:
        dist, pred, over = oracle.dijkstra(g.R, g.C, W, src)
        ref = scipy_dist(g, src, W)
        want = np.where(np.isinf(ref), oracle.INF32, ref).astype(np.int64)
        assert not over
        assert (dist.astype(np.int64) == want).all()
        assert oracle.sssp_certificate(g.R, g.C, W, src, dist, pred) == 0


def test_directed_bfs_matches_scipy():
    rng = np.random.default_rng(9)
    n = 300
    s, d = rng.integers(0, n, 1200), rng.integers(0, n, 1200)
    keep = s != d
    pairs = np.unique(np.stack([s[keep], d[keep]], 1), axis=0)
    g = gg.directed(n, pairs[:, 0], pairs[:, 1])
    for src in (0, 17, 299):
        depth, _ = oracle.bfs(g.R, g.C, src)
        ref = scipy_dist(g, src)
        assert (depth == np.where(np.isinf(ref), -1, ref)).all()


def test_floyd_warshall_matches_scipy():
    cs = pytest.importorskip("scipy.sparse.csgraph")
    g = gg.rmat(6, 4, seed=3)
    W = gg.weights(g, 1, 9, seed=4)
    D = oracle.floyd_warshall(g.R, g.C, W)
    ref = cs.floyd_warshall(scipy_csr(g, W), directed=True)
    want = np.where(np.isinf(ref), float(INF64), ref)
    assert (D.astype(np.float64) == want).all()


# ------------------------------------------------- brute-force agreement ---

def test_bfs_vs_floyd_warshall_all_sources():
    for seed in range(4):
        g = gg.rmat(6, 3, seed=100 + seed)
        D = oracle.floyd_warshall(g.R, g.C)
        for src in range(g.n):
            d, _ = oracle.bfs(g.R, g.C, src)
            want = np.where(D[src] == INF64, -1, D[src].astype(np.int64))
            assert (d == want).all()


def test_dijkstra_vs_bellman_ford():
    g = gg.rmat(11, 4, seed=21)
    W = gg.weights(g, 1, 1000, seed=22)
    for src in (0, 5, 1000):
        dist, _, _ = oracle.dijkstra(g.R, g.C, W, src)
        bf = oracle.bellman_ford(g.R, g.C, W, src)
        want = np.where(bf == INF64, oracle.INF32, bf)
        assert (dist.astype(np.uint64) == want).all()


def test_bellman_ford_unit_weights_is_bfs():
    g = gg.grid(20, 0.2, seed=8)
    bf = oracle.bellman_ford(g.R, g.C, None, 0)
    d, _ = oracle.bfs(g.R, g.C, 0)
    assert (np.where(bf == INF64, -1, bf.astype(np.int64)) == d).all()


# -------------------------------------------------- canonical parents ---

def _numpy_min_parent(g, level_of, tight):
    """Independent restatement with numpy scatter-min over the edge list."""
    u = np.repeat(np.arange(g.n), np.diff(g.R.astype(np.int64)))
    v = g.C.astype(np.int64)
    ok = tight(u, v)
    best = np.full(g.n, np.iinfo(np.int64).max)
    np.minimum.at(best, v[ok], u[ok])
    return np.where(best == np.iinfo(np.int64).max, -1, best)


def test_bfs_min_parent_vs_numpy():
    g = gg.rmat(11, 8, seed=31)
    d, _ = oracle.bfs(g.R, g.C, 0)
    p = oracle.bfs_min_parent(g.R, g.C, d)
    want = _numpy_min_parent(g, d, lambda u, v: (d[u] >= 0) & (d[v] == d[u] + 1))
    assert (p == want).all()
    assert oracle.bfs_certificate(g.R, g.C, 0, d, p) == 0


def test_sssp_min_parent_vs_numpy():
    g = gg.rmat(11, 8, seed=32)
    W = gg.weights(g, 1, 64, seed=33)
    dist, _, _ = oracle.dijkstra(g.R, g.C, W, 0)
    p = oracle.sssp_min_parent(g.R, g.C, W, dist, 0)
    dd = dist.astype(np.int64)
    tight = lambda u, v: (dist[u] != oracle.INF32) & (v != 0) & (dd[u] + W.astype(np.int64) == dd[v])
    assert (p == _numpy_min_parent(g, None, tight)).all()
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, p) == 0


# --------------------------------------------------------- certificates ---

def test_bfs_certificate_rejects_planted_mistakes():
    g = gg.rmat(10, 8, seed=41)
    src = 0
    d, p = oracle.bfs(g.R, g.C, src)
    assert oracle.bfs_certificate(g.R, g.C, src, d, p) == 0
    reached = np.nonzero(d > 1)[0]
    v = int(reached[0])
    bad = d.copy(); bad[v] += 1                       # one level too deep
    assert oracle.bfs_certificate(g.R, g.C, src, bad, p) != 0
    bad = d.copy(); bad[v] -= 1                       # one level too shallow
    assert oracle.bfs_certificate(g.R, g.C, src, bad, p) != 0
    bad = d.copy(); bad[v] = -1                       # dropped vertex
    assert oracle.bfs_certificate(g.R, g.C, src, bad, p) != 0
    # a parent one level up that is not a neighbour of v (one always exists here)
    up = [int(u) for u in np.nonzero(d == d[v] - 1)[0] if not np.isin(v, g.C[g.R[u]:g.R[u + 1]])]
    assert up
    badp = p.copy(); badp[v] = up[0]
    assert oracle.bfs_certificate(g.R, g.C, src, d, badp) == 11
    badp = p.copy(); badp[v] = v                      # parent at the same level
    assert oracle.bfs_certificate(g.R, g.C, src, d, badp) != 0
    badp = p.copy(); badp[src] = 0 if src else 1
    assert oracle.bfs_certificate(g.R, g.C, src, d, badp) != 0


def test_bfs_certificate_without_preds_needs_a_parent_level():
    # path 0 - 1 - 2 with vertex 2 claimed at depth 1: every edge rule holds, but
    # 2 has no neighbour at depth 0, which only the no-predecessor check sees
    g = undirected(3, [(0, 1), (1, 2)])
    assert oracle.bfs_certificate(g.R, g.C, 0, np.array([0, 1, 2], np.int32)) == 0
    assert oracle.bfs_certificate(g.R, g.C, 0, np.array([0, 1, 1], np.int32)) == 13


def test_certificates_on_a_hub_are_linear_and_still_strict():
    # a 400,000-leaf star with a second hub on every third leaf: every leaf's
    # parent is the hub, so an edge check that walks the parent's row costs
    # O(deg^2); the certificates must stay O(m) and still see planted parents
    import time
    k = 400_000
    leaves = np.arange(1, k + 1)
    pairs = np.concatenate([np.stack([np.zeros(k, np.int64), leaves], 1),
                            np.stack([leaves[::3], np.full(len(leaves[::3]), k + 1)], 1)])
    g = undirected(k + 2, pairs)
    W = np.ones(g.m, np.uint32)
    d, p = oracle.bfs(g.R, g.C, 0)
    dist, pred, _ = oracle.dijkstra(g.R, g.C, W, 0)
    t0 = time.perf_counter()
    assert oracle.bfs_certificate(g.R, g.C, 0, d, p) == 0
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, pred) == 0
    assert time.perf_counter() - t0 < 5.0
    # the second hub sits at depth 2 and its row holds leaves 1, 4, 7, ...
    # only: leaf 2 is one level up but not a neighbour
    badp = p.copy(); badp[k + 1] = 2
    assert oracle.bfs_certificate(g.R, g.C, 0, d, badp) == 11
    badp = pred.copy(); badp[k + 1] = 2
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, badp) == 8


def test_sssp_certificate_rejects_planted_mistakes():
    g = gg.rmat(10, 8, seed=42)
    W = gg.weights(g, 1, 64, seed=43)
    dist, pred, _ = oracle.dijkstra(g.R, g.C, W, 0)
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, pred) == 0
    v = int(np.nonzero((dist != oracle.INF32) & (dist > 0))[0][3])
    bad = dist.copy(); bad[v] += 1                    # relaxable edge remains
    assert oracle.sssp_certificate(g.R, g.C, W, 0, bad, pred) != 0
    bad = dist.copy(); bad[v] -= 1                    # no tight predecessor
    assert oracle.sssp_certificate(g.R, g.C, W, 0, bad, pred) != 0
    badp = pred.copy(); badp[v] = v                   # self-parent
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, badp) != 0


def test_sssp_certificate_detects_zero_weight_cycle():
    # 0 -1- 1 -0- 2 -0- 1 : preds 1<-2, 2<-1 form a cycle at equal distance
    g = undirected(3, [(0, 1), (1, 2)])
    W = np.array([1, 1, 0, 0], np.uint32)  # rows: 0:[1], 1:[0,2], 2:[1]
    dist = np.array([0, 1, 1], np.uint32)
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, np.array([-1, 0, 1])) == 0
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, np.array([-1, 2, 1])) != 0


# --------------------------------------------------- advance and filter ---

def test_advance_hand_case():
    #   0:[1,2]  1:[0,3]  2:[0]  3:[1]
    g = undirected(4, [(0, 1), (0, 2), (1, 3)])
    assert list(g.R) == [0, 2, 4, 5, 6] and list(g.C) == [1, 2, 0, 3, 0, 1]
    assert list(oracle.advance(g.R, g.C, [3, 0, 3])) == [1, 1, 2, 1]
    assert list(oracle.advance(g.R, g.C, [1, 2], edge_ids=True)) == [2, 3, 4]
    assert len(oracle.advance(g.R, g.C, [])) == 0


def test_advance_properties():
    g = gg.rmat(10, 8, seed=51)
    rng = np.random.default_rng(1)
    F = rng.integers(0, g.n, 300).astype(np.int32)
    out = oracle.advance(g.R, g.C, F)
    E = oracle.advance(g.R, g.C, F, edge_ids=True)
    deg = np.diff(g.R.astype(np.int64))
    assert len(out) == deg[F].sum() == len(E)
    assert (g.C[E] == out).all()                      # V->E and V->V agree
    starts = np.concatenate([[0], np.cumsum(deg[F])[:-1]])
    for i in (0, 5, 299):                             # segment i = row of F[i]
        seg = out[starts[i]:starts[i] + deg[F[i]]]
        assert (seg == g.C[g.R[F[i]]:g.R[F[i] + 1]]).all()


def test_filter_unique_vs_numpy_first_index():
    rng = np.random.default_rng(2)
    items = rng.integers(-3, 120, 2000).astype(np.int32)
    got = oracle.filter_unique(100, items)
    valid = items[(items >= 0) & (items < 100)]
    _, first = np.unique(valid, return_index=True)
    assert (got == valid[np.sort(first)]).all()


def test_filter_unvisited_and_near_far():
    rng = np.random.default_rng(3)
    depth = rng.integers(-1, 4, 1000).astype(np.int32)
    assert (oracle.filter_unvisited(depth) == np.flatnonzero(depth == -1)).all()
    dist = rng.integers(0, 100, 1000).astype(np.uint32)
    items = rng.integers(0, 1000, 3000).astype(np.int32)
    near, far = oracle.filter_near_far(1000, items, dist, 40)
    assert (near == items[dist[items] < 40]).all()
    assert (far == items[dist[items] >= 40]).all()


def test_advance_bfs_iterated_is_bfs():
    g = gg.rmat(11, 8, seed=61)
    src = gg.max_degree_vertex(g)
    depth = np.full(g.n, -1, np.int32); depth[src] = 0
    pred = np.full(g.n, -1, np.int32)
    F, level = np.array([src], np.int32), 0
    while len(F):
        F, depth, pred = oracle.advance_bfs(g.R, g.C, F, level, depth, pred)
        assert len(np.unique(F)) == len(F)           # each vertex discovered once
        level += 1
    want, _ = oracle.bfs(g.R, g.C, src)
    assert (depth == want).all()
    assert oracle.bfs_certificate(g.R, g.C, src, depth, pred) == 0


def test_pull_levels_match_bfs_with_min_parent():
    g = gg.rmat(11, 8, seed=62)
    src = 0
    want, _ = oracle.bfs(g.R, g.C, src)
    depth = np.full(g.n, -1, np.int32); depth[src] = 0
    pred = np.full(g.n, -1, np.int32)
    cand = oracle.filter_unvisited(depth)
    level = 0
    while True:
        act, cand, depth, pred = oracle.pull(g.R, g.C, cand, level, depth, pred)
        assert (np.sort(act) == np.flatnonzero(want == level + 1)).all()
        if not len(act):
            break
        level += 1
    assert (depth == want).all()
    assert (pred == oracle.bfs_min_parent(g.R, g.C, want)).all()


def test_advance_relax_hand_case():
    # path 0-1-2 with w(0,1)=5, w(1,2)=1 plus edge 0-2 with w=9
    g = undirected(3, [(0, 1), (1, 2), (0, 2)])     # rows 0:[1,2] 1:[0,2] 2:[0,1]
    W = np.array([5, 9, 5, 1, 9, 1], np.uint32)
    inf = oracle.INF32
    out, dist, pred = oracle.advance_relax(g.R, g.C, W, [0], [0, inf, inf], [-1, -1, -1])
    assert list(out) == [1, 2] and list(dist) == [0, 5, 9] and list(pred) == [-1, 0, 0]
    out, dist, pred = oracle.advance_relax(g.R, g.C, W, [1, 2], dist, pred)
    assert list(out) == [2] and list(dist) == [0, 5, 6] and list(pred) == [-1, 0, 1]


def test_advance_relax_iterated_is_dijkstra():
    g = gg.rmat(10, 8, seed=63)
    W = gg.weights(g, 1, 64, seed=64)
    dist = np.full(g.n, oracle.INF32, np.uint32); dist[0] = 0
    pred = np.full(g.n, -1, np.int32)
    F = np.array([0], np.int32)
    while len(F):
        F, dist, pred = oracle.advance_relax(g.R, g.C, W, F, dist, pred)
    want, _, _ = oracle.dijkstra(g.R, g.C, W, 0)
    assert (dist == want).all()
    assert oracle.sssp_certificate(g.R, g.C, W, 0, dist, pred) == 0


def test_bfs_multi_stacks_single_runs():
    g = gg.rmat(9, 8, seed=71)
    srcs = gg.sources(g, 5, seed=4)
    D = oracle.bfs_multi(g.R, g.C, srcs)
    for i, s in enumerate(srcs):
        ref = scipy_dist(g, int(s))
        assert (D[i] == np.where(np.isinf(ref), -1, ref)).all()
