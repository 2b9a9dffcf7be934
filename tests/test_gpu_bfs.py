"""GPU parity of gr_bfs (persistent direction-optimising BFS) against the CPU oracle.

Depths must equal the oracle's bit for bit; predecessors must pass the BFS
certificate (any valid BFS tree is a correct answer, Sec. 6.1).  Every
direction policy and split threshold must give the same depths.
"""
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


def run_bfs(gr, G, src, **opts):
    import torch
    depth = torch.empty(G.n, dtype=torch.int32, device="cuda")
    pred = torch.empty_like(depth)
    o = gr.bfs_opts(**opts) if opts else None
    gr.gr_bfs(G.handle, src, depth, pred, o)
    st = G.sync_status()
    assert st == gr.GR_OK, gr.status_str(st)
    return host(depth), host(pred)


def check(g, src, depth, pred):
    want, _ = oracle.bfs(g.R, g.C, src)
    assert np.array_equal(depth, want)
    assert oracle.bfs_certificate(g.R, g.C, src, depth, pred) == 0


@pytest.fixture(scope="module")
def s16(gr):
    g = gg.rmat(16, 16, seed=1)
    return g, gr.Graph.from_csr(g)


def test_config_s16_from_vertex0(gr, s16):
    g, G = s16
    d, p = run_bfs(gr, G, 0)
    check(g, 0, d, p)


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("big", [32, 100, 1024, 1 << 30])
@pytest.mark.parametrize("bulk", [0, 1, -1])
def test_directions_and_split_thresholds_agree(gr, s16, direction, big, bulk):
    # bulk: push levels of at least bulk_edges frontier edges mark a bitmap and list it
    # afterwards (0 = default threshold, 1 = every push level, -1 = none)
    g, G = s16
    for src in (0, 12345, int(gg.sources(g, 1, seed=9)[0])):
        d, p = run_bfs(gr, G, src, direction=direction, big_degree=big, bulk_edges=bulk)
        check(g, src, d, p)


@pytest.mark.parametrize("do_a,do_b", [(0.0, 0.0), (1e-4, 1e-6), (0.5, 0.1), (1e9, 0.0)])
def test_switch_parameters_do_not_change_depths(gr, s16, do_a, do_b):
    g, G = s16
    d, p = run_bfs(gr, G, 0, do_a=do_a, do_b=do_b)
    check(g, 0, d, p)


def test_level_stats(gr, s16):
    import torch
    g, G = s16
    stats = torch.full((4 * 64,), -7, dtype=torch.int32, device="cuda")
    d, p = run_bfs(gr, G, 0, level_stats=stats.data_ptr(), max_levels=64)
    check(g, 0, d, p)
    s = host(stats).reshape(64, 4)
    levels = int(d.max()) + 1
    counts = np.bincount(d[d >= 0], minlength=levels)
    assert np.array_equal(s[:levels, 0], counts)        # frontier size per level
    deg = g.degrees()
    for L in range(levels):                              # m_f per level = sum of degrees
        assert s[L, 2] == min(int(deg[d == L].sum()), 2**31 - 1)
    assert s[0, 3] >= 0 and (np.diff(s[:levels, 3]) >= 0).all()   # level start times
    end = s[levels]                                       # the loop's end row
    assert end[0] == 0 and end[3] >= s[levels - 1, 3]


def test_small_and_degenerate_graphs(gr):
    cases = [
        (undirected(1, np.zeros((0, 2))), 0),                  # single vertex, no edge
        (undirected(5, [(0, 1), (2, 3)]), 4),                  # isolated source
        (undirected(5, [(0, 1), (2, 3)]), 1),                  # two components
        (undirected(2000, [(i, i + 1) for i in range(1999)]), 0),   # long path
        (undirected(40, [(i, j) for i in range(40) for j in range(i + 1, 40)]), 3),  # K_40
    ]
    for deg in (31, 32, 33, 255, 256, 257, 1023, 1024, 1025, 5000):
        cases.append((star_plus(deg), 0))
        cases.append((star_plus(deg), 1))
    for g, src in cases:
        G = gr.Graph.from_csr(g)
        for direction in (0, 1, 2):
            for big in (32, 1024):
                for bulk in (1, -1):
                    d, p = run_bfs(gr, G, src, direction=direction, big_degree=big,
                                   bulk_edges=bulk)
                    check(g, src, d, p)
        G.close()


@pytest.mark.parametrize("direction", [0, 1])
def test_mesh_graph(gr, direction):
    # hundreds of levels with frontiers of a few hundred vertices
    g = gg.grid(128, 0.1, seed=4)
    G = gr.Graph.from_csr(g)
    for src in (0, 8256):
        d, p = run_bfs(gr, G, src, direction=direction)
        check(g, src, d, p)
    G.close()


def dumbbell(path_len=100, leaves=40000):
    """path -> hub A -> `leaves` leaves -> hub B -> path: small, huge, small frontiers."""
    a = path_len - 1
    b = path_len + leaves
    n = b + path_len
    pairs = [(i, i + 1) for i in range(path_len - 1)]
    pairs += [(a, path_len + i) for i in range(leaves)]
    pairs += [(path_len + i, b) for i in range(leaves)]
    pairs += [(b + i, b + i + 1) for i in range(path_len - 1)]
    return undirected(n, pairs)


@pytest.mark.parametrize("direction", [0, 1])
def test_frontier_grows_and_shrinks(gr, direction):
    # tiny frontiers along the paths, 40000 vertices (80000 edges) at the
    # leaves: with direction 0 some levels run pull and others push
    import torch
    g = dumbbell()
    G = gr.Graph.from_csr(g)
    levels = 201   # path 0..99, the leaves, hub B, then depths 102..200
    stats = torch.full((4 * 256,), -7, dtype=torch.int32, device="cuda")
    d, p = run_bfs(gr, G, 0, direction=direction, level_stats=stats.data_ptr(), max_levels=256)
    check(g, 0, d, p)
    s = host(stats).reshape(256, 4)
    assert int(d.max()) + 1 == levels
    assert np.array_equal(s[:levels, 0], np.bincount(d, minlength=levels))
    assert (np.diff(s[:levels, 3]) >= 0).all()
    if direction == 0:
        assert s[:levels, 1].any() and not s[:levels, 1].all()
    for src in (g.n - 1, 100 + 7):
        d, p = run_bfs(gr, G, src, direction=direction)
        check(g, src, d, p)
    G.close()


def hubs_behind_a_path(fill=3000, hubs=1200, plen=6):
    """A path 0 - p1 - ... - p_plen on the highest ids, `fill` leaves on ids
    1..fill hanging off the path's end, and `hubs` hubs that each see every
    leaf and one path vertex.  Rows are sorted, so a hub's path neighbour is
    its last entry: on pull levels every hub scans its whole row of fill + 1
    entries, long enough to go to the grid-shared deferred list; the hubs of
    later path vertices stay unmatched for several levels, and more hubs than
    the list holds are candidates at once."""
    n = 1 + fill + hubs + plen
    path = [0] + [n - 1 - i for i in range(plen)]
    pairs = [(path[i], path[i + 1]) for i in range(plen)]
    leaves = np.arange(1, fill + 1)
    pairs += [(int(x), path[-1]) for x in leaves]
    h = np.arange(fill + 1, fill + 1 + hubs)
    hp = np.repeat(h, fill)
    lp = np.tile(leaves, hubs)
    pairs = np.concatenate([np.asarray(pairs, np.int64), np.stack([hp, lp], 1),
                            np.stack([h, [path[1 + j % plen] for j in range(hubs)]], 1)])
    return undirected(n, pairs)


@pytest.mark.parametrize("direction", [0, 2])
def test_long_unvisited_rows_are_shared_by_the_grid(gr, direction):
    # pull levels (forced with direction 2) where hundreds of long rows end in
    # their only frontier neighbour: matched ones, unmatched ones that stay
    # listed for the next level, and more than the deferred list holds
    import torch
    g = hubs_behind_a_path()
    G = gr.Graph.from_csr(g)
    cap = 64
    stats = torch.zeros(4 * cap, dtype=torch.int32, device="cuda")
    d, p = run_bfs(gr, G, 0, direction=direction, level_stats=stats.data_ptr(), max_levels=cap)
    check(g, 0, d, p)
    levels = int(d.max()) + 1
    s = host(stats).reshape(cap, 4)
    assert np.array_equal(s[:levels, 0], np.bincount(d[d >= 0], minlength=levels))
    for src in (g.n - 1, 5):
        d, p = run_bfs(gr, G, src, direction=direction)
        check(g, src, d, p)
    G.close()


def test_directed_graph_push_only(gr):
    rng = np.random.default_rng(3)
    n = 3000
    s, t = rng.integers(0, n, 20000), rng.integers(0, n, 20000)
    keep = s != t
    pairs = np.unique(np.stack([s[keep], t[keep]], 1), axis=0)
    g = gg.directed(n, pairs[:, 0], pairs[:, 1])
    G = gr.Graph.from_csr(g, symmetric=False)
    for bulk in (0, 1, -1):        # bulk push levels work without a transpose too
        d, p = run_bfs(gr, G, 0, bulk_edges=bulk)
        check(g, 0, d, p)
    with pytest.raises(gr.GrError):
        run_bfs(gr, G, 0, direction=gr.GR_DIR_PULL)


def test_invalid_arguments_rejected(gr, s16):
    import torch
    g, G = s16
    depth = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for bad in (-1, g.n):
        with pytest.raises(gr.GrError) as e:
            gr.gr_bfs(G.handle, bad, depth)
        assert e.value.status == gr.GR_ERR_INVALID_ARG


def test_invalid_graphs_rejected(gr):
    import torch
    R = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    C = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    bad_cases = [
        (torch.tensor([0, 1, 3], dtype=torch.int32, device="cuda"), C, None, 0),  # R[n] != m
        (torch.tensor([1, 1, 2], dtype=torch.int32, device="cuda"), C, None, 0),  # R[0] != 0
        (R, torch.tensor([1, 2], dtype=torch.int32, device="cuda"), None, 0),     # col >= n
        (R, torch.tensor([1, -1], dtype=torch.int32, device="cuda"), None, 0),    # col < 0
        (R, C, torch.tensor([3, 0], dtype=torch.int32, device="cuda"), 0),        # zero weight
        (R, C, torch.tensor([3, 4], dtype=torch.int32, device="cuda"), 2),        # asym weight
        (R, torch.tensor([1, 1], dtype=torch.int32, device="cuda"), None, 2),     # asym edge
    ]
    for r, c, w, flags in bad_cases:
        with pytest.raises(gr.GrError) as e:
            gr.gr_graph_create_csr(2, 2, r, c, w, flags)
        assert e.value.status == gr.GR_ERR_INVALID_GRAPH
    h = gr.gr_graph_create_csr(2, 2, R, C, None, gr.GR_SYMMETRIC | gr.GR_COPY)
    gr.gr_graph_destroy(h)


def test_barrier_timeout_is_reported_and_recoverable(gr, s16):
    import torch
    g, G = s16
    depth = torch.empty(g.n, dtype=torch.int32, device="cuda")
    seen = None
    for _ in range(3):   # a budget of one poll runs out while other CTAs still work
        gr.gr_bfs(G.handle, 0, depth, None, gr.bfs_opts(spin_limit=1))
        seen = G.sync_status()
        if seen == gr.GR_ERR_TIMEOUT:
            break
    assert seen == gr.GR_ERR_TIMEOUT
    d, p = run_bfs(gr, G, 0)      # the context and the workspace are still usable
    check(g, 0, d, p)


@pytest.mark.parametrize("cap", [1, 7, 38])
def test_cta_cap_does_not_change_depths(gr, s16, cap):
    g, G = s16
    for src in (0, 12345):
        d, p = run_bfs(gr, G, src, max_blocks=cap)
        check(g, src, d, p)
    mesh = gg.grid(128, 0.1, seed=4)
    M = gr.Graph.from_csr(mesh)
    d, p = run_bfs(gr, M, 0, max_blocks=cap)
    check(mesh, 0, d, p)
    M.close()


def test_capped_queries_run_side_by_side(gr):
    # four capped BFS on four streams with their own workspaces at once
    import torch
    g = gg.grid(256, 0.1, seed=4)
    G = gr.Graph.from_csr(g)
    srcs = [0, 999, 30000, 65535]
    wss = [gr.gr_workspace_create(G.handle, gr.GR_OP_BFS) for _ in srcs]
    streams = [torch.cuda.Stream() for _ in srcs]
    outs = []
    torch.cuda.synchronize()
    for src, ws, s in zip(srcs, wss, streams):
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        p = torch.empty_like(d)
        gr.gr_bfs(G.handle, src, d, p, gr.bfs_opts(ws=ws, blocks_per_sm=1, max_blocks=16), stream=s)
        outs.append((d, p))
    torch.cuda.synchronize()
    for src, ws, (d, p) in zip(srcs, wss, outs):
        assert G.sync_status(ws) == 0
        check(g, src, host(d), host(p))
        gr.gr_workspace_destroy(ws)
    with pytest.raises(gr.GrError):
        gr.gr_bfs(G.handle, 0, outs[0][0], None, gr.bfs_opts(max_blocks=-1))
    G.close()


def test_separate_workspaces_on_streams(gr, s16):
    import torch
    g, G = s16
    srcs = [0, 7, 99, 1234]
    wss = [gr.gr_workspace_create(G.handle, gr.GR_OP_BFS) for _ in srcs]
    streams = [torch.cuda.Stream() for _ in srcs]
    outs = []
    torch.cuda.synchronize()
    for src, ws, s in zip(srcs, wss, streams):
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        p = torch.empty_like(d)
        gr.gr_bfs(G.handle, src, d, p, gr.bfs_opts(ws=ws, blocks_per_sm=1), stream=s)
        outs.append((d, p))
    torch.cuda.synchronize()
    for src, ws, (d, p) in zip(srcs, wss, outs):
        assert G.sync_status(ws) == 0
        check(g, src, host(d), host(p))
        gr.gr_workspace_destroy(ws)


@pytest.mark.slow
def test_config_s22_full_size(gr):
    g = gg.rmat(22, 16, seed=2)
    G = gr.Graph.from_csr(g)
    hub = gg.max_degree_vertex(g)
    for src in [hub] + list(gg.sources(g, 2, seed=2)):
        d, p = run_bfs(gr, G, int(src))
        check(g, int(src), d, p)
    for bulk in (0, -1):           # push only: bulk levels (default) and atomic claims
        d2, p2 = run_bfs(gr, G, hub, direction=gr.GR_DIR_PUSH, bulk_edges=bulk)
        check(g, hub, d2, p2)
    G.close()


@pytest.mark.slow
def test_config_grid4096_full_size(gr):
    g = gg.grid(4096, 0.1, seed=3)
    G = gr.Graph.from_csr(g)
    d, p = run_bfs(gr, G, 0)
    check(g, 0, d, p)
    assert d.max() > 8000       # thousands of small-frontier levels
    G.close()
