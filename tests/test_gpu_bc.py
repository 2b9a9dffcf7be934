"""GPU parity of gr_bc (Brandes' betweenness centrality, Sec. 6.3) against the CPU oracle.

Depths and shortest-path counts are integers and must equal the oracle's bit
for bit.  Dependencies are double-precision sums of positive terms whose order
differs between the kernel and the oracle: a k-term sum of positive terms in any
order lies within (k - 1) u of the exact sum (u = 2^-53), and the error carried
through D levels stays below D * max_degree * u relative, about 1e-10 for the
graphs here.  The tests use a relative tolerance of 1e-9.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _helpers import host, star_plus, undirected

pytestmark = pytest.mark.gpu
RTOL = 1e-9


@pytest.fixture(scope="module")
def gr():
    import paper_1701_01170_gb300 as m
    m.load()
    return m


def run_bc(gr, G, src, bc=None, expect=0, **opts):
    import torch
    depth = torch.empty(G.n, dtype=torch.int32, device="cuda")
    sigma = torch.empty(G.n, dtype=torch.int64, device="cuda")
    delta = torch.empty(G.n, dtype=torch.float64, device="cuda")
    gr.gr_bc(G.handle, src, depth, sigma, delta, bc, gr.bc_opts(**opts) if opts else None)
    st = G.sync_status()
    assert st == expect, gr.status_str(st)
    return host(depth), host(sigma), host(delta)


def close(got, want):
    scale = max(1.0, float(np.abs(want).max()) if len(want) else 1.0)
    assert np.allclose(got, want, rtol=RTOL, atol=RTOL * scale), \
        float(np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-300)))


def check(g, src, depth, sigma, delta):
    d, s, dl, ovf = oracle.bc_source(g.R, g.C, src)
    assert not ovf
    assert np.array_equal(depth, d)
    assert np.array_equal(sigma, s)
    close(delta, dl)


@pytest.fixture(scope="module")
def s16(gr):
    g = gg.rmat(16, 16, seed=1)
    return g, gr.Graph.from_csr(g)


@pytest.mark.parametrize("big", [32, 256, 1 << 30])
def test_s16_single_sources(gr, s16, big):
    g, G = s16
    for src in (0, gg.max_degree_vertex(g), int(gg.sources(g, 1, seed=3)[0])):
        check(g, src, *run_bc(gr, G, src, big_degree=big))


def test_s16_bc_accumulates_over_sources(gr, s16):
    import torch
    g, G = s16
    srcs = [0] + [int(s) for s in gg.sources(g, 5, seed=4)]
    bc = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    for s in srcs:
        run_bc(gr, G, s, bc=bc)
    close(host(bc), oracle.bc(g.R, g.C, srcs))


@pytest.mark.slow
def test_s20_sources(gr):
    g = gg.rmat(20, 16, seed=1)
    G = gr.Graph.from_csr(g)
    for src in (gg.max_degree_vertex(g), int(gg.sources(g, 1, seed=5)[0])):
        check(g, src, *run_bc(gr, G, src))
    G.close()


def test_small_and_degenerate_graphs(gr):
    import torch
    n = 30
    cases = [
        undirected(1, np.zeros((0, 2))),                                       # one vertex
        undirected(n, [(i, i + 1) for i in range(n - 1)]),                     # path
        undirected(n, [(0, i) for i in range(1, n)]),                          # star
        undirected(12, [(i, j) for i in range(12) for j in range(i + 1, 12)]),  # K_12
        undirected(11, [(i, (i + 1) % 11) for i in range(11)]),                # cycle
        undirected(6, [(0, 1), (2, 3)]),                                       # pieces, isolated
        star_plus(300), star_plus(1500),                                       # long rows
    ]
    for g in cases:
        G = gr.Graph.from_csr(g)
        for src in sorted({0, g.n - 1, g.n // 2}):
            for big in (32, 1 << 30):
                check(g, src, *run_bc(gr, G, src, big_degree=big))
        bc = torch.zeros(g.n, dtype=torch.float64, device="cuda")
        for s in range(g.n if g.n <= 40 else 3):
            run_bc(gr, G, s, bc=bc)
        close(host(bc), oracle.bc(g.R, g.C, list(range(g.n if g.n <= 40 else 3))))
        G.close()


def test_directed_graph(gr):
    rng = np.random.default_rng(3)
    n = 2000
    s, t = rng.integers(0, n, 12000), rng.integers(0, n, 12000)
    keep = s != t
    pairs = np.unique(np.stack([s[keep], t[keep]], 1), axis=0)
    g = gg.directed(n, pairs[:, 0], pairs[:, 1])
    G = gr.Graph.from_csr(g, symmetric=False)
    for src in (0, 17):
        check(g, src, *run_bc(gr, G, src))
    G.close()


def test_path_count_overflow_is_reported(gr):
    def diamonds(k):
        pairs, top = [], 0
        for i in range(k):
            a, b, bot = 3 * i + 1, 3 * i + 2, 3 * i + 3
            pairs += [(top, a), (top, b), (a, bot), (b, bot)]
            top = bot
        return undirected(3 * k + 1, pairs), top
    g, end = diamonds(62)                      # 2^62 paths: representable
    G = gr.Graph.from_csr(g)
    d, s, dl = run_bc(gr, G, 0)
    assert int(s[end]) == 2 ** 62
    check(g, 0, d, s, dl)
    G.close()
    g, end = diamonds(63)                      # 2^63 paths: one more than INT64_MAX
    G = gr.Graph.from_csr(g)
    run_bc(gr, G, 0, expect=gr.GR_ERR_OVERFLOW)
    d, s, dl = run_bc(gr, G, 0, expect=gr.GR_ERR_OVERFLOW)
    assert G.sync_status() == gr.GR_OK          # the status word was read and cleared
    G.close()


def test_invalid_arguments_rejected(gr, s16):
    import torch
    g, G = s16
    with pytest.raises(gr.GrError):
        gr.gr_bc(G.handle, -1)
    with pytest.raises(gr.GrError):
        gr.gr_bc(G.handle, g.n)
    with pytest.raises(ValueError):
        gr.gr_bc(G.handle, 0, sigma=torch.empty(g.n, dtype=torch.int32, device="cuda"))
