"""GPU parity at the full workload sizes, in the configuration bench.py times
(the library's tuned schedules, sched = NULL), against the CPU oracle:

* RMAT scale 22 (4,194,304 vertices, ~128M arcs): BFS depth and parent
  bit-exact, CC labels bit-exact, PageRank (20 rounds, d = 0.85) with
  L1 <= 1e-5 against the fp64 oracle.
* Road grid 4096 x 4096 (16.8M vertices, 10% deletions, 1% shortcuts,
  weights U[1, 1000]): delta-stepping SSSP (plain and fused, several deltas)
  and BFS (plain and fused) bit-exact.
* RMAT scale 21 batched: 64-source BFS and 32-source SSSP on sampled rows,
  BC from 16 sources (relative 1e-6).
"""
import numpy as np
import pytest

import oracle
from paper_2012_07990_gb300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2 as mod
    return mod


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def rmat22():
    return gg.rmat(22, seed=1)


@pytest.fixture(scope="module")
def grid4096():
    g = gg.road_grid(4096, seed=1)
    return g, gg.pair_weights(g, 1000, seed=1)


def test_rmat22_bfs_cc_pr(g2, rmat22):
    g = rmat22
    dg = g2.load_graph(g)
    src = g.max_degree_vertex()
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    g2.g2_bfs(dg, src, d, p, None)
    od, op = oracle.bfs_graph(g, src)
    assert np.array_equal(host(d), od)
    assert np.array_equal(host(p), op)
    lab = torch.empty(g.n, dtype=torch.int32, device="cuda")
    g2.g2_cc(dg, lab, None)
    assert np.array_equal(host(lab), oracle.cc_graph(g))
    rank = torch.empty(g.n, dtype=torch.float32, device="cuda")
    g2.g2_pagerank(dg, 0.85, 20, rank, None)
    ref = oracle.pagerank_graph(g, 0.85, 20)
    l1 = float(np.abs(host(rank).astype(np.float64) - ref).sum())
    assert l1 <= 1e-5, l1


def test_grid4096_sssp_and_bfs(g2, grid4096):
    g, w = grid4096
    dg = g2.load_graph(g, w)
    src = 0
    want = oracle.sssp_graph(g, w, src)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for delta, sched in ((4096, None), (1024, g2.schedule("VERTEX_BASED", kernel_fusion=True)),
                         (4096, g2.schedule("WM", kernel_fusion=True)),
                         (64, g2.schedule("CM", kernel_fusion=True))):
        g2.g2_sssp_delta(dg, src, delta, dist, sched)
        assert np.array_equal(host(dist), want), delta
    od, op = oracle.bfs_graph(g, src)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for sched in (None, g2.schedule("VERTEX_BASED", kernel_fusion=True)):
        g2.g2_bfs(dg, src, d, p, sched)
        assert np.array_equal(host(d), od)
        assert np.array_equal(host(p), op)


def test_rmat21_batched(g2):
    g = gg.rmat(21, seed=1)
    srcs = gg.random_sources(g, 64, seed=1)
    dg = g2.load_graph(g)
    depth = torch.empty(64 * g.n, dtype=torch.int32, device="cuda")
    g2.g2_bfs_batch(dg, srcs, depth, None)
    got = host(depth).reshape(64, g.n)
    for i in (0, 17, 40, 63):
        assert np.array_equal(got[i], oracle.bfs_graph(g, srcs[i], want_parent=False)[0]), i
    w = gg.pair_weights(g, 255, seed=1)
    dgw = g2.load_graph(g, w)
    s32 = srcs[:32]
    dist = torch.empty(32 * g.n, dtype=torch.int32, device="cuda")
    g2.g2_sssp_batch(dgw, s32, 64, dist, None)
    gotd = host(dist).reshape(32, g.n)
    for i in (0, 31):
        assert np.array_equal(gotd[i], oracle.sssp_graph(g, w, s32[i])), i
    s16 = srcs[:16]
    bc = torch.empty(g.n, dtype=torch.float64, device="cuda")
    g2.g2_bc(dg, s16, bc, None)
    want = oracle.bc_graph(g, s16)
    got = host(bc)
    tol = 1e-6 * np.abs(want) + 1e-12 * max(np.abs(want).max(), 1.0)
    assert np.all(np.abs(got - want) <= tol)
