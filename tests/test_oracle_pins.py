"""Pins for the CPU oracle: each oracle function is checked against something
other than itself -- hand-worked fixtures (tests/golden), closed forms, brute
force on tiny graphs, library routines (scipy.sparse.csgraph, networkx where
installed) and invariants -- so that a dropped term, a wrong sign or index or a
transposed operand fails at least one test.  CPU only.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
from paper_2012_07990_gb300 import graphgen as gg

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def adj_matrix(g):
    a = np.zeros((g.n, g.n), dtype=bool)
    for u in range(g.n):
        a[u, g.col[g.rowptr[u]:g.rowptr[u + 1]]] = True
    return a


def scipy_csr(g, data=None):
    d = np.ones(g.m) if data is None else np.asarray(data, dtype=np.float64)
    return sp.csr_matrix((d, g.col, g.rowptr), shape=(g.n, g.n))


def tiny_graphs():
    out = [gg.path(1), gg.path(2), gg.path(7), gg.star(6), gg.cycle(5), gg.cycle(6),
           gg.complete(5), gg.full_grid(3, 4),
           gg.disjoint_union(gg.path(3), gg.cycle(4), gg.star(4)),
           gg.from_arcs(5, [], [], name="empty5")]
    for seed in range(6):
        out.append(gg.gnp(9, 0.3, seed))
        out.append(gg.gnp(8, 0.35, 100 + seed, symmetric=False))
    return out


# ------------------------------------------------------------------ brute force helpers
def bf_depth(g, s):
    """Hop distances by boolean matrix powers (no queue)."""
    a = adj_matrix(g)
    depth = np.full(g.n, -1)
    reach = np.zeros(g.n, bool)
    reach[s] = True
    depth[s] = 0
    k = 0
    while True:
        k += 1
        nxt = (reach[:, None] & a).any(axis=0) & (depth < 0)
        if not nxt.any():
            break
        depth[nxt] = k
        reach = nxt
    return depth


def all_shortest_paths(g, s, t, depth):
    """Every shortest s->t path, by depth-first enumeration of arc sequences."""
    a = adj_matrix(g)
    L = depth[t]
    if L < 0:
        return []
    out = []

    def rec(path):
        u = path[-1]
        if len(path) - 1 == L:
            if u == t:
                out.append(list(path))
            return
        for v in np.nonzero(a[u])[0]:
            path.append(int(v))
            rec(path)
            path.pop()

    rec([s])
    return out


# ----------------------------------------------------------------------------- BFS
def test_bfs_golden():
    gd = load_gold("bfs_small.json")
    e = np.array(gd["edges"])
    g = gg.from_arcs(gd["n"], e[:, 0], e[:, 1])
    depth, parent = oracle.bfs_graph(g, gd["src"])
    assert depth.tolist() == gd["depth"]
    assert parent.tolist() == gd["parent"]


@pytest.mark.parametrize("gi", range(22))
def test_bfs_bruteforce(gi):
    g = tiny_graphs()[gi]
    for s in range(g.n):
        depth, parent = oracle.bfs_graph(g, s)
        assert depth.tolist() == bf_depth(g, s).tolist()
        for v in range(g.n):
            paths = all_shortest_paths(g, s, v, depth) if v != s else []
            if v == s:
                assert parent[v] == s
            elif depth[v] < 0:
                assert parent[v] == -1
            else:
                assert parent[v] == min(p[-2] for p in paths)


def test_bfs_closed_forms():
    g = gg.path(9)
    d, p = oracle.bfs_graph(g, 3)
    assert d.tolist() == [abs(i - 3) for i in range(9)]
    assert p.tolist() == [1, 2, 3, 3, 3, 4, 5, 6, 7]
    W, H = 7, 5
    g = gg.full_grid(W, H)
    d, p = oracle.bfs_graph(g, 0)
    for y in range(H):
        for x in range(W):
            v = y * W + x
            assert d[v] == x + y
            if v:
                assert p[v] == ((y - 1) * W + x if y > 0 else v - 1)


def test_bfs_scipy_and_invariants_rmat():
    g = gg.rmat(12)
    s = g.max_degree_vertex()
    depth, parent = oracle.bfs_graph(g, s)
    ref = csg.shortest_path(scipy_csr(g), unweighted=True, indices=s)
    ref = np.where(np.isinf(ref), -1, ref).astype(np.int64)
    assert np.array_equal(depth, ref)
    src = np.repeat(np.arange(g.n), g.degrees())
    both = (depth[src] >= 0) & (depth[g.col] >= 0)
    assert np.all(np.abs(depth[src][both] - depth[g.col][both]) <= 1)
    reached = np.nonzero(depth > 0)[0]
    pp = parent[reached]
    assert np.all(depth[pp] == depth[reached] - 1)
    a = scipy_csr(g)
    assert np.all(np.asarray(a[pp, reached]).ravel() == 1)
    # reached set == component of the source
    _, comp = csg.connected_components(a, directed=False)
    assert np.array_equal(depth >= 0, comp == comp[s])


# ------------------------------------------------------------------------------ CC
def canon_min(labels):
    out = np.empty_like(labels)
    for c in np.unique(labels):
        idx = np.nonzero(labels == c)[0]
        out[idx] = idx.min()
    return out


@pytest.mark.parametrize("gi", range(22))
def test_cc_bruteforce(gi):
    g = tiny_graphs()[gi]
    a = adj_matrix(g)
    a = a | a.T | np.eye(g.n, dtype=bool)
    reach = a.copy()
    for _ in range(g.n):
        reach = (reach.astype(np.int64) @ a.astype(np.int64)) > 0
    want = np.array([np.nonzero(reach[v])[0].min() for v in range(g.n)]) if g.n else np.zeros(0)
    assert oracle.cc_graph(g).tolist() == want.tolist()


def test_cc_scipy():
    for g in [gg.rmat(12), gg.road_grid(48, 40, p_delete=0.45, seed=3)]:
        _, lab = csg.connected_components(scipy_csr(g), directed=False)
        got = oracle.cc_graph(g)
        assert np.array_equal(got, canon_min(lab))
        src = np.repeat(np.arange(g.n), g.degrees())
        assert np.all(got[src] == got[g.col])
        assert np.all(got <= np.arange(g.n))


# ---------------------------------------------------------------------------- SSSP
def floyd_warshall(g, w):
    INF = np.iinfo(np.int64).max // 4
    d = np.full((g.n, g.n), INF, dtype=np.int64)
    np.fill_diagonal(d, 0)
    for u in range(g.n):
        for e in range(g.rowptr[u], g.rowptr[u + 1]):
            d[u, g.col[e]] = min(d[u, g.col[e]], w[e])
    for k in range(g.n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return d, INF


@pytest.mark.parametrize("gi", range(22))
def test_sssp_bruteforce(gi):
    g = tiny_graphs()[gi]
    w = gg.pair_weights(g, 9, seed=gi) if g.symmetric else \
        (np.arange(g.m, dtype=np.int32) * 7 % 5 + 1).astype(np.int32)
    d, INF = floyd_warshall(g, w)
    for s in range(g.n):
        got = oracle.sssp_graph(g, w, s)
        want = np.where(d[s] >= INF, oracle.INF32, d[s])
        assert got.tolist() == want.tolist()


def test_sssp_scipy_and_invariants():
    for g, wmax in [(gg.rmat(12), 255), (gg.road_grid(40), 1000)]:
        w = gg.pair_weights(g, wmax, seed=1)
        s = g.max_degree_vertex()
        got = oracle.sssp_graph(g, w, s)
        ref = csg.dijkstra(scipy_csr(g, w), indices=s)
        want = np.where(np.isinf(ref), oracle.INF32, ref).astype(np.int64)
        assert np.array_equal(got.astype(np.int64), want)
        src = np.repeat(np.arange(g.n), g.degrees())
        fin = got[src] < oracle.INF32
        assert np.all(got[g.col][fin].astype(np.int64) <= got[src][fin].astype(np.int64) + w[fin])
        # witness arc with equality for every reached vertex except the source
        tight = fin & (got[g.col].astype(np.int64) == got[src].astype(np.int64) + w)
        has = np.zeros(g.n, bool)
        has[g.col[tight]] = True
        reached = got < oracle.INF32
        reached[s] = False
        assert np.all(has[reached])


def test_sssp_unit_weights_equal_bfs():
    g = gg.rmat(11)
    s = g.max_degree_vertex()
    d = oracle.sssp_graph(g, np.ones(g.m, np.int32), s)
    depth, _ = oracle.bfs_graph(g, s, want_parent=False)
    assert np.array_equal(np.where(depth < 0, oracle.INF32, depth), d)


# ------------------------------------------------------------------------ PageRank
def google_power(g, d, iters):
    """Dense Google-matrix power iteration (a different code path: matrix form)."""
    n = g.n
    a = adj_matrix(g).astype(np.float64)
    out = a.sum(axis=1)
    P = np.zeros((n, n))
    for u in range(n):
        P[:, u] = a[u] / out[u] if out[u] > 0 else 1.0 / n
    M = d * P + (1 - d) / n
    return np.linalg.matrix_power(M, iters) @ np.full(n, 1.0 / n)


def test_pagerank_golden_fractions():
    gd = load_gold("pagerank_dangling.json")
    arcs = np.array(gd["arcs"])
    g = gg.from_arcs(gd["n"], arcs[:, 0], arcs[:, 1], symmetric=False)
    x = oracle.pagerank_graph(g, gd["damping"], gd["iters"])
    want = [float(Fraction(a, b)) for a, b in zip(gd["x_num"], gd["x_den"])]
    assert np.allclose(x, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("gi", range(22))
def test_pagerank_dense(gi):
    g = tiny_graphs()[gi]
    for iters in (1, 2, 20):
        x = oracle.pagerank_graph(g, 0.85, iters)
        assert np.allclose(x, google_power(g, 0.85, iters), rtol=1e-12, atol=1e-15)


def test_pagerank_closed_forms_and_sum():
    for g in [gg.cycle(11), gg.complete(7), gg.from_arcs(6, [], [])]:
        x = oracle.pagerank_graph(g, 0.85, 20)
        assert np.allclose(x, 1.0 / g.n, rtol=0, atol=1e-15)
    # K_c beside k isolated vertices: every vertex of K_c holds a_t, every
    # isolated one b_t, and only the isolated ones are dangling (D = k b), so
    #   a_t = (1-d)/n + d (a_{t-1} + k b_{t-1} / n),  b_t = (1-d)/n + d k b_{t-1} / n
    # from a_0 = b_0 = 1/n (by symmetry, in exact fractions)
    c, k = 6, 9
    n = c + k
    g = gg.disjoint_union(gg.complete(c), gg.from_arcs(k, [], []))
    d = Fraction(85, 100)
    a = b = Fraction(1, n)
    for _ in range(20):
        a, b = (1 - d) / n + d * (a + k * b / n), (1 - d) / n + d * k * b / n
    x = oracle.pagerank_graph(g, 0.85, 20)
    assert np.allclose(x[:c], float(a), rtol=0, atol=1e-15)
    assert np.allclose(x[c:], float(b), rtol=0, atol=1e-15)
    assert c * a + k * b == 1
    g = gg.rmat(12)
    x = oracle.pagerank_graph(g, 0.85, 20)
    assert abs(x.sum() - 1.0) < 1e-12
    nx = pytest.importorskip("networkx")
    # networkx's uniform-dangling PageRank, run to convergence, agrees after many rounds
    G = nx.DiGraph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), g.degrees())
    G.add_edges_from(zip(src.tolist(), g.col.tolist()))
    ref = nx.pagerank(G, alpha=0.85, tol=1e-15, max_iter=500)
    x200 = oracle.pagerank_graph(g, 0.85, 200)
    assert np.abs(x200 - np.array([ref[v] for v in range(g.n)])).sum() < 1e-9


# ------------------------------------------------------------------------------ BC
def bf_bc(g, sources):
    """Sum over s in sources and t != s of sigma_st(v)/sigma_st, by enumerating
    every shortest path explicitly."""
    bc = np.zeros(g.n)
    for s in sources:
        depth = bf_depth(g, s)
        for t in range(g.n):
            if t == s or depth[t] < 0:
                continue
            paths = all_shortest_paths(g, s, t, depth)
            for p in paths:
                for v in p[1:-1]:
                    bc[v] += 1.0 / len(paths)
    return bc


def test_bc_golden():
    gd = load_gold("bc_small.json")
    e = np.array(gd["edges"])
    g = gg.from_arcs(gd["n"], e[:, 0], e[:, 1])
    assert np.allclose(oracle.bc_graph(g, gd["sources"]), gd["bc"], rtol=0, atol=1e-15)


@pytest.mark.parametrize("gi", range(22))
def test_bc_bruteforce(gi):
    g = tiny_graphs()[gi]
    if g.n > 10:
        pytest.skip("enumeration too large")
    srcs = list(range(g.n))
    got = oracle.bc_graph(g, srcs)
    assert np.allclose(got, bf_bc(g, srcs), rtol=1e-12, atol=1e-12)
    if g.n:
        sub = srcs[::3]
        assert np.allclose(oracle.bc_graph(g, sub), bf_bc(g, sub), rtol=1e-12, atol=1e-12)


def test_bc_closed_forms():
    n = 9
    x = oracle.bc_graph(gg.path(n), list(range(n)))
    assert x.tolist() == [2.0 * i * (n - 1 - i) for i in range(n)]
    x = oracle.bc_graph(gg.star(n), list(range(n)))
    assert x[0] == (n - 1) * (n - 2) and np.all(x[1:] == 0)


def test_bc_networkx():
    nx = pytest.importorskip("networkx")
    g = gg.gnp(40, 0.12, 7)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), g.degrees())
    G.add_edges_from(zip(src.tolist(), g.col.tolist()))
    ref = nx.betweenness_centrality(G, normalized=False)
    got = oracle.bc_graph(g, list(range(g.n)))
    # networkx halves undirected betweenness; this definition does not
    assert np.allclose(got, [2 * ref[v] for v in range(g.n)], rtol=1e-12, atol=1e-9)


def test_bc_long_double_large_counts():
    """Path counts beyond fp64 on a full grid stay finite (long double)."""
    W = 600  # corner-to-corner path count C(1198, 599) ~ 1e359 > fp64 max
    g = gg.full_grid(W, W)
    x = oracle.bc_graph(g, [0])
    assert np.all(np.isfinite(x)) and x.max() > 0
    # by symmetry of the square grid about its diagonal from the corner
    v = np.arange(g.n)
    xs, ys = v % W, v // W
    assert np.allclose(x, x[xs * W + ys], rtol=1e-9)


# -------------------------------------------------------------------- EdgeBlocking
def test_edgeblock_golden():
    gd = load_gold("edgeblock_small.json")
    os_, od, seg_end, ns = oracle.edgeblock(gd["n"], gd["src"], gd["dst"], gd["N"])
    assert ns == 3
    assert os_.tolist() == gd["out_src"]
    assert od.tolist() == gd["out_dst"]
    assert seg_end.tolist() == gd["seg_end"]


@pytest.mark.parametrize("N", [1, 3, 64, 1000, 5000])
def test_edgeblock_is_stable_sort(N):
    g = gg.rmat(10)
    src = np.repeat(np.arange(g.n, dtype=np.int32), g.degrees())
    dst = g.col
    os_, od, seg_end, ns = oracle.edgeblock(g.n, src, dst, N)
    order = np.argsort(dst // N, kind="stable")
    assert np.array_equal(os_, src[order]) and np.array_equal(od, dst[order])
    counts = np.bincount(dst // N, minlength=ns)
    assert np.array_equal(seg_end[:ns], np.cumsum(counts))
    assert seg_end[ns] == g.m


# ------------------------------------------------------------------------ ETWC split
@pytest.mark.parametrize("deg", [0, 1, 31, 32, 33, 255, 256, 257, 300, 1000, 4096, 5000])
def test_etwc_split(deg):
    start = 1000
    parts = oracle.etwc_split(start, start + deg, 32, 256)
    (t0, t1), (w0, w1), (c0, c1) = parts
    assert c0 == start and (c1 - c0) == (deg // 256) * 256
    assert w0 == c1 and (w1 - w0) == ((deg % 256) // 32) * 32
    assert t0 == w1 and t1 == start + deg and (t1 - t0) == deg % 32
    covered = list(itertools.chain(range(c0, c1), range(w0, w1), range(t0, t1)))
    assert covered == list(range(start, start + deg))
