"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs, element by element.

Tolerances: BFS depth/parent, CC labels, SSSP distances and EdgeBlocking
arrays bit-exact; PageRank L1(gpu, fp64 oracle) <= 1e-5; BC
|gpu - oracle| <= 1e-6 |oracle| + 1e-12 max|oracle|.

Sizes: RMAT scale 14 (16,384 vertices, ~426K arcs: many CTA tiles and a
ragged tail), road grids up to 256^2, tiny and degenerate graphs.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2012_07990_gb300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PR_L1 = 1e-5
BC_REL, BC_ABS = 1e-6, 1e-12


@pytest.fixture(scope="module")
def g2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2 as mod
    return mod


def dev(n, dtype=torch.int32):
    return torch.empty(n, dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def rmat14():
    return gg.rmat(14, seed=1)


@pytest.fixture(scope="module")
def grid():
    return gg.road_grid(128, seed=1)


def edge_cases():
    return [
        gg.from_arcs(1, [], [], name="single"),
        gg.from_arcs(4, [], [], name="isolated4"),
        gg.path(2), gg.path(37), gg.star(300), gg.cycle(1000), gg.complete(40),
        gg.disjoint_union(gg.path(5), gg.star(70), gg.complete(9)),
        gg.full_grid(33, 7),
        gg.gnp(200, 0.02, 3, symmetric=False),
        gg.gnp(500, 0.01, 4, symmetric=False),
    ]


LBS = ["VERTEX_BASED", "WM", "CM", "STRICT", "TWC", "ETWC"]


def push_scheds(g2):
    out = []
    for lb in LBS:
        out.append((f"{lb}/fused", g2.schedule(lb)))
    out.append(("VB/unfused-bitmap", g2.schedule("VERTEX_BASED", frontier_creation=g2.G2_UNFUSED_BITMAP)))
    out.append(("WM/unfused-boolmap", g2.schedule("WM", frontier_creation=g2.G2_UNFUSED_BOOLMAP)))
    out.append(("CM/dedup-bitmap", g2.schedule("CM", dedup_type=g2.G2_DEDUP_BITMAP)))
    out.append(("ETWC/dedup-boolmap", g2.schedule("ETWC", dedup_type=g2.G2_DEDUP_BOOLMAP)))
    out.append(("TWC/no-dedup", g2.schedule("TWC", dedup=False)))
    return out


def pull_sched(g2, lb="VERTEX_BASED", rep=None, fc=None):
    return g2.schedule(lb, direction=g2.G2_PULL, pull_frontier=rep if rep is not None else g2.G2_BITMAP,
                       frontier_creation=fc if fc is not None else g2.G2_UNFUSED_BITMAP, dedup=False)


# ----------------------------------------------------------------------- BFS
def run_bfs(g2, g, src, sched, parent=True):
    dg = g2.load_graph(g)
    d = dev(g.n)
    p = dev(g.n) if parent else None
    g2.g2_bfs(dg, src, d, p, sched)
    return host(d), (host(p) if parent else None)


def test_bfs_push_schedules(g2, rmat14):
    src = rmat14.max_degree_vertex()
    od, op = oracle.bfs_graph(rmat14, src)
    for name, s in push_scheds(g2):
        d, p = run_bfs(g2, rmat14, src, s)
        assert np.array_equal(d, od), name
        assert np.array_equal(p, op), name


@pytest.mark.parametrize("lb", ["VERTEX_BASED", "WM", "CM"])
@pytest.mark.parametrize("rep", ["bitmap", "boolmap"])
@pytest.mark.parametrize("fc", ["fused", "bitmap", "boolmap"])
def test_bfs_direction_optimising(g2, rmat14, lb, rep, fc):
    src = rmat14.max_degree_vertex()
    od, op = oracle.bfs_graph(rmat14, src)
    r = g2.G2_BITMAP if rep == "bitmap" else g2.G2_BOOLMAP
    f = {"fused": g2.G2_FUSED, "bitmap": g2.G2_UNFUSED_BITMAP, "boolmap": g2.G2_UNFUSED_BOOLMAP}[fc]
    for tau in (0.0, 0.02, 2.0):  # always pull / switching / always push
        h = g2.hybrid(g2.schedule("ETWC"), pull_sched(g2, lb, r, f), tau)
        d, p = run_bfs(g2, rmat14, src, h)
        assert np.array_equal(d, od), (lb, rep, fc, tau)
        assert np.array_equal(p, op), (lb, rep, fc, tau)


@pytest.mark.parametrize("lb", ["VERTEX_BASED", "WM", "CM", "ETWC"])
def test_bfs_fused(g2, rmat14, grid, lb, monkeypatch):
    """The grid-wide persistent loop (the one-cluster loop switched off)."""
    monkeypatch.setenv("G2_FUSED_CLUSTER", "0")
    for g in (rmat14, grid):
        src = g.max_degree_vertex()
        od, op = oracle.bfs_graph(g, src)
        d, p = run_bfs(g2, g, src, g2.schedule(lb, kernel_fusion=True))
        assert np.array_equal(d, od) and np.array_equal(p, op), lb
        st = g2.g2_last_stats()
        assert st["launches"] == 1 and st["iterations"] == od.max() + 1


@pytest.mark.parametrize("lb", ["CM", "WM", "VERTEX_BASED", "ETWC", "STRICT"])
def test_bfs_fused_direction_optimising(g2, rmat14, grid, lb):
    """The direction-optimising hybrid in one launch: PUSH levels from a list,
    PULL levels over a bitmap, the representation converted where the
    direction changes; depth and the canonical parent bit-exact for the
    thresholds that always pull, switch, and always push, on power-law,
    grid, directed, star and path graphs."""
    # star(10000): ETWC hands the centre's 9,984-arc CTA part to the
    # grid-wide pass inside the launch; STRICT takes its prefix sum over the
    # grid inside the launch (the path: one vertex per level)
    graphs = [rmat14, grid, gg.gnp(400, 0.02, 11, symmetric=False), gg.star(3000),
              gg.star(10000), gg.path(700), gg.from_arcs(5, [], [])]
    pull = g2.schedule("VERTEX_BASED", direction=g2.G2_PULL, pull_frontier=g2.G2_BITMAP,
                       frontier_creation=g2.G2_UNFUSED_BITMAP, dedup=False, kernel_fusion=True)
    for g in graphs:
        src = g.max_degree_vertex() if g.m else 0
        od, op = oracle.bfs_graph(g, src)
        for tau in (0.0, 0.02, 0.3, 2.0):
            h = g2.hybrid(g2.schedule(lb, kernel_fusion=True), pull, tau)
            d, p = run_bfs(g2, g, src, h)
            assert np.array_equal(d, od), (g.name, lb, tau)
            assert np.array_equal(p, op), (g.name, lb, tau)
            st = g2.g2_last_stats()
            assert st["launches"] == 1 and st["iterations"] == od.max() + 1, (g.name, lb, tau, st)


def _handover_launches(levels, hi, lo):
    """Launches of a fused WM BFS whose levels (vertex counts by depth) move
    between the one-cluster loop (until a level holds more than `hi`) and the
    grid-wide loop (until a level holds fewer than `lo`); each launch runs its
    first level unconditionally."""
    level, in_cluster, launches = 0, True, 0
    while True:
        launches += 1
        d = level + 1
        while d < len(levels) and levels[d] > 0:
            if (levels[d] > hi) if in_cluster else (levels[d] < lo):
                break
            d += 1
        if d >= len(levels) or levels[d] == 0:
            return launches
        level, in_cluster = d, not in_cluster


@pytest.mark.parametrize("hi,lo", [(16384, 8192), (64, 16), (1, 1)])
def test_bfs_in_one_cluster(g2, rmat14, grid, monkeypatch, hi, lo):
    """A fused WM BFS runs its small levels inside one thread-block cluster
    (frontier queues in shared memory, cluster barriers) and its large ones in
    the grid-wide loop, handing the frontier over at level boundaries; the
    launch count follows the level sizes.  A level that outgrows a CTA's queue
    (a star's 30,000 leaves found by one CTA) is rebuilt from the depths and
    the grid-wide loop finishes (three launches)."""
    monkeypatch.delenv("G2_FUSED_CLUSTER", raising=False)
    monkeypatch.setenv("G2_CLUSTER_HI", str(hi))
    monkeypatch.setenv("G2_CLUSTER_LO", str(lo))
    star = gg.star(30001)
    for g in (grid, rmat14, gg.road_grid(300, seed=4), star, gg.path(5000)):
        dg = g2.load_graph(g)
        for src in (0, g.n - 1, g.n // 3):
            od, op = oracle.bfs_graph(g, src)
            d, p = dev(g.n), dev(g.n)
            g2.g2_bfs(dg, src, d, p, g2.schedule("WM", kernel_fusion=True))
            assert np.array_equal(host(d), od) and np.array_equal(host(p), op), (g.name, src)
            st = g2.g2_last_stats()
            assert st["iterations"] == od.max() + 1, (g.name, src)
            levels = np.bincount(od[od >= 0])
            want = 3 if g is star else _handover_launches(levels, hi, lo)
            assert st["launches"] == want, (g.name, src, st["launches"], want)
            # depths alone (no parent array)
            d2 = dev(g.n)
            g2.g2_bfs(dg, src, d2, None, g2.schedule("WM", kernel_fusion=True))
            assert np.array_equal(host(d2), od), (g.name, src)


def test_half_fused_hybrid_is_rejected(g2, grid):
    """A hybrid whose s1 asks for kernel fusion and whose s2 does not is
    rejected by BFS, SSSP and BC (a fused loop runs s1 throughout); with s2
    fused as well it runs, and gives the oracle's result."""
    w = gg.pair_weights(grid, 100, seed=2)
    dg = g2.load_graph(grid, w)
    fused = g2.schedule("WM", kernel_fusion=True)
    half = g2.hybrid(fused, g2.schedule("VERTEX_BASED"), 0.02)
    calls = (lambda s: g2.g2_bfs(dg, 0, dev(grid.n), None, s),
             lambda s: g2.g2_sssp_delta(dg, 0, 64, dev(grid.n), s),
             lambda s: g2.g2_bc(dg, [0], dev(grid.n, torch.float64), s))
    for call in calls:
        with pytest.raises(g2.G2Error) as e:
            call(half)
        assert e.value.status == g2.G2_EUNSUPPORTED
    both = g2.hybrid(fused, fused, 0.02)
    d = dev(grid.n)
    g2.g2_bfs(dg, 0, d, None, both)
    assert np.array_equal(host(d), oracle.bfs_graph(grid, 0)[0])
    dist = dev(grid.n)
    g2.g2_sssp_delta(dg, 0, 64, dist, both)
    assert np.array_equal(host(dist), oracle.sssp_graph(grid, w, 0))


def test_eight_cta_clusters(g2, grid, monkeypatch):
    """The one-cluster loops with 8-CTA clusters (the portable size, used
    where a 16-CTA cluster does not fit): BFS, delta-stepping SSSP and BC on
    road grids, with low hand-over thresholds so that the grid-wide kernels
    take part too."""
    monkeypatch.setenv("G2_FUSED_CLUSTER", "8")
    monkeypatch.setenv("G2_CLUSTER_HI", "200")
    monkeypatch.setenv("G2_CLUSTER_LO", "100")
    monkeypatch.setenv("G2_CLUSTER_FAR_LO", "100")
    monkeypatch.setenv("G2_CLUSTER_BC_HI", "200")
    monkeypatch.setenv("G2_CLUSTER_BC_LO", "100")
    s = g2.schedule("WM", kernel_fusion=True)
    for g in (grid, gg.road_grid(300, seed=4)):
        w = gg.pair_weights(g, 1000, seed=6)
        dg = g2.load_graph(g, w)
        for src in (0, g.n // 2):
            od, op = oracle.bfs_graph(g, src)
            d, p = dev(g.n), dev(g.n)
            g2.g2_bfs(dg, src, d, p, s)
            assert np.array_equal(host(d), od) and np.array_equal(host(p), op), (g.name, src)
            dist = dev(g.n)
            g2.g2_sssp_delta(dg, src, 700, dist, s)
            assert np.array_equal(host(dist), oracle.sssp_graph(g, w, src)), (g.name, src)
        srcs = np.array([0, g.n - 1, g.n // 3], dtype=np.int32)
        bc = dev(g.n, torch.float64)
        g2.g2_bc(dg, srcs, bc, s)
        assert bc_close(host(bc), oracle.bc_graph(g, srcs)), g.name


def test_null_schedule_follows_the_degree_bound(g2, rmat14, grid):
    """With no schedule, a bounded-degree graph (road grid, largest degree
    <= 32) runs BFS, SSSP and BC as one fused kernel; on a power-law graph
    BFS runs the direction-optimising hybrid fused into one launch, with
    PULL levels.  Results are the oracle's either way."""
    w = gg.pair_weights(grid, 1000, seed=2)
    dg = g2.load_graph(grid, w)
    od, op = oracle.bfs_graph(grid, 3)
    d, p = dev(grid.n), dev(grid.n)
    g2.g2_bfs(dg, 3, d, p, None)
    assert np.array_equal(host(d), od) and np.array_equal(host(p), op)
    assert g2.g2_last_stats()["launches"] == 1
    dist = dev(grid.n)
    g2.g2_sssp_delta(dg, 3, 512, dist, None)
    assert np.array_equal(host(dist), oracle.sssp_graph(grid, w, 3))
    assert g2.g2_last_stats()["launches"] == 1
    bc = dev(grid.n, torch.float64)
    g2.g2_bc(dg, [3, 77], bc, None)
    assert bc_close(host(bc), oracle.bc_graph(grid, [3, 77]))
    dr = g2.load_graph(rmat14)
    d = dev(rmat14.n)
    p = dev(rmat14.n)
    g2.g2_bfs(dr, 0, d, p, None)
    od, op = oracle.bfs_graph(rmat14, 0)
    assert np.array_equal(host(d), od) and np.array_equal(host(p), op)
    st = g2.g2_last_stats()
    assert st["launches"] == 1 and st["pull_rounds"] > 0, st


def test_bfs_edge_cases(g2):
    for g in edge_cases():
        for src in sorted({0, g.n - 1, g.n // 2}):
            od, op = oracle.bfs_graph(g, src)
            for s in (g2.schedule("ETWC"), g2.schedule("TWC"), g2.schedule("STRICT"),
                      g2.hybrid(g2.schedule("WM"), pull_sched(g2), 0.1),
                      g2.schedule("CM", kernel_fusion=True)):
                d, p = run_bfs(g2, g, src, s)
                assert np.array_equal(d, od), g.name
                assert np.array_equal(p, op), g.name


def test_bfs_default_and_depth_only(g2, rmat14):
    src = 123
    od, _ = oracle.bfs_graph(rmat14, src)
    d, _ = run_bfs(g2, rmat14, src, None, parent=False)
    assert np.array_equal(d, od)


# ------------------------------------------------------------------------ CC
def cc_scheds(g2):
    out = [(lb, g2.schedule(lb)) for lb in LBS + ["EDGE_ONLY"]]
    out += [(f"pull-{lb}", pull_sched(g2, lb)) for lb in ("VERTEX_BASED", "WM", "CM")]
    out.append(("hybrid", g2.hybrid(g2.schedule("ETWC"), pull_sched(g2, "VERTEX_BASED", g2.G2_BOOLMAP), 0.3)))
    return out


def test_cc(g2, rmat14):
    grid_sparse = gg.road_grid(96, p_delete=0.45, seed=5)
    for g in (rmat14, grid_sparse, gg.disjoint_union(gg.path(5), gg.star(70), gg.complete(9))):
        want = oracle.cc_graph(g)
        dg = g2.load_graph(g)
        for name, s in cc_scheds(g2) + [("default", None)]:
            lab = dev(g.n)
            g2.g2_cc(dg, lab, s)
            assert np.array_equal(host(lab), want), (g.name, name)


# ---------------------------------------------------------------------- SSSP
def test_sssp_delta_sweep(g2, rmat14, grid):
    cases = [(rmat14, gg.pair_weights(rmat14, 255, seed=1)), (grid, gg.pair_weights(grid, 1000, seed=1))]
    for g, w in cases:
        src = 0 if g is grid else g.max_degree_vertex()
        want = oracle.sssp_graph(g, w, src)
        dg = g2.load_graph(g, w)
        for delta in (1, 7, 64, 1000, 4096):
            for lb in ("VERTEX_BASED", "WM", "CM", "STRICT", "TWC", "ETWC"):
                dist = dev(g.n)
                g2.g2_sssp_delta(dg, src, delta, dist, g2.schedule(lb))
                assert np.array_equal(host(dist), want), (g.name, delta, lb)


@pytest.mark.parametrize("lb", ["VERTEX_BASED", "WM", "CM", "ETWC"])
def test_sssp_fused(g2, rmat14, grid, lb, monkeypatch):
    """The grid-wide persistent near/far loop (the one-cluster loop off)."""
    monkeypatch.setenv("G2_FUSED_CLUSTER", "0")
    for g, wmax in ((rmat14, 255), (grid, 1000)):
        w = gg.pair_weights(g, wmax, seed=2)
        src = 5
        want = oracle.sssp_graph(g, w, src)
        dg = g2.load_graph(g, w)
        for delta in (1, 100, 4096):
            dist = dev(g.n)
            g2.g2_sssp_delta(dg, src, delta, dist, g2.schedule(lb, kernel_fusion=True))
            assert np.array_equal(host(dist), want), (g.name, lb, delta)
            assert g2.g2_last_stats()["launches"] == 1


@pytest.mark.parametrize("hi,far_lo", [(None, None), (64, 64), (64, 1), (1, 1)])
def test_sssp_in_one_cluster(g2, rmat14, grid, monkeypatch, hi, far_lo):
    """Fused WM delta-stepping starts in one thread-block cluster (near lists
    and far piles in shared memory) and moves to the grid-wide loop before a
    near round of more than `hi` vertices, back at a bucket boundary whose
    pile holds at most `far_lo` entries.  A near list that outgrows a CTA's
    buffer (a star's 30,000 leaves) is rebuilt from the distances.  Every
    combination gives the oracle's distances."""
    monkeypatch.delenv("G2_FUSED_CLUSTER", raising=False)
    if hi is None:
        monkeypatch.delenv("G2_CLUSTER_HI", raising=False)
        monkeypatch.delenv("G2_CLUSTER_FAR_LO", raising=False)
    else:
        monkeypatch.setenv("G2_CLUSTER_HI", str(hi))
        monkeypatch.setenv("G2_CLUSTER_FAR_LO", str(far_lo))
    star = gg.star(30001)
    graphs = [(grid, 1000), (rmat14, 255), (gg.road_grid(300, seed=4), 1000), (star, 50),
              (gg.path(3000), 20)]
    for g, wmax in graphs:
        w = gg.pair_weights(g, wmax, seed=3)
        dg = g2.load_graph(g, w)
        for src in (0, g.n - 1):
            want = oracle.sssp_graph(g, w, src)
            for delta in (1, 100, 4096, 1 << 30):
                dist = dev(g.n)
                g2.g2_sssp_delta(dg, src, delta, dist, g2.schedule("WM", kernel_fusion=True))
                assert np.array_equal(host(dist), want), (g.name, src, delta)
                st = g2.g2_last_stats()
                if g is star:
                    assert st["launches"] >= 3, (src, delta, st)  # cluster, rebuild, grid
                elif hi is None and g.n <= 16384:
                    assert st["launches"] == 1, (g.name, src, delta, st)  # all in the cluster


def test_sssp_dedup_variants_and_edge_cases(g2, rmat14):
    w = gg.pair_weights(rmat14, 255, seed=3)
    want = oracle.sssp_graph(rmat14, w, 7)
    dg = g2.load_graph(rmat14, w)
    for s in (g2.schedule("ETWC", dedup_type=g2.G2_DEDUP_BITMAP),
              g2.schedule("WM", dedup_type=g2.G2_DEDUP_BOOLMAP),
              g2.schedule("CM", dedup=False)):
        dist = dev(rmat14.n)
        g2.g2_sssp_delta(dg, 7, 50, dist, s)
        assert np.array_equal(host(dist), want)
    for g in edge_cases():
        w = gg.pair_weights(g, 9, seed=1) if g.symmetric else \
            (np.arange(g.m, dtype=np.int32) % 7 + 1).astype(np.int32)
        want = oracle.sssp_graph(g, w, 0)
        dg = g2.load_graph(g, w)
        for s in (g2.schedule("TWC"), g2.schedule("VERTEX_BASED", kernel_fusion=True)):
            dist = dev(g.n)
            g2.g2_sssp_delta(dg, 0, 3, dist, s)
            assert np.array_equal(host(dist), want), g.name


# ------------------------------------------------------------------ PageRank
def pr_scheds(g2):
    out = [("default", None),
           ("pull-edge-only", g2.schedule("EDGE_ONLY", direction=g2.G2_PULL))]
    out += [(f"pull-{lb}", g2.schedule(lb, direction=g2.G2_PULL)) for lb in ("VERTEX_BASED", "WM", "CM")]
    out += [(f"push-{lb}", g2.schedule(lb)) for lb in LBS + ["EDGE_ONLY"]]
    out.append(("push-edge-only-blocked", g2.schedule("EDGE_ONLY", edge_blocking=True, blocking_size=1000)))
    return out


def test_pagerank(g2, rmat14, grid):
    for g in (rmat14, grid, gg.gnp(300, 0.02, 9, symmetric=False), gg.from_arcs(5, [], [])):
        ref = oracle.pagerank_graph(g, 0.85, 20)
        dg = g2.load_graph(g)
        for name, s in pr_scheds(g2):
            rank = dev(g.n, torch.float32)
            g2.g2_pagerank(dg, 0.85, 20, rank, s)
            x = host(rank).astype(np.float64)
            l1 = np.abs(x - ref).sum()
            assert l1 <= PR_L1, (g.name, name, l1)


@pytest.mark.parametrize("kernel,ipt,cta", [("merge", "8", "1024"), ("merge", "16", "1024"),
                                            ("seg", "8", "512"), ("seg", "8", "1024")])
@pytest.mark.parametrize("hot", ["0", "4", "1024", "100000"])
def test_pagerank_tile_configs(g2, rmat14, grid, monkeypatch, kernel, ipt, cta, hot):
    """The arc-balanced round kernels under every tuning knob: merge-path
    tiles (items per thread, one resident CTA per SM) or the segmented warp
    sweep (CTA size), each with and without the shared-memory share cache
    (renumbered columns)."""
    monkeypatch.setenv("G2_PR_KERNEL", kernel)
    monkeypatch.setenv("G2_PR_IPT", ipt)
    monkeypatch.setenv("G2_PR_SEG_CTA", cta)
    monkeypatch.setenv("G2_PR_HOT", hot)
    monkeypatch.setenv("G2_PR_CTAS_PER_SM", "1")
    for g in (rmat14, grid, gg.gnp(300, 0.02, 9, symmetric=False)):
        ref = oracle.pagerank_graph(g, 0.85, 20)
        rank = dev(g.n, torch.float32)
        g2.g2_pagerank(g2.load_graph(g), 0.85, 20, rank)
        assert np.abs(host(rank).astype(np.float64) - ref).sum() <= PR_L1, (g.name, ipt, hot)


@pytest.mark.parametrize("S", ["256", "1024", "4096", "12288", "49152"])
def test_pagerank_source_blocked(g2, rmat14, grid, monkeypatch, S):
    """The source-blocked sweep (EdgeBlocking by source block, shares staged
    in shared memory) at block sizes from 256 sources (64 blocks on RMAT-14,
    so runs cross chunk and block boundaries and most blocks carry padding)
    to the largest; directed and degenerate graphs included."""
    monkeypatch.setenv("G2_PR_KERNEL", "blk")
    monkeypatch.setenv("G2_PR_BLK_S", S)
    graphs = [rmat14, grid, gg.gnp(300, 0.02, 9, symmetric=False), gg.star(3000), gg.path(1000),
              gg.from_arcs(5, [], []), gg.from_arcs(1, [], []),
              gg.disjoint_union(gg.complete(30), gg.star(700), gg.from_arcs(3, [], []))]
    for g in graphs:
        ref = oracle.pagerank_graph(g, 0.85, 20)
        dg = g2.load_graph(g)
        for iters in (20, 0, 1):
            want = ref if iters == 20 else oracle.pagerank_graph(g, 0.85, iters)
            rank = dev(g.n, torch.float32)
            g2.g2_pagerank(dg, 0.85, iters, rank)
            l1 = np.abs(host(rank).astype(np.float64) - want).sum()
            assert l1 <= PR_L1, (g.name, S, iters, l1)


def test_pagerank_iteration_counts(g2, rmat14):
    dg = g2.load_graph(rmat14)
    for iters in (0, 1, 2, 7):
        ref = oracle.pagerank_graph(rmat14, 0.85, iters)
        rank = dev(rmat14.n, torch.float32)
        g2.g2_pagerank(dg, 0.85, iters, rank)
        assert np.abs(host(rank) - ref).sum() <= PR_L1


# ------------------------------------------------------------------------ BC
def bc_close(got, want):
    tol = BC_REL * np.abs(want) + BC_ABS * max(np.abs(want).max(), 1.0)
    return np.all(np.abs(got - want) <= tol)


def test_bc(g2, rmat14):
    g = gg.rmat(12, seed=2)
    srcs = gg.random_sources(g, 4, seed=3)
    want = oracle.bc_graph(g, srcs)
    dg = g2.load_graph(g)
    for s in (None, g2.schedule("ETWC"), g2.schedule("VERTEX_BASED"),
              g2.hybrid(g2.schedule("WM"), pull_sched(g2, "VERTEX_BASED", g2.G2_BITMAP, g2.G2_FUSED), 0.05),
              g2.schedule("VERTEX_BASED", kernel_fusion=True), g2.schedule("WM", kernel_fusion=True),
              g2.schedule("CM", kernel_fusion=True), g2.schedule("ETWC", kernel_fusion=True)):
        bc = dev(g.n, torch.float64)
        g2.g2_bc(dg, srcs, bc, s)
        assert bc_close(host(bc), want)
    for g in edge_cases()[:9]:
        srcs = np.arange(g.n, dtype=np.int32)[:50]
        want = oracle.bc_graph(g, srcs)
        bc = dev(g.n, torch.float64)
        g2.g2_bc(g2.load_graph(g), srcs, bc, g2.schedule("CM"))
        assert bc_close(host(bc), want), g.name


def test_bc_level_spread_beyond_fp64(g2):
    """Full 1200 x 1200 grid from a corner: on level k the path counts run
    from 1 (the border) to about C(k, k/2), more than 2^1074 apart near k = 1199,
    so no common scale per level keeps all of them in fp64; per-vertex
    exponents do.  Plain and fused against the long double oracle."""
    g = gg.full_grid(1200, 1200)
    want = oracle.bc_graph(g, [0])
    dg = g2.load_graph(g)
    for s in (None, g2.schedule("WM", kernel_fusion=True)):
        bc = dev(g.n, torch.float64)
        g2.g2_bc(dg, [0], bc, s)
        got = host(bc)
        assert np.all(np.isfinite(got))
        assert bc_close(got, want)


@pytest.mark.parametrize("cluster", ["default", "0", "64,32", "1,1"])
def test_bc_fused_in_one_cluster(g2, grid, monkeypatch, cluster):
    """Fused WM BC on symmetric bounded-degree graphs: the forward pass runs
    small levels inside one thread-block cluster and large ones in the
    grid-wide kernel, handing over at level boundaries (thresholds hi,lo
    forced low to make many hand-overs); the backward pass runs ranges of
    small / large levels on one or the other.  With the cluster switched off,
    the grid-wide kernel alone (init + one launch per source).  A 31-ary tree,
    whose last level (923,521 leaves) outgrows a CTA's buffer, rebuilds that
    level's list from the depths.  Sums over several sources against the long
    double oracle."""
    if cluster == "0":
        monkeypatch.setenv("G2_FUSED_CLUSTER", "0")
    else:
        monkeypatch.delenv("G2_FUSED_CLUSTER", raising=False)
    if "," in cluster:
        hi, lo = cluster.split(",")
        monkeypatch.setenv("G2_CLUSTER_BC_HI", hi)
        monkeypatch.setenv("G2_CLUSTER_BC_LO", lo)
    else:
        monkeypatch.delenv("G2_CLUSTER_BC_HI", raising=False)
        monkeypatch.delenv("G2_CLUSTER_BC_LO", raising=False)
    kids = np.arange(1, 1 + 31 + 961 + 29791 + 923521)
    tree = gg.from_arcs(len(kids) + 1, (kids - 1) // 31, kids, name="tree31")
    cases = [(grid, gg.random_sources(grid, 6, seed=7)), (gg.road_grid(300, seed=4), [0, 89999, 45150]),
             (gg.path(4000), [0, 3999, 1234]), (gg.full_grid(200, 200), [0, 20100]), (tree, [0, 5])]
    for g, srcs in cases:
        srcs = np.asarray(srcs, dtype=np.int32)
        want = oracle.bc_graph(g, srcs)
        dg = g2.load_graph(g)
        bc = dev(g.n, torch.float64)
        g2.g2_bc(dg, srcs, bc, g2.schedule("WM", kernel_fusion=True))
        assert bc_close(host(bc), want), g.name
        st = g2.g2_last_stats()
        if cluster == "0":
            assert st["launches"] == 2 * len(srcs), (g.name, st)
        elif cluster == "default" and g is not tree:
            # every level fits: init, forward and (with two or more levels)
            # backward in the cluster
            want_l = sum(3 if oracle.bfs_graph(g, int(x))[0].max() >= 1 else 2 for x in srcs)
            assert st["launches"] == want_l, (g.name, st)


def test_bc_path_counts_beyond_fp64(g2):
    """Full 600x600 grid from a corner: path counts reach C(1198, 599) ~ 1e359,
    past fp64; per-level power-of-two rescaling keeps the result exact to
    rounding (the oracle counts in long double)."""
    g = gg.full_grid(600, 600)
    want = oracle.bc_graph(g, [0])
    bc = dev(g.n, torch.float64)
    g2.g2_bc(g2.load_graph(g), [0], bc, g2.schedule("WM"))
    got = host(bc)
    assert np.all(np.isfinite(got))
    assert bc_close(got, want)


# ----------------------------------------------------------- edgeset.apply
def test_apply_pr_add_covers_each_arc_once(g2, rmat14):
    """acc[v] = sum over in-arcs of contrib[u]: every load-balancing strategy
    must visit each arc of the input vertexset exactly once."""
    g = rmat14
    rng = np.random.default_rng(0)
    contrib = rng.integers(1, 64, g.n).astype(np.float32)  # small integers: exact float sums
    active = np.sort(rng.choice(g.n, 3000, replace=False)).astype(np.int32)
    src = np.repeat(np.arange(g.n), g.degrees())
    mask = np.isin(src, active)
    want = np.bincount(g.col[mask], weights=contrib[src[mask]], minlength=g.n)
    want_all = np.bincount(g.col, weights=contrib[src], minlength=g.n)
    dg = g2.load_graph(g)
    fin = g2.Frontier(dg, g2.G2_FRONTIER_SPARSE)
    fin.set(active)
    c = torch.from_numpy(contrib).cuda()
    for lb in LBS + ["EDGE_ONLY"]:
        acc = torch.zeros(g.n, dtype=torch.float32, device="cuda")
        if lb == "EDGE_ONLY":
            g2.g2_edgeset_apply(dg, g2.G2_OP_PR_ADD, None, c, acc, g2.schedule(lb))
            assert np.array_equal(host(acc), want_all.astype(np.float32)), lb
            continue
        g2.g2_edgeset_apply(dg, g2.G2_OP_PR_ADD, fin, c, acc, g2.schedule(lb))
        assert np.array_equal(host(acc), want.astype(np.float32)), lb
    for lb in ("VERTEX_BASED", "WM", "CM"):
        for rep in (g2.G2_FRONTIER_BITMAP, g2.G2_FRONTIER_BOOLMAP):
            f2 = g2.Frontier(dg, rep)
            f2.set(active)
            acc = torch.zeros(g.n, dtype=torch.float32, device="cuda")
            g2.g2_edgeset_apply(dg, g2.G2_OP_PR_ADD, f2, c, acc, g2.schedule(lb, direction=g2.G2_PULL))
            assert np.array_equal(host(acc), want.astype(np.float32)), ("pull", lb, rep)


def _brandes_by_levels(g2, g, src, sched_sigma, sched_delta, fmt):
    """Single-source BC through the operator alone: path counts by
    G2_OP_BC_SIGMA from the source's level down, then dependencies by
    G2_OP_BC_DELTA from the deepest level up (depths from the oracle's BFS)."""
    depth, _ = oracle.bfs_graph(g, src, want_parent=False)
    dg = g2.load_graph(g)
    d = torch.from_numpy(depth.astype(np.int32)).cuda()
    sd = torch.zeros(2 * g.n, dtype=torch.float64, device="cuda")  # sigma, then delta
    sd[src] = 1.0
    levels = [np.nonzero(depth == k)[0].astype(np.int32) for k in range(int(depth.max()) + 1)]
    for lv in levels[:-1]:
        f = g2.Frontier(dg, fmt)
        f.set(lv)
        g2.g2_edgeset_apply(dg, g2.G2_OP_BC_SIGMA, f, d, sd[: g.n], sched_sigma)
    for lv in reversed(levels[1:]):
        f = g2.Frontier(dg, fmt)
        f.set(lv)
        g2.g2_edgeset_apply(dg, g2.G2_OP_BC_DELTA, f, d, sd, sched_delta)
    delta = host(sd)[g.n:].copy()
    delta[src] = 0.0  # delta_s(s) is excluded from BC
    return delta


def test_apply_bc_delta_gives_brandes_dependencies(g2, rmat14, grid):
    """G2_OP_BC_DELTA, Brandes' backward step of one level: run level by level
    after G2_OP_BC_SIGMA's forward path counts, the dependencies of every
    vertex equal the oracle's single-source BC, PUSH (every frontier load
    balancing) and PULL (bitmap and boolmap input)."""
    g12 = gg.rmat(12, seed=3)
    cases = [(g12, g12.max_degree_vertex()), (grid, 0), (rmat14, 5), (gg.star(200), 7), (gg.path(50), 0)]
    for g, src in cases:
        want = oracle.bc_graph(g, np.array([src], np.int32))
        scheds = [(g2.schedule(lb), g2.schedule(lb), g2.G2_FRONTIER_SPARSE) for lb in LBS]
        scheds += [(pull_sched(g2, lb, rep), pull_sched(g2, lb, rep), fmt)
                   for lb in ("VERTEX_BASED", "WM", "CM")
                   for rep, fmt in ((g2.G2_BITMAP, g2.G2_FRONTIER_BITMAP),
                                    (g2.G2_BOOLMAP, g2.G2_FRONTIER_BOOLMAP))]
        for s_sigma, s_delta, fmt in scheds:
            got = _brandes_by_levels(g2, g, src, s_sigma, s_delta, fmt)
            assert bc_close(got, want), (g.name, src, s_delta.load_balance, s_delta.direction)
    # a directed graph is rejected before any launch
    gd = gg.gnp(50, 0.1, 2, symmetric=False)
    dg = g2.load_graph(gd)
    f = g2.Frontier(dg, g2.G2_FRONTIER_SPARSE)
    f.set(np.array([0], np.int32))
    with pytest.raises(Exception):
        g2.g2_edgeset_apply(dg, g2.G2_OP_BC_DELTA, f, dev(gd.n), torch.zeros(2 * gd.n, dtype=torch.float64,
                                                                              device="cuda"))


def test_apply_bfs_round_and_frontier_formats(g2, rmat14):
    """One applyModified round of the Fig. 2 program from a frontier: the
    output vertexset is exactly the unvisited out-neighbours."""
    g = rmat14
    rng = np.random.default_rng(1)
    depth0 = np.full(g.n, -1, np.int32)
    front = np.sort(rng.choice(g.n, 500, replace=False)).astype(np.int32)
    depth0[front] = 3
    visited = rng.choice(g.n, 2000, replace=False)
    depth0[visited] = np.where(depth0[visited] == -1, 2, depth0[visited])
    src = np.repeat(np.arange(g.n), g.degrees())
    hit = np.isin(src, front) & (depth0[g.col] == -1)
    want_out = np.unique(g.col[hit])
    want_depth = depth0.copy()
    want_depth[want_out] = 4
    dg = g2.load_graph(g)
    for fmt_in, fmt_out, s in itertools.product(
            (g2.G2_FRONTIER_SPARSE, g2.G2_FRONTIER_BITMAP, g2.G2_FRONTIER_BOOLMAP),
            (g2.G2_FRONTIER_SPARSE, g2.G2_FRONTIER_BITMAP, g2.G2_FRONTIER_BOOLMAP),
            (g2.schedule("ETWC"), g2.schedule("TWC", frontier_creation=g2.G2_UNFUSED_BOOLMAP),
             pull_sched(g2, "WM", g2.G2_BOOLMAP, g2.G2_FUSED))):
        fin = g2.Frontier(dg, fmt_in)
        fin.set(front)
        fout = g2.Frontier(dg, fmt_out)
        d = torch.from_numpy(depth0).cuda()
        k = g2.g2_edgeset_apply(dg, g2.G2_OP_BFS, fin, d, None, s, fout)
        assert k == want_out.size
        assert np.array_equal(host(d), want_depth)
        lst = dev(g.n)
        kk = fout.to_list(lst)
        assert kk == k and np.array_equal(np.sort(host(lst)[:kk]), want_out)


def test_apply_label_min_round_invariants(g2, rmat14):
    """One LABEL_MIN round over all vertices.  Updates are in place (a source
    may already carry a value lowered earlier in the same round), so the
    round's result is bracketed: at or below one synchronous round from the
    initial labels, at or above the fixpoint, and the output vertexset is
    exactly the set of lowered labels."""
    g = rmat14
    rng = np.random.default_rng(2)
    lab0 = rng.permutation(g.n).astype(np.int32)
    src = np.repeat(np.arange(g.n), g.degrees())
    one = lab0.copy()
    np.minimum.at(one, g.col, lab0[src])
    fix = one.copy()
    while True:
        nxt = fix.copy()
        np.minimum.at(nxt, g.col, fix[src])
        if np.array_equal(nxt, fix):
            break
        fix = nxt
    dg = g2.load_graph(g, gg.pair_weights(g, 100))
    for s in (g2.schedule("WM"), g2.schedule("STRICT", dedup_type=g2.G2_DEDUP_BITMAP),
              g2.schedule("EDGE_ONLY"), pull_sched(g2, "CM", g2.G2_BOOLMAP, g2.G2_FUSED)):
        lab = torch.from_numpy(lab0).cuda()
        fout = g2.Frontier(dg, g2.G2_FRONTIER_SPARSE)
        k = g2.g2_edgeset_apply(dg, g2.G2_OP_LABEL_MIN, None, lab, None, s, fout)
        got = host(lab)
        assert np.all(got <= one) and np.all(got >= fix)
        changed = np.nonzero(got < lab0)[0]
        lst = dev(g.n)
        assert fout.to_list(lst) == k == changed.size
        assert np.array_equal(np.sort(host(lst)[:k]), changed)


# ---------------------------------------------------------------- EdgeBlocking
@pytest.mark.parametrize("N", [1, 5, 1000, 16384])
def test_edge_blocking_matches_algorithm1(g2, rmat14, N):
    g = rmat14
    src = np.repeat(np.arange(g.n, dtype=np.int32), g.degrees())
    osrc, odst, oseg, ns = oracle.edgeblock(g.n, src, g.col, N)
    dg = g2.load_graph(g)
    assert g2.g2_edge_block(dg, N) == ns
    s = dev(g.m)
    d = dev(g.m)
    seg = dev(ns + 1, torch.int64)
    g2.g2_edge_block_export(dg, s, d, seg)
    assert np.array_equal(host(s), osrc) and np.array_equal(host(d), odst)
    assert np.array_equal(host(seg), oseg)


# ------------------------------------------------------------------- batched
def test_bfs_batch(g2):
    g = gg.rmat(13, seed=4)
    srcs = gg.random_sources(g, 64, seed=1)
    dg = g2.load_graph(g)
    want = np.stack([oracle.bfs_graph(g, s, want_parent=False)[0] for s in srcs])
    for s in (None, g2.schedule("ETWC"), g2.schedule("WM"),
              g2.hybrid(g2.schedule("CM"), g2.schedule("WM", direction=g2.G2_PULL), 0.05),
              g2.schedule("VERTEX_BASED", direction=g2.G2_PULL),
              g2.schedule("WM", kernel_fusion=True)):
        for k in (1, 17, 64):
            depth = dev(k * g.n)
            g2.g2_bfs_batch(dg, srcs[:k], depth, s)
            assert np.array_equal(host(depth).reshape(k, g.n), want[:k]), k


def test_bfs_batch_fused_on_a_road_grid(g2, grid, monkeypatch):
    """Bounded-degree graph, with repeated sources and a ragged k.  The NULL
    schedule splits the batch into single-source fused queries on worker
    streams (k = 1 runs one); with the split switched off it, like the
    explicit fused schedule, runs the fused multi-source loop in one launch."""
    srcs = np.concatenate([gg.random_sources(grid, 40, seed=3), [7, 7, 0]]).astype(np.int32)
    want = np.stack([oracle.bfs_graph(grid, s, want_parent=False)[0] for s in srcs])
    dg = g2.load_graph(grid)
    for k in (len(srcs), 2, 1):
        depth = dev(k * grid.n)
        g2.g2_bfs_batch(dg, srcs[:k], depth, None)
        assert np.array_equal(host(depth).reshape(k, grid.n), want[:k]), k
    monkeypatch.setenv("G2_BATCH_SPLIT_WORKERS", "0")
    for s in (None, g2.schedule("WM", kernel_fusion=True)):
        depth = dev(len(srcs) * grid.n)
        g2.g2_bfs_batch(dg, srcs, depth, s)
        assert np.array_equal(host(depth).reshape(len(srcs), grid.n), want)
        st = g2.g2_last_stats()
        assert st["iterations"] == want.max() + 1 and st["launches"] == 2
    with pytest.raises(g2.G2Error) as e:
        g2.g2_bfs_batch(dg, srcs[:4], dev(4 * grid.n), g2.schedule("CM", kernel_fusion=True))
    assert e.value.status == g2.G2_EUNSUPPORTED


def test_sssp_batch(g2):
    g = gg.rmat(12, seed=5)
    w = gg.pair_weights(g, 255, seed=5)
    srcs = gg.random_sources(g, 32, seed=2)
    want = np.stack([oracle.sssp_graph(g, w, s) for s in srcs])
    dg = g2.load_graph(g, w)
    for delta in (0, 1, 40, 1000):
        for sch in [g2.schedule(lb) for lb in ("VERTEX_BASED", "WM", "CM", "ETWC")] + \
                   [g2.schedule("WM", kernel_fusion=True)]:
            for k in (1, 32):
                dist = dev(k * g.n)
                g2.g2_sssp_batch(dg, srcs[:k], delta, dist, sch)
                assert np.array_equal(host(dist).reshape(k, g.n), want[:k]), (delta, k)


def test_sssp_batch_fused_on_a_road_grid(g2, grid, monkeypatch):
    """Bounded-degree graph, every delta, with repeated sources and a ragged
    k.  The NULL schedule splits the batch into single-source fused queries on
    worker streams; with the split switched off it runs the fused multi-source
    near/far loop (one launch after seeding)."""
    w = gg.pair_weights(grid, 1000, seed=4)
    srcs = np.concatenate([gg.random_sources(grid, 27, seed=4), [9, 9]]).astype(np.int32)
    want = np.stack([oracle.sssp_graph(grid, w, s) for s in srcs])
    dg = g2.load_graph(grid, w)
    for split in ("", "0"):
        if split:
            monkeypatch.setenv("G2_BATCH_SPLIT_WORKERS", split)
        for delta in (0, 1, 300, 5000, 1 << 30):
            dist = dev(len(srcs) * grid.n)
            g2.g2_sssp_batch(dg, srcs, delta, dist, None)
            assert np.array_equal(host(dist).reshape(len(srcs), grid.n), want), (delta, split)
            if split:
                assert g2.g2_last_stats()["launches"] == 3
    with pytest.raises(g2.G2Error) as e:
        g2.g2_sssp_batch(dg, srcs[:3], 64, dev(3 * grid.n), g2.schedule("ETWC", kernel_fusion=True))
    assert e.value.status == g2.G2_EUNSUPPORTED


# ------------------------------------------------------------- errors, views
def test_argument_errors(g2, rmat14):
    dg = g2.load_graph(rmat14)
    d = dev(rmat14.n)
    with pytest.raises(g2.G2Error) as e:
        g2.g2_bfs(dg, rmat14.n, d)
    assert e.value.status == g2.G2_EINVAL
    with pytest.raises(g2.G2Error) as e:
        g2.g2_sssp_delta(dg, 0, 1, d)  # no weights
    assert e.value.status == g2.G2_EINVAL
    with pytest.raises(g2.G2Error) as e:
        g2.g2_bfs(dg, 0, d, None, g2.schedule("EDGE_ONLY"))
    assert e.value.status == g2.G2_EUNSUPPORTED
    with pytest.raises(g2.G2Error) as e:  # unsorted adjacency list
        g2.g2_load_csr(3, np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32))
    assert e.value.status == g2.G2_EINVAL
    with pytest.raises(g2.G2Error) as e:  # id out of range
        g2.g2_load_csr(2, np.array([0, 1, 2], np.int32), np.array([1, 5], np.int32))
    assert e.value.status == g2.G2_EINVAL


def test_bounded_wait_times_out(g2):
    """The bounded device-side wait used by grid barriers gives up after its
    limit on a flag nothing sets, records G2_ETIMEOUT and returns; the context
    stays usable afterwards."""
    assert g2.g2_selftest_wait_timeout(2_000_000) == g2.G2_ETIMEOUT
    x = torch.arange(10, device="cuda").sum().item()
    assert x == 45


def test_views_on_threads_build_shared_layouts_once(g2, rmat14):
    """Views on four threads, each with its own stream, all ask at once for
    the lazily built layouts of one fresh topology (PageRank's renumbering
    and segment flags, the degree statistic)."""
    import threading
    g = rmat14
    ref = oracle.pagerank_graph(g, 0.85, 20)
    od = oracle.bfs_graph(g, 0)[0]
    base = g2.load_graph(g)
    views = [base.view() for _ in range(4)]
    errors, outs = [], {}

    def work(i):
        try:
            with torch.cuda.stream(torch.cuda.Stream()):
                r = torch.empty(g.n, dtype=torch.float32, device="cuda")
                d = torch.empty(g.n, dtype=torch.int32, device="cuda")
                s = torch.cuda.current_stream().cuda_stream
                g2.g2_pagerank(views[i], 0.85, 20, r, None, s)
                g2.g2_bfs(views[i], 0, d, None, None, s)
                torch.cuda.current_stream().synchronize()
                outs[i] = (r.cpu().numpy().astype(np.float64), d.cpu().numpy())
        except Exception as e:  # reported below
            errors.append(e)

    ts = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
    for i in range(4):
        assert np.abs(outs[i][0] - ref).sum() <= PR_L1
        assert np.array_equal(outs[i][1], od)


def test_views_and_device_pointer_load(g2, rmat14):
    g = rmat14
    rp = torch.from_numpy(g.rowptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    dg = g2.g2_load_csr(g.n, rp, cl, None, True)
    v = dg.view()
    od, op = oracle.bfs_graph(g, 9)
    for h in (dg, v):
        d = dev(g.n)
        p = dev(g.n)
        g2.g2_bfs(h, 9, d, p, g2.schedule("ETWC"))
        assert np.array_equal(host(d), od) and np.array_equal(host(p), op)
    info = dg.info()
    assert info["n"] == g.n and info["m"] == g.m and info["sm_count"] > 0


def test_load_paths_and_memory_reuse(g2, rmat14):
    """Every way of handing the CSR to g2_load_csr gives the same graph: pinned
    host arrays and pageable ones (read by the validating copy kernel where the
    device can address them), a misaligned host view (plain copy, then
    validation), device arrays; invalid input is rejected on each path; and
    graphs loaded and freed many times over reuse pooled memory correctly."""
    g = rmat14
    w = gg.pair_weights(g, 255, seed=3)
    od, op = oracle.bfs_graph(g, 5)
    osd = oracle.sssp_graph(g, w, 5)

    def check(dg):
        d, p, s = dev(g.n), dev(g.n), dev(g.n)
        g2.g2_bfs(dg, 5, d, p, None)
        g2.g2_sssp_delta(dg, 5, 64, s, None)
        assert np.array_equal(host(d), od) and np.array_equal(host(p), op)
        assert np.array_equal(host(s), osd)
        dg.free()

    # pageable numpy arrays
    check(g2.load_graph(g, w))
    # pinned host memory
    prp = torch.from_numpy(g.rowptr).pin_memory()
    pcl = torch.from_numpy(g.col).pin_memory()
    pw = torch.from_numpy(w).pin_memory()
    as_np = lambda t: np.frombuffer(t.numpy().data, dtype=np.int32)
    check(g2.g2_load_csr(g.n, as_np(prp), as_np(pcl), as_np(pw), True))
    # the same through the copy engines (a load that overlaps other work)
    check(g2.g2_load_csr(g.n, as_np(prp), as_np(pcl), as_np(pw), True, overlap=True))
    # an overlapping load of pageable arrays: the copy kernel on a quarter of
    # the SMs (16-byte aligned numpy arrays)
    assert g.col.ctypes.data % 16 == 0 and w.ctypes.data % 16 == 0
    check(g2.g2_load_csr(g.n, g.rowptr, g.col, w, True, overlap=True))
    # 4-byte misaligned host views of the same data
    buf = np.empty(g.m + 1, np.int32)
    col_mis = buf[1:]
    col_mis[:] = g.col
    wbuf = np.empty(g.m + 1, np.int32)
    w_mis = wbuf[1:]
    w_mis[:] = w
    assert col_mis.ctypes.data % 16 != 0
    check(g2.g2_load_csr(g.n, g.rowptr, col_mis, w_mis, True))
    # device arrays
    check(g2.g2_load_csr(g.n, torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(),
                         torch.from_numpy(w).cuda(), True))
    # invalid input on the pinned and misaligned paths
    bad = g.col.copy()
    bad[g.m // 2 + 3] = g.n  # id out of range
    for c in (as_np(torch.from_numpy(bad).pin_memory()), np.concatenate([np.zeros(1, np.int32), bad])[1:],
              bad):
        for ov in (False, True):
            with pytest.raises(g2.G2Error) as e:
                g2.g2_load_csr(g.n, g.rowptr, c, None, True, overlap=ov)
            assert e.value.status == g2.G2_EINVAL
    wneg = w.copy()
    wneg[g.m - 1] = -1  # negative weight in the ragged tail
    with pytest.raises(g2.G2Error) as e:
        g2.g2_load_csr(g.n, g.rowptr, g.col, wneg, True)
    assert e.value.status == g2.G2_EINVAL
    # swapped neighbours inside one adjacency list (the swap crosses a 4-arc quad)
    uns = g.col.copy()
    v = next(u for u in range(g.n) if g.rowptr[u + 1] - g.rowptr[u] >= 8 and g.rowptr[u] % 4 == 1)
    b = int(g.rowptr[v]) + 2
    uns[b], uns[b + 1] = uns[b + 1], uns[b]
    with pytest.raises(g2.G2Error) as e:
        g2.g2_load_csr(g.n, g.rowptr, uns, None, True)
    assert e.value.status == g2.G2_EINVAL
    # load / run / free repeatedly: pooled blocks are handed out again
    for _ in range(12):
        dg = g2.load_graph(g)
        d = dev(g.n)
        g2.g2_bfs(dg, 5, d, None, None)
        assert np.array_equal(host(d), od)
        r = torch.empty(g.n, dtype=torch.float32, device="cuda")
        g2.g2_pagerank(dg, 0.85, 3, r)
        dg.free()


def test_diag_gather_sums_and_rejects_bad_indices(g2):
    """The diagnostic gather pass adds up x[idx[e]] exactly once per element
    (mode 0) or the indices themselves (mode 1); indices outside [0, n) are
    refused without being loaded."""
    rng = np.random.default_rng(3)
    n, m, grid = 5000, 123457, 7
    idx = rng.integers(0, n, m, dtype=np.int32)
    x = rng.random(n).astype(np.float32)
    out = torch.empty(grid * 256, device="cuda")
    di, dx = torch.from_numpy(idx).cuda(), torch.from_numpy(x).cuda()
    ms = g2.g2_diag_gather(di, dx, 0, out, grid)
    assert ms > 0
    assert abs(host(out).astype(np.float64).sum() - x[idx].astype(np.float64).sum()) < 1e-2
    g2.g2_diag_gather(di, None, 1, out, grid)
    assert abs(host(out).astype(np.float64).sum() - idx.astype(np.float64).sum()) < 1e-4 * idx.sum()
    bad = idx.copy()
    bad[777] = n
    with pytest.raises(g2.G2Error) as e:
        g2.g2_diag_gather(torch.from_numpy(bad).cuda(), dx, 0, out, grid)
    assert e.value.status == g2.G2_EINVAL


def test_pipelined_overlapped_loads(g2, rmat14):
    """A stream of requests served the way bench.py's end-to-end line is: a
    loader thread uploads graph k+1 (pinned host arrays with weights,
    G2_LOAD_OVERLAP, its own stream, PageRank preparation in the background)
    while BFS, CC, PageRank and SSSP of graph k run on the caller's stream.  Every graph gives the
    oracle's results; two different graphs alternate so that a mix-up of the
    resident graphs would show."""
    from concurrent.futures import ThreadPoolExecutor
    ga, gb = rmat14, gg.road_grid(160, seed=9)
    want, pinned = {}, {}
    for g in (ga, gb):
        w = gg.pair_weights(g, 255, seed=11)
        want[g.name] = (oracle.bfs_graph(g, 3)[0], oracle.cc_graph(g), oracle.pagerank_graph(g, 0.85, 20),
                        oracle.sssp_graph(g, w, 3))
        rp = torch.from_numpy(g.rowptr).pin_memory()
        cl = torch.from_numpy(g.col).pin_memory()
        pw = torch.from_numpy(w).pin_memory()
        as_np = lambda t: np.frombuffer(t.numpy().data, dtype=np.int32)
        pinned[g.name] = (rp, cl, pw, as_np(rp), as_np(cl), as_np(pw))
    side = torch.cuda.Stream()

    def load(g):
        _, _, _, rp, cl, w = pinned[g.name]
        return g2.g2_load_csr(g.n, rp, cl, w, True, stream=side, prepare_pagerank=True,
                              overlap=True), g

    order = [ga, gb, ga, gb, gb, ga]
    with ThreadPoolExecutor(1) as ex:
        fut = ex.submit(load, order[0])
        for i in range(len(order)):
            dg, g = fut.result()
            if i + 1 < len(order):
                fut = ex.submit(load, order[i + 1])
            d, lab, r, dist = dev(g.n), dev(g.n), dev(g.n, torch.float32), dev(g.n)
            g2.g2_bfs(dg, 3, d, None, None)
            g2.g2_cc(dg, lab, None)
            g2.g2_pagerank(dg, 0.85, 20, r)
            g2.g2_sssp_delta(dg, 3, 0, dist, None)
            od, ol, opr, osd = want[g.name]
            assert np.array_equal(host(d), od) and np.array_equal(host(lab), ol), (i, g.name)
            assert np.abs(host(r).astype(np.float64) - opr).sum() <= PR_L1, (i, g.name)
            assert np.array_equal(host(dist), osd), (i, g.name)
            dg.free()


def test_background_pagerank_preparation(g2, rmat14):
    """G2_PREPARE_PAGERANK: PageRank's layouts are built by a background thread
    on its own stream while BFS and CC run on the caller's; PageRank waits for
    them; a graph freed while the preparation still runs waits for it too."""
    g = rmat14
    ref = oracle.pagerank_graph(g, 0.85, 20)
    od = oracle.bfs_graph(g, 0)[0]
    ol = oracle.cc_graph(g)
    for _ in range(3):
        dg = g2.g2_load_csr(g.n, g.rowptr, g.col, None, True, prepare_pagerank=True)
        d, lab = dev(g.n), dev(g.n)
        g2.g2_bfs(dg, 0, d, None, None)
        g2.g2_cc(dg, lab, None)
        r = dev(g.n, torch.float32)
        g2.g2_pagerank(dg, 0.85, 20, r)
        assert np.array_equal(host(d), od) and np.array_equal(host(lab), ol)
        assert np.abs(host(r).astype(np.float64) - ref).sum() <= PR_L1
        dg.free()
    # freed at once: the free joins the preparation
    for _ in range(3):
        g2.g2_load_csr(g.n, g.rowptr, g.col, None, True, prepare_pagerank=True).free()
    # a directed graph (CSC built at load) and an empty one
    gd = gg.gnp(2000, 0.003, 5, symmetric=False)
    dg = g2.g2_load_csr(gd.n, gd.rowptr, gd.col, None, False, prepare_pagerank=True)
    r = dev(gd.n, torch.float32)
    g2.g2_pagerank(dg, 0.85, 20, r)
    assert np.abs(host(r).astype(np.float64) - oracle.pagerank_graph(gd, 0.85, 20)).sum() <= PR_L1
    g0 = gg.from_arcs(5, [], [])
    dg = g2.g2_load_csr(g0.n, g0.rowptr, g0.col, None, True, prepare_pagerank=True)
    r = dev(5, torch.float32)
    g2.g2_pagerank(dg, 0.85, 3, r)
    assert np.allclose(host(r), 0.2)



# ------------------------------------------------------------ asynchronous
@pytest.mark.parametrize("cap", [None, "1"])
def test_async_sssp_and_bfs(g2, rmat14, grid, monkeypatch, cap):
    """The asynchronous SSSP and BFS (no barrier inside a bucket; buckets of
    width delta, or one bucket for delta <= 0) against the oracle, bit-exact:
    road grids 128^2 and 300^2 from a corner and the centre, a star from a
    leaf and from the centre, RMAT-14, a path, directed G(n, p) and a graph
    with unreachable parts.  cap=1 gives the worklist room for n appends only,
    so runs that need more go through the overflow-and-retry path."""
    if cap:
        monkeypatch.setenv("G2_ASYNC_CAP", cap)
    g300 = gg.road_grid(300, seed=4)
    star = gg.star(30001)
    cases = [(grid, 0), (grid, grid.n // 2 + 64), (g300, 0), (g300, g300.n - 1), (star, 17), (star, 0),
             (rmat14, rmat14.max_degree_vertex()), (gg.path(3000), 0),
             (gg.gnp(400, 0.01, 5, symmetric=False), 3),
             (gg.disjoint_union(gg.road_grid(40, seed=2), gg.star(50)), 5)]
    for g, src in cases:
        w = gg.pair_weights(g, 1000, seed=3) if g.symmetric else \
            np.random.default_rng(7).integers(1, 1000, g.m).astype(np.int32)
        dg = g2.load_graph(g, w)
        want = oracle.sssp_graph(g, w, src)
        od, op = oracle.bfs_graph(g, src)
        for delta in (0, 1, 700, 5000):
            dist = dev(g.n)
            g2.g2_sssp_async(dg, src, delta, dist)
            assert np.array_equal(host(dist), want), (g.name, src, delta)
            st = g2.g2_last_stats()
            assert st["iterations"] >= int((want < 2**31 - 1).sum())  # each reached vertex at least once
        for delta in (0, 1, 3):
            d, p = dev(g.n), dev(g.n)
            g2.g2_bfs_async(dg, src, delta, d, p)
            assert np.array_equal(host(d), od) and np.array_equal(host(p), op), (g.name, src, delta)
            d2 = dev(g.n)
            g2.g2_bfs_async(dg, src, delta, d2)
            assert np.array_equal(host(d2), od), (g.name, src, delta)


def test_etwc_hands_large_entries_to_the_grid(g2):
    """ETWC PUSH where vertices have 4,096 arcs or more at CTA granularity:
    their CTA-stage entries go to a frontier-wide list that a second pass
    spreads over every CTA.  BFS from a hub equals the oracle, and an
    accumulate over a frontier holding several hubs visits each arc exactly
    once."""
    g = gg.disjoint_union(gg.star(9000), gg.star(20000), gg.rmat(12, seed=5), gg.complete(70))
    for src in (0, 9000, 9001, g.n - 1):
        od, op = oracle.bfs_graph(g, src)
        d, p = run_bfs(g2, g, src, g2.schedule("ETWC"))
        assert np.array_equal(d, od) and np.array_equal(p, op), src
    rng = np.random.default_rng(3)
    contrib = rng.integers(1, 64, g.n).astype(np.float32)  # small integers: exact float sums
    active = np.unique(np.concatenate([[0, 9000], rng.choice(g.n, 2000, replace=False)])).astype(np.int32)
    src = np.repeat(np.arange(g.n), g.degrees())
    mask = np.isin(src, active)
    want = np.bincount(g.col[mask], weights=contrib[src[mask]], minlength=g.n)
    dg = g2.load_graph(g)
    fin = g2.Frontier(dg, g2.G2_FRONTIER_SPARSE)
    fin.set(active)
    acc = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    g2.g2_edgeset_apply(dg, g2.G2_OP_PR_ADD, fin, torch.from_numpy(contrib).cuda(), acc, g2.schedule("ETWC"))
    assert np.array_equal(host(acc), want.astype(np.float32))
