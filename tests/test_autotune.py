"""Autotuner: search logic on CPU with synthetic cost functions; on the GPU,
tuned schedules must reproduce the oracle's results."""
import random

import numpy as np
import pytest

from paper_2012_07990_gb300 import autotune as at


def test_samples_are_valid_points():
    rng = random.Random(0)
    for algo in ("bfs", "sssp", "cc", "pr", "bc", "bfs_batch"):
        for _ in range(200):
            d = at.sample_schedule(algo, rng)
            if d.get("tuned_default"):
                continue
            for s in (d["s1"], d["s2"]):
                assert s["lb"] in at.LBS
                assert s["direction"] in (0, 1)
                if s["direction"] == 1:
                    # PageRank's PULL + EDGE_ONLY is the arc-balanced CSC sweep
                    assert s["lb"] in at.PULL_LBS or (algo == "pr" and s["lb"] == "EDGE_ONLY")
                if s["kernel_fusion"] and d["criteria"] == 1:
                    # the direction-optimising BFS hybrid fused into one launch
                    assert algo == "bfs" and d["s1"]["kernel_fusion"] and d["s2"]["kernel_fusion"]
                    assert d["s1"]["direction"] == 0 and d["s1"]["lb"] in at.FUSED_DO_PUSH_LBS
                    assert d["s2"]["direction"] == 1 and d["s2"]["lb"] == "VERTEX_BASED"
                    assert d["s2"]["pull_frontier"] == 1
                elif s["kernel_fusion"]:
                    assert s["lb"] in ("VERTEX_BASED", "WM", "CM", "ETWC") and s["direction"] == 0
                if s["edge_blocking"]:
                    assert s["lb"] == "EDGE_ONLY"
            if algo == "sssp":
                assert d["s1"]["delta"] >= 1


def test_exhaustive_space_enumerates_every_table_ii_point_once():
    """Per direction the space is the cartesian product of the Table II
    fields: 7 load balancers x EdgeBlocking (2) x frontier creation (3) x
    kernel fusion (2) x deduplication (PUSH 4: off or one of 3 types; PULL 2,
    times the 2 PULL input representations) = 336 distinct points, each with
    the direction's value."""
    for direction in (0, 1):
        pts = at.enumerate_direction(direction)
        assert len(pts) == 7 * 2 * 3 * 2 * 4 == 336
        assert len({at.key_of(p) for p in pts}) == len(pts)
        assert all(p["direction"] == direction for p in pts)
        assert {p["lb"] for p in pts} == set(at.LBS)
        assert sum(p["edge_blocking"] for p in pts) == 168
        assert sum(p["kernel_fusion"] for p in pts) == 168
    push = at.enumerate_direction(0)
    assert {(p["dedup"], p["dedup_type"]) for p in push} == {(False, 0), (True, 0), (True, 1), (True, 2)}
    pull = at.enumerate_direction(1)
    assert {(p["dedup"], p["pull_frontier"]) for p in pull} == {(a, b) for a in (False, True) for b in (0, 1)}


def test_exhaustive_search_finds_the_optimum_and_drops_rejected_points():
    """On a synthetic cost (refusing EdgeBlocking and fused PULL as the
    library does) the exhaustive search returns the true minimum over simple
    and hybrid schedules, counts every point, and reports each direction's
    best."""
    def base(s):
        if s["edge_blocking"] or (s["direction"] == 1 and s["kernel_fusion"]):
            raise RuntimeError("unsupported")
        return (5.0 + at.LBS.index(s["lb"]) + s["frontier_creation"] + (0.5 if s["dedup"] else 0.0)
                + (1.7 if s["kernel_fusion"] else 0.0))

    def cost(d):
        if d["criteria"] == 0:
            return base(d["s1"])
        return 0.6 * base(d["s1"]) + 0.3 * base(d["s2"]) + (0.0 if d["threshold"] == 0.02 else 0.1)

    res = at.exhaustive(cost, reps=1)
    assert res.per_direction[0]["ms"] == 5.0 and res.per_direction[1]["ms"] == 5.0
    assert res.best["criteria"] == 1 and res.best["threshold"] == 0.02
    assert abs(res.best_ms - 4.5) < 1e-9
    assert res.rejected >= 336  # every EdgeBlocking point of both directions, fused PULL
    # every simple point of both directions, then the hybrids of the 4
    # fastest PUSH x the 4 fastest PULL schedules (none fused here) at each
    # threshold, then the fused direction-optimising hybrid with each of its
    # PUSH load balancings at each threshold (refused here: fused PULL)
    nt = len(at.HYBRID_THRESHOLDS)
    assert res.evaluated == 2 * 336 + 4 * 4 * nt + len(at.FUSED_DO_PUSH_LBS) * nt
    assert res.rejected >= 336 + len(at.FUSED_DO_PUSH_LBS) * nt


def test_exhaustive_search_includes_the_fused_direction_optimising_hybrid():
    """Where the fused hybrid runs and is fastest (STRICT PUSH at 2% here),
    the exhaustive search returns it, with both halves fused."""
    def cost(d):
        s1, s2 = d["s1"], d["s2"]
        if s1["edge_blocking"] or s2["edge_blocking"]:
            raise RuntimeError("unsupported")
        if d["criteria"] == 1 and s1["kernel_fusion"] and s2["kernel_fusion"]:
            return 1.0 + (0.0 if s1["lb"] == "STRICT" else 0.5) + abs(d["threshold"] - 0.02)
        if s1["kernel_fusion"] != s2["kernel_fusion"] or (s1["direction"] == 1 and s1["kernel_fusion"]):
            raise RuntimeError("unsupported")
        return 3.0 + at.LBS.index(s1["lb"])

    res = at.exhaustive(cost, reps=1)
    assert res.best == at.fused_do_hybrid("STRICT", 0.02)
    assert res.best_ms == 1.0
    assert at.seeds("bfs")[0] == at.fused_do_hybrid("STRICT", 0.02)
    assert all(not (s["s1"]["kernel_fusion"] and s["criteria"] == 1) for s in at.seeds("bc"))


def test_successive_halving_finds_the_minimum_under_noise():
    rng = random.Random(3)
    cands = [{"x": i} for i in range(40)]
    true = {i: 10.0 + abs(i - 17) for i in range(40)}

    def cost(d):
        return true[d["x"]] + rng.random() * 0.5  # noise below the gap between neighbours

    res = at.successive_halving(cost, cands, eta=3)
    assert res.best == {"x": 17}
    assert res.evaluated >= 40


def test_failing_candidates_are_dropped_and_budget_respected():
    def cost(d):
        if d["x"] % 2:
            raise RuntimeError("unsupported")
        return float(d["x"])

    res = at.successive_halving(cost, [{"x": i} for i in range(1, 30)], eta=2)
    assert res.best == {"x": 2}
    assert any("error" in h for h in res.history)
    res2 = at.successive_halving(lambda d: float(d["x"]), [{"x": i} for i in range(100)],
                                 max_evals=10)
    assert res2.evaluated <= 10 and res2.best["x"] <= 9


def test_cache_roundtrip(tmp_path):
    from paper_2012_07990_gb300 import graphgen as gg
    g = gg.rmat(8)
    fp = at.graph_fingerprint(g.n, g.rowptr, g.col)
    assert fp == at.graph_fingerprint(g.n, g.rowptr.copy(), g.col.copy())
    assert fp != at.graph_fingerprint(g.n, g.rowptr, np.roll(g.col, 1))
    cache = at.TuneCache(str(tmp_path / "tune.json"))
    calls = []

    def cost(d):
        calls.append(1)
        return 1.0 if d.get("tuned_default") else 2.0

    best = at.tune_cached(cache, fp, "pr", cost, n_samples=5)
    assert best == {"tuned_default": True}
    n_calls = len(calls)
    again = at.TuneCache(str(tmp_path / "tune.json"))
    assert at.tune_cached(again, fp, "pr", cost) == best
    assert len(calls) == n_calls  # served from the cache


def test_graph_features_separate_graph_families():
    from paper_2012_07990_gb300 import graphgen as gg
    r10, r11 = gg.rmat(10, seed=1), gg.rmat(11, seed=1)
    g64, g90 = gg.road_grid(64, seed=1), gg.road_grid(90, seed=1)
    f = {k: at.graph_features(g.n, g.rowptr) for k, g in
         (("r10", r10), ("r11", r11), ("g64", g64), ("g90", g90))}
    import math
    assert math.dist(f["r10"], f["r11"]) < math.dist(f["r10"], f["g90"])
    assert math.dist(f["g64"], f["g90"]) < math.dist(f["g64"], f["r11"])
    assert all(len(v) == 6 and all(math.isfinite(x) for x in v) for v in f.values())


def test_warm_start_seeds_from_the_nearest_tuned_graph(tmp_path):
    """A synthetic cost model in which the best schedule depends on the graph
    family: tuning a power-law and a grid graph fills the cache; a new graph
    of either family gets the matching family's best schedules as warm seeds
    and, with a budget too small for random search alone, still finds its
    optimum."""
    from paper_2012_07990_gb300 import graphgen as gg
    cache = at.TuneCache(str(tmp_path / "tune.json"))

    def cost_for(family):
        def cost(d):
            s = d["s1"]
            if family == "powerlaw":
                return 1.0 if (s["lb"] == "STRICT" and d["threshold"] == 0.02) else 5.0
            return 1.0 if (s["lb"] == "WM" and s["kernel_fusion"]) else 5.0
        return cost

    graphs = {"powerlaw": (gg.rmat(10, seed=1), gg.rmat(11, seed=2)),
              "grid": (gg.road_grid(64, seed=1), gg.road_grid(80, seed=2))}
    for fam, (g, _) in graphs.items():
        fp = at.graph_fingerprint(g.n, g.rowptr, g.col)
        at.tune_cached(cache, fp, "bfs", cost_for(fam), features=at.graph_features(g.n, g.rowptr),
                       n_samples=12, seed=3)
    for fam, (_, g) in graphs.items():
        feats = at.graph_features(g.n, g.rowptr)
        warm = cache.warm_start(feats, "bfs", k=1)
        assert warm and cost_for(fam)(warm[0]) == 1.0
        # a budget of one evaluation: only the first candidate (the warm seed) is timed
        res = at.tune("bfs", cost_for(fam), n_samples=0, warm=warm, max_evals=1)
        assert res.best_ms == 1.0
    again = at.TuneCache(str(tmp_path / "tune.json"))
    assert len(again.warm_start(feats, "bfs", k=2)) >= 2


@pytest.mark.gpu
def test_tuned_schedules_reproduce_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2012_07990_gb300 import build_native
    from paper_2012_07990_gb300 import graphgen as gg
    build_native.build()
    from paper_2012_07990_gb300 import g2
    g = gg.rmat(12, seed=7)
    w = gg.pair_weights(g, 255, seed=7)
    dg = g2.load_graph(g, w)
    src = g.max_degree_vertex()
    for algo in ("bfs", "sssp", "cc"):
        res = at.tune(algo, at.gpu_evaluator(g2, dg, algo, src=src), n_samples=10, seed=2)
        h = at.to_hybrid(g2, res.best)
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        if algo == "bfs":
            g2.g2_bfs(dg, src, out, None, h)
            want = oracle.bfs_graph(g, src, want_parent=False)[0]
        elif algo == "sssp":
            g2.g2_sssp_delta(dg, src, 0, out, h)
            want = oracle.sssp_graph(g, w, src)
        else:
            g2.g2_cc(dg, out, h)
            want = oracle.cc_graph(g)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want), (algo, res.best)
