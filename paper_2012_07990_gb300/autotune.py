"""Schedule autotuner (the role OpenTuner plays in Sec. VI-F of the paper).

The space is the scheduling language's (Table II fields and the Table III
hybrid threshold) plus the integer parameters the paper names: the delta of
delta-stepping and the EdgeBlocking segment size.  Search: random sampling of
the space (plus known-good seeds), then successive halving -- every surviving
candidate is timed again with more repetitions and the slower part dropped --
until one remains.  Results are cached in a JSON file keyed by a fingerprint of
the graph and the algorithm.

The evaluator is a callable ``cost(schedule_dict) -> milliseconds`` so the
search logic runs without a GPU; ``gpu_evaluator`` builds one that times the
CUDA library with CUDA events.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
import random
from dataclasses import dataclass, field

LBS = ["VERTEX_BASED", "CM", "WM", "STRICT", "EDGE_ONLY", "ETWC", "TWC"]
PUSH_FRONTIER_LBS = ["VERTEX_BASED", "CM", "WM", "STRICT", "ETWC", "TWC"]
# PUSH load balancing of a direction-optimising BFS hybrid fused into one
# launch (its PULL half: VERTEX_BASED over a bitmap, fused too)
FUSED_DO_PUSH_LBS = ["VERTEX_BASED", "WM", "CM", "ETWC", "STRICT"]
PULL_LBS = ["VERTEX_BASED", "WM", "CM"]


# ----------------------------------------------------------------- space
def _simple(**kw):
    d = {"lb": "VERTEX_BASED", "direction": 0, "pull_frontier": 0, "frontier_creation": 0,
         "dedup": True, "dedup_type": 0, "delta": 0, "kernel_fusion": False,
         "edge_blocking": False, "blocking_size": 0}
    d.update(kw)
    return d


def sample_schedule(algo: str, rng: random.Random) -> dict:
    """One random point of the schedule space for `algo`."""
    if algo in ("bfs", "bc"):
        push = _simple(lb=rng.choice(PUSH_FRONTIER_LBS), dedup=rng.random() < 0.5,
                       dedup_type=rng.randrange(3))
        if algo == "bfs" and rng.random() < 0.15:
            push.update(lb=rng.choice(["VERTEX_BASED", "WM", "CM", "ETWC"]), kernel_fusion=True)
            return {"criteria": 0, "threshold": 0.0, "s1": push, "s2": push}
        if algo == "bfs" and rng.random() < 0.15:
            return fused_do_hybrid(rng.choice(FUSED_DO_PUSH_LBS),
                                   rng.choice([0.002, 0.005, 0.01, 0.02, 0.05, 0.1]))
        pull = _simple(lb=rng.choice(PULL_LBS), direction=1, pull_frontier=rng.randrange(2),
                       frontier_creation=rng.randrange(3), dedup=False)
        tau = rng.choice([0.0, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1, 1e9])
        return {"criteria": 1, "threshold": tau, "s1": push, "s2": pull}
    if algo == "sssp":
        # deltas below 8 turn delta-stepping into thousands of near-empty
        # buckets on every input here (weights >= 1, means 128-500)
        delta = 2 ** rng.randrange(3, 15)
        fused = rng.random() < 0.3
        lb = rng.choice(["VERTEX_BASED", "WM", "CM", "ETWC"] if fused else PUSH_FRONTIER_LBS)
        s = _simple(lb=lb, delta=delta, kernel_fusion=fused,
                    dedup_type=0 if fused else rng.randrange(3))
        return {"criteria": 0, "threshold": 0.0, "s1": s, "s2": s}
    if algo == "cc":
        if rng.random() < 0.3:
            return {"tuned_default": True}
        if rng.random() < 0.5:
            s = _simple(lb=rng.choice(LBS))
        else:
            s = _simple(lb=rng.choice(PULL_LBS), direction=1, pull_frontier=rng.randrange(2))
        return {"criteria": 0, "threshold": 0.0, "s1": s, "s2": s}
    if algo == "pr":
        r = rng.random()
        if r < 0.4:
            return {"tuned_default": True}
        if r < 0.6:
            s = _simple(lb="EDGE_ONLY", direction=1)
        elif r < 0.8:
            s = _simple(lb=rng.choice(PULL_LBS), direction=1)
        else:
            eb = rng.random() < 0.5
            s = _simple(lb="EDGE_ONLY", edge_blocking=eb,
                        blocking_size=rng.choice([0, 1 << 16, 1 << 18, 1 << 20, 1 << 22]) if eb else 0)
        return {"criteria": 0, "threshold": 0.0, "s1": s, "s2": s}
    if algo == "bfs_batch":
        push = _simple(lb=rng.choice(PUSH_FRONTIER_LBS))
        pull = _simple(lb=rng.choice(["VERTEX_BASED", "WM"]), direction=1)
        return {"criteria": 1, "threshold": rng.choice([0.0, 0.005, 0.02, 0.05, 1e9]), "s1": push,
                "s2": pull}
    raise ValueError(f"unknown algorithm {algo}")


def fused_do_hybrid(lb: str, tau: float) -> dict:
    """The direction-optimising BFS hybrid in one cooperative launch: PUSH with
    load balancing `lb` while the frontier holds fewer than tau * n vertices,
    VERTEX_BASED PULL over a bitmap otherwise, kernel fusion on both."""
    return {"criteria": 1, "threshold": tau, "s1": _simple(lb=lb, kernel_fusion=True),
            "s2": _simple(lb="VERTEX_BASED", direction=1, pull_frontier=1, frontier_creation=2,
                          dedup=False, kernel_fusion=True)}


def seeds(algo: str) -> list[dict]:
    """Known-good starting points always included in the sample."""
    if algo == "bfs":
        # the library's tuned hybrid fused and as per-level launches, and the
        # fused WM loop of bounded-degree graphs
        return [fused_do_hybrid("STRICT", 0.02)] + seeds("bc")
    if algo == "bc":
        return [{"criteria": 1, "threshold": 0.02, "s1": _simple(lb="STRICT"),
                 "s2": _simple(lb="VERTEX_BASED", direction=1, pull_frontier=1, frontier_creation=2,
                               dedup=False)},
                {"criteria": 0, "threshold": 0.0, "s1": _simple(lb="WM", kernel_fusion=True),
                 "s2": _simple(lb="WM", kernel_fusion=True)}]
    if algo == "sssp":
        return [{"criteria": 0, "threshold": 0.0, "s1": _simple(lb="STRICT", delta=d),
                 "s2": _simple(lb="STRICT", delta=d)} for d in (64, 1024)] + \
               [{"criteria": 0, "threshold": 0.0, "s1": _simple(lb="WM", delta=4096, kernel_fusion=True),
                 "s2": _simple(lb="WM", delta=4096, kernel_fusion=True)}]
    if algo in ("cc", "pr"):
        return [{"tuned_default": True}]
    if algo == "bfs_batch":
        return [{"criteria": 1, "threshold": 0.02, "s1": _simple(lb="STRICT"),
                 "s2": _simple(lb="VERTEX_BASED", direction=1)}]
    return []


def key_of(d: dict) -> str:
    return json.dumps(d, sort_keys=True)


# ---------------------------------------------------------- exhaustive search
HYBRID_THRESHOLDS = (0.0, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1)


def enumerate_direction(direction: int) -> list[dict]:
    """Every simple schedule of one traversal direction: the cartesian
    product of the Table II fields (Sec. V, Table I counts 288 per direction
    for the paper's compiler): load balancing (7) x EdgeBlocking (2) x output
    frontier creation (3) x kernel fusion (2) x deduplication (PUSH: disabled,
    or enabled with one of the 3 dedup types -- 4; PULL: disabled or enabled
    -- 2, times the 2 representations of the PULL input frontier) = 336 points
    per direction.  Points an algorithm cannot run (EdgeBlocking outside
    EDGE_ONLY sweeps, EDGE_ONLY without the all-vertices frontier, PULL with
    a load balancing it has no pull form for, ...) are part of the space; the
    library rejects them and the search drops them."""
    out = []
    for lb in LBS:
        for eb in (False, True):
            for fc in (0, 1, 2):
                for kf in (False, True):
                    if direction == 0:
                        for dd in ((False, 0), (True, 0), (True, 1), (True, 2)):
                            out.append(_simple(lb=lb, edge_blocking=eb, frontier_creation=fc,
                                               kernel_fusion=kf, dedup=dd[0], dedup_type=dd[1]))
                    else:
                        for dedup in (False, True):
                            for pf in (0, 1):
                                out.append(_simple(lb=lb, direction=1, edge_blocking=eb,
                                                   frontier_creation=fc, kernel_fusion=kf,
                                                   dedup=dedup, pull_frontier=pf))
    return out


@dataclass
class ExhaustiveResult:
    best: dict
    best_ms: float
    evaluated: int          # points timed (rejected ones included)
    rejected: int           # points the library refused
    per_direction: dict     # direction -> (best schedule, ms, points, rejected)


def exhaustive(cost, reps: int = 2, top: int = 4,
               thresholds=HYBRID_THRESHOLDS) -> ExhaustiveResult:
    """Time every simple schedule of both directions (each alone, criteria
    NONE), then every hybrid of the `top` fastest unfused PUSH and PULL
    schedules at each threshold, and the direction-optimising hybrid fused
    into one launch with each of its PUSH load balancings at each threshold
    (algorithms without that form refuse it); the fastest of all is the
    optimum of the space."""
    timed = []
    evaluated = rejected = 0
    per_dir = {}
    for direction in (0, 1):
        ok = []
        pts = enumerate_direction(direction)
        for s in pts:
            d = {"criteria": 0, "threshold": 0.0, "s1": s, "s2": s}
            evaluated += 1
            try:
                t = min(cost(d) for _ in range(reps))
            except Exception:
                rejected += 1
                continue
            ok.append((t, s))
            timed.append((t, d))
        ok.sort(key=lambda x: x[0])
        per_dir[direction] = {"best": ok[0][1] if ok else None, "ms": ok[0][0] if ok else None,
                              "points": len(pts), "rejected": len(pts) - len(ok)}
        per_dir[direction]["top"] = [s for _, s in ok[:top]]
    for s1 in per_dir[0]["top"]:
        for s2 in per_dir[1]["top"]:
            if s1["kernel_fusion"] or s2["kernel_fusion"]:
                continue  # a fused loop runs s1 throughout: no hybrid
            for tau in thresholds:
                d = {"criteria": 1, "threshold": tau, "s1": s1, "s2": s2}
                evaluated += 1
                try:
                    t = min(cost(d) for _ in range(reps))
                except Exception:
                    rejected += 1
                    continue
                timed.append((t, d))
    for lb in FUSED_DO_PUSH_LBS:
        for tau in thresholds:
            d = fused_do_hybrid(lb, tau)
            evaluated += 1
            try:
                t = min(cost(d) for _ in range(reps))
            except Exception:
                rejected += 1
                continue
            timed.append((t, d))
    timed.sort(key=lambda x: x[0])
    if not timed:
        raise RuntimeError("no schedule could be evaluated")
    for v in per_dir.values():
        v.pop("top", None)
    return ExhaustiveResult(timed[0][1], timed[0][0], evaluated, rejected, per_dir)


# ------------------------------------------------------------ the search
@dataclass
class TuneResult:
    best: dict
    best_ms: float
    evaluated: int
    history: list = field(default_factory=list)


def successive_halving(cost, candidates: list[dict], reps0: int = 1, eta: int = 3,
                       max_evals: int | None = None) -> TuneResult:
    """Time every candidate with reps0 repetitions, keep the best 1/eta, time
    the survivors with eta-times more repetitions, ... until one is left.
    Candidates whose evaluation raises are dropped (unsupported combinations)."""
    alive = []
    seen = set()
    for c in candidates:
        k = key_of(c)
        if k not in seen:
            seen.add(k)
            alive.append(c)
    history = []
    evals = 0
    reps = reps0
    scores: dict[str, float] = {}
    while alive:
        scored = []
        for c in alive:
            if max_evals is not None and evals >= max_evals:
                break
            try:
                t = min(cost(c) for _ in range(reps))
            except Exception as e:  # unsupported / invalid: drop it
                history.append({"schedule": c, "error": str(e)[:120]})
                evals += 1
                continue
            evals += reps
            scores[key_of(c)] = t
            scored.append((t, c))
            history.append({"schedule": c, "ms": t, "reps": reps})
        if not scored:
            break
        scored.sort(key=lambda x: x[0])
        if len(scored) == 1 or (max_evals is not None and evals >= max_evals):
            best_ms, best = scored[0]
            return TuneResult(best, best_ms, evals, history)
        keep = max(1, int(math.ceil(len(scored) / eta)))
        alive = [c for _, c in scored[:keep]]
        reps *= eta
    raise RuntimeError("no schedule could be evaluated")


def tune(algo: str, cost, n_samples: int = 24, seed: int = 1, eta: int = 3,
         max_evals: int | None = None, warm: list[dict] | None = None) -> TuneResult:
    """Search `n_samples` random points plus the known-good seeds and any
    warm-start schedules (tried first)."""
    rng = random.Random(seed)
    cands = list(warm or []) + seeds(algo) + [sample_schedule(algo, rng) for _ in range(n_samples)]
    return successive_halving(cost, cands, eta=eta, max_evals=max_evals)


# ----------------------------------------------------------------- cache
def graph_fingerprint(n: int, rowptr, col) -> str:
    """Stable fingerprint of a CSR graph: sizes and a strided sample of arrays."""
    import numpy as np
    h = hashlib.sha256()
    h.update(np.int64([n, len(col)]).tobytes())
    rp = np.asarray(rowptr)
    cl = np.asarray(col)
    step_r = max(1, rp.size // 4096)
    step_c = max(1, cl.size // 65536)
    h.update(np.ascontiguousarray(rp[::step_r]).tobytes())
    h.update(np.ascontiguousarray(cl[::step_c]).tobytes())
    return h.hexdigest()[:24]


def graph_features(n: int, rowptr) -> list[float]:
    """What the best schedule depends on, as a small vector: log2 of the
    vertex and arc counts, log2 of the mean and maximum degree, the share of
    vertices without arcs, and the coefficient of variation of the degrees
    (power-law graphs: large; road-like grids: small)."""
    import numpy as np
    deg = np.diff(np.asarray(rowptr, dtype=np.int64))
    m = int(deg.sum())
    mean = m / max(n, 1)
    cv = float(deg.std() / mean) if mean > 0 else 0.0
    return [math.log2(max(n, 1)), math.log2(max(m, 1)), math.log2(max(mean, 1e-9) + 1.0),
            math.log2(float(deg.max(initial=0)) + 1.0), float((deg == 0).mean()) * 10.0,
            math.log2(cv + 1.0) * 4.0]


class TuneCache:
    """JSON cache: per graph fingerprint and algorithm, the best schedules
    found (best first) and the graph's features, which warm-start the search
    on graphs that were never tuned."""

    def __init__(self, path: str):
        self.path = path
        self.data = {}
        if os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)

    def get(self, fp: str, algo: str):
        return self.data.get(f"{fp}:{algo}")

    def put(self, fp: str, algo: str, result: TuneResult, features: list[float] | None = None,
            top: int = 3):
        ranked = sorted((h for h in result.history if "ms" in h),
                        key=lambda h: (-h["reps"], h["ms"]))
        best, seen = [], set()
        for h in [{"schedule": result.best}] + ranked:
            k = key_of(h["schedule"])
            if k not in seen:
                seen.add(k)
                best.append(h["schedule"])
            if len(best) == top:
                break
        self.data[f"{fp}:{algo}"] = {"schedule": result.best, "ms": result.best_ms,
                                      "evaluated": result.evaluated, "top": best,
                                      "features": features}
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def warm_start(self, features: list[float], algo: str, k: int = 2) -> list[dict]:
        """The best schedules of the k cached graphs nearest to `features`
        (Euclidean distance), nearest first."""
        near = []
        for key, v in self.data.items():
            if not key.endswith(f":{algo}") or not v.get("features"):
                continue
            d = math.dist(v["features"], features)
            near.append((d, v.get("top") or [v["schedule"]]))
        near.sort(key=lambda x: x[0])
        out, seen = [], set()
        for _, tops in near[:k]:
            for sch in tops:
                if key_of(sch) not in seen:
                    seen.add(key_of(sch))
                    out.append(sch)
        return out


def tune_cached(cache: TuneCache, fp: str, algo: str, cost, features: list[float] | None = None,
                warm_k: int = 2, **kw) -> dict:
    """The cached best schedule of this graph, else a search warm-started
    from the nearest tuned graphs (when features are given), then cached."""
    hit = cache.get(fp, algo)
    if hit is not None:
        return hit["schedule"]
    warm = cache.warm_start(features, algo, warm_k) if features is not None else None
    res = tune(algo, cost, warm=warm, **kw)
    cache.put(fp, algo, res, features)
    return res.best


# --------------------------------------------------------- GPU binding
def to_hybrid(g2, d: dict):
    """Schedule dict -> g2_hybrid (None for the library's tuned default)."""
    if d.get("tuned_default"):
        return None

    def mk(s):
        return g2.schedule(s["lb"], direction=s["direction"], pull_frontier=s["pull_frontier"],
                           frontier_creation=s["frontier_creation"], dedup=s["dedup"],
                           dedup_type=s["dedup_type"], delta=s["delta"],
                           kernel_fusion=s["kernel_fusion"], edge_blocking=s["edge_blocking"],
                           blocking_size=s["blocking_size"])

    h = g2.g2_hybrid()
    h.criteria = d["criteria"]
    h.threshold = float(min(d["threshold"], 3.0e38))
    h.s1 = mk(d["s1"])
    h.s2 = mk(d["s2"])
    return h


def gpu_evaluator(g2, dg, algo: str, src: int = 0, srcs=None, n: int | None = None):
    """cost(schedule) in milliseconds, timed with CUDA events on the current
    stream, for algorithm `algo` on the loaded graph `dg`."""
    import torch
    n = dg.n if n is None else n
    out_i = torch.empty(n * (64 if algo == "bfs_batch" else 1), dtype=torch.int32, device="cuda")
    out_f = torch.empty(n, dtype=torch.float32, device="cuda")
    out_d = torch.empty(n, dtype=torch.float64, device="cuda")

    def run(d):
        h = to_hybrid(g2, d)
        if algo == "bfs":
            g2.g2_bfs(dg, src, out_i, None, h)
        elif algo == "sssp":
            g2.g2_sssp_delta(dg, src, 0, out_i, h)
        elif algo == "cc":
            g2.g2_cc(dg, out_i, h)
        elif algo == "pr":
            g2.g2_pagerank(dg, 0.85, 20, out_f, h)
        elif algo == "bc":
            g2.g2_bc(dg, [src], out_d, h)
        elif algo == "bfs_batch":
            g2.g2_bfs_batch(dg, srcs, out_i, h)

    def cost(d):
        run(d)  # warm (layouts, workspace)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run(d)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    return cost
