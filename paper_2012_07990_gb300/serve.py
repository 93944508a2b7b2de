"""Continuous-batching query server over a resident pool of graphs.

Requests (BFS, SSSP or single-source BC from one vertex of one graph) arrive
on an open-loop trace.  The dispatcher keeps one queue per (graph, kind); as
soon as an execution slot is free and the memory budget allows, it takes the
queue whose oldest request has waited longest and forms a batch of everything
waiting there, up to the batch cap (64 BFS sources -> one g2_bfs_batch call,
32 SSSP sources -> one g2_sssp_batch call, BC one source per call).  Each slot
is a host thread with its own CUDA stream and its own view of every graph
(g2_graph_view: shared topology, private workspace), so batches on different
slots run concurrently on the device while new requests keep being admitted.

Memory admission: every batch reserves its output bytes plus a workspace
estimate from a budget (default: half of the free device memory at start-up)
and returns them when it completes; a batch that does not fit is shrunk, or
waits until enough memory is released.

Latency = completion - arrival (open loop).  Throughput (GTEPS) counts, per
request, the arcs of the source's connected component (what BFS / SSSP / BC
from that source traverse) over the makespan.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np

KINDS = ("bfs", "sssp", "bc")


@dataclass
class Request:
    rid: int
    t_arrival: float
    graph: str
    kind: str
    src: int


@dataclass
class GraphSpec:
    name: str
    make: object          # callable -> graphgen.Graph
    wmax: int             # weights U[1, wmax]
    delta: int            # delta-stepping bucket width for this graph
    road: bool = False    # high diameter: single queries run fused loops


@dataclass
class PoolGraph:
    spec: GraphSpec
    host: object
    weights: np.ndarray
    handle: object
    comp_arcs: np.ndarray  # arcs of each vertex's connected component
    nonisolated: np.ndarray


def default_pool_specs(scales=(16, 18, 20, 22), grids=(512, 1024, 2048, 4096)) -> list[GraphSpec]:
    """The serving pool of the workload: RMAT scales 16-22 and road grids
    512^2-4096^2, seed 1."""
    from paper_2012_07990_gb300 import graphgen as gg
    specs = [GraphSpec(f"rmat{s}", (lambda s=s: gg.rmat(s, seed=1)), 255, 64) for s in scales]
    specs += [GraphSpec(f"grid{w}", (lambda w=w: gg.road_grid(w, seed=1)), 1000, 4096, True)
              for w in grids]
    return specs


class GraphPool:
    """Graphs resident on the device, with per-graph request metadata."""

    def __init__(self, g2, specs: list[GraphSpec]):
        import torch
        from paper_2012_07990_gb300 import graphgen as gg
        self.graphs: dict[str, PoolGraph] = {}
        for sp in specs:
            G = sp.make()
            w = gg.pair_weights(G, sp.wmax, seed=1)
            h = g2.load_graph(G, w)
            lab = torch.empty(G.n, dtype=torch.int32, device="cuda")
            g2.g2_cc(h, lab, None)
            lab = lab.cpu().numpy()
            arcs = np.bincount(lab, weights=G.degrees(), minlength=G.n)
            self.graphs[sp.name] = PoolGraph(sp, G, w, h, arcs[lab].astype(np.int64),
                                             np.nonzero(G.degrees() > 0)[0].astype(np.int32))

    def footprint_bytes(self) -> int:
        return sum(4 * (g.host.n + 1) + 8 * g.host.m for g in self.graphs.values())


def make_trace(pool, rate: float, duration: float, mix=(0.6, 0.3, 0.1), seed: int = 1):
    """Poisson arrivals at `rate` per second for `duration` seconds; kind by
    `mix` (BFS, SSSP, BC), graph uniform over the pool, source uniform over the
    graph's non-isolated vertices."""
    rng = np.random.default_rng(seed)
    names = list(pool.graphs)
    p = np.asarray(mix, dtype=np.float64)
    p = p / p.sum()
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        kind = KINDS[int(rng.choice(3, p=p))]
        gname = names[int(rng.integers(len(names)))]
        cand = pool.graphs[gname].nonisolated
        src = int(cand[rng.integers(cand.size)]) if cand.size else 0
        out.append(Request(len(out), t, gname, kind, src))
    return out


@dataclass
class ServeStats:
    latencies_ms: np.ndarray
    makespan_s: float
    arcs: int
    batches: int
    mean_batch: float
    max_concurrent: int
    results: dict = field(default_factory=dict)

    @property
    def p50(self):
        return float(np.percentile(self.latencies_ms, 50)) if self.latencies_ms.size else 0.0

    @property
    def p99(self):
        return float(np.percentile(self.latencies_ms, 99)) if self.latencies_ms.size else 0.0

    @property
    def gteps(self):
        return self.arcs / self.makespan_s / 1e9 if self.makespan_s > 0 else 0.0

    def summary(self) -> dict:
        return {"requests": int(self.latencies_ms.size), "p50_ms": round(self.p50, 3),
                "p99_ms": round(self.p99, 3), "gteps": round(self.gteps, 3),
                "makespan_s": round(self.makespan_s, 3), "batches": self.batches,
                "mean_batch": round(self.mean_batch, 2), "max_concurrent": self.max_concurrent}


def batch_bytes(kind: str, k: int, n: int) -> int:
    """Device bytes a batch holds while it runs: outputs + workspace estimate."""
    out = {"bfs": 4 * k * n, "sssp": 4 * k * n, "bc": 8 * n}[kind]
    work = {"bfs": 40 * n, "sssp": 48 * n, "bc": 44 * n}[kind]
    return out + work


class GpuExecutor:
    """Runs one batch on one slot: the slot's stream, the slot's graph views."""

    def __init__(self, g2, pool: GraphPool, slots: int, keep_results: bool = False):
        import torch
        self.g2 = g2
        self.pool = pool
        self.nslots = slots
        self.keep_results = keep_results
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.views = [{name: g.handle.view() for name, g in pool.graphs.items()} for _ in range(slots)]
        self.fused = g2.schedule("WM", kernel_fusion=True)
        # A single BFS on a power-law graph: with several slots, the tuned
        # hybrid's schedules as per-level launches, whose small kernels
        # interleave with the other slots' work (the fused form's cooperative
        # launch needs every SM at once, so the slots' launches would run one
        # at a time); with one slot, the library's tuned schedule (NULL).
        self.powerlaw_bfs = None
        if slots > 1:
            pull = g2.schedule("VERTEX_BASED", direction=g2.G2_PULL, pull_frontier=g2.G2_BITMAP,
                               frontier_creation=g2.G2_UNFUSED_BITMAP, dedup=False)
            self.powerlaw_bfs = g2.hybrid(g2.schedule("STRICT"), pull, 0.02)

    def execute(self, slot: int, batch: list[Request]) -> dict:
        import torch
        g2 = self.g2
        r0 = batch[0]
        pg = self.pool.graphs[r0.graph]
        n = pg.host.n
        view = self.views[slot][r0.graph]
        srcs = np.array([r.src for r in batch], dtype=np.int32)
        k = len(batch)
        single = self.fused if pg.spec.road else None
        with torch.cuda.stream(self.streams[slot]):
            if r0.kind == "bfs":
                out = torch.empty(k * n, dtype=torch.int32, device="cuda")
                if k == 1:
                    g2.g2_bfs(view, int(srcs[0]), out, None,
                              single if pg.spec.road else self.powerlaw_bfs)
                else:
                    g2.g2_bfs_batch(view, srcs, out, None)
            elif r0.kind == "sssp":
                out = torch.empty(k * n, dtype=torch.int32, device="cuda")
                if k == 1:
                    g2.g2_sssp_delta(view, int(srcs[0]), pg.spec.delta, out, single)
                else:
                    g2.g2_sssp_batch(view, srcs, pg.spec.delta, out, None)
            else:
                out = torch.empty(n, dtype=torch.float64, device="cuda")
                g2.g2_bc(view, srcs, out, single)
            if self.keep_results:
                host = out.cpu().numpy()
                rows = host.reshape(k, n) if r0.kind != "bc" else host.reshape(1, n)
                return {r.rid: rows[i].copy() for i, r in enumerate(batch)}
        return {}


class CostModel:
    """Execution seconds of a batch per (graph, kind): an exponentially
    weighted average of the batches seen so far (None before the first)."""

    def __init__(self, alpha: float = 0.3):
        self.alpha = alpha
        self.est: dict = {}

    def get(self, key):
        return self.est.get(key)

    def update(self, key, seconds: float):
        old = self.est.get(key)
        self.est[key] = seconds if old is None else (1 - self.alpha) * old + self.alpha * seconds


def _pick_queue(policy, cost, pending, now):
    """The (graph, kind) queue to dispatch next under `policy`."""
    if policy == "fifo":
        return min(pending, key=lambda kk: pending[kk][0].t_arrival)
    best, best_r = None, -1.0
    for kk, q in pending.items():
        c = cost.get(kk)
        if c is None:
            return kk  # never measured: run it to learn its cost
        wait = max(0.0, now - q[0].t_arrival)
        r = (wait + c) / max(c, 1e-6)
        if r > best_r:
            best, best_r = kk, r
    return best


class Server:
    """Continuous-batching dispatcher over `executor.nslots` slots.

    policy "hrrn" (default): highest response ratio next -- among the
    non-empty queues take the one maximising (wait + cost) / cost, where wait
    is the age of its oldest request and cost the learned execution time of
    a batch of it (a queue never run yet goes first, to be measured); short
    batches overtake long ones, and a long one's ratio grows with its wait.
    policy "fifo": the queue whose oldest request has waited longest."""

    def __init__(self, executor, pool, max_batch=None, mem_budget: int | None = None,
                 policy: str = "hrrn"):
        if policy not in ("hrrn", "fifo"):
            raise ValueError(f"unknown policy {policy}")
        self.policy = policy
        self.cost = CostModel()
        self.ex = executor
        self.pool = pool
        self.max_batch = dict(bfs=64, sssp=32, bc=1)
        if max_batch is not None:
            self.max_batch.update(max_batch)
        if mem_budget is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            mem_budget = free // 2
        self.mem_budget = int(mem_budget)

    def _pick(self, pending, now):
        return _pick_queue(self.policy, self.cost, pending, now)

    def run(self, trace: list[Request], clock=time.perf_counter) -> ServeStats:
        pending = {}  # (graph, kind) -> deque of requests that have arrived
        lock = threading.Condition()
        free_slots = list(range(self.ex.nslots))
        mem_used = [0]
        running = [0]
        max_running = [0]
        done_t = {}
        results = {}
        sizes = []
        errors = []
        t0 = clock()

        def worker(slot, batch, nbytes):
            ts = clock()
            try:
                res = self.ex.execute(slot, batch)
            except Exception as e:  # re-raised by the dispatcher
                errors.append(e)
                res = {}
            t = clock() - t0
            with lock:
                self.cost.update((batch[0].graph, batch[0].kind), clock() - ts)
                for r in batch:
                    done_t[r.rid] = t
                results.update(res)
                mem_used[0] -= nbytes
                running[0] -= 1
                free_slots.append(slot)
                lock.notify_all()

        order = sorted(trace, key=lambda r: r.t_arrival)
        i, total = 0, len(order)
        with lock:
            while len(done_t) < total:
                if errors:
                    raise errors[0]
                now = clock() - t0
                while i < total and order[i].t_arrival <= now:
                    r = order[i]
                    pending.setdefault((r.graph, r.kind), collections.deque()).append(r)
                    i += 1
                launched = False
                while free_slots and pending:
                    key = self._pick(pending, clock() - t0)
                    q = pending[key]
                    kind = key[1]
                    n = self.pool.graphs[key[0]].host.n
                    k = min(len(q), self.max_batch[kind])
                    nbytes = batch_bytes(kind, k, n)
                    while k > 1 and mem_used[0] + nbytes > self.mem_budget:
                        k = max(1, k // 2)
                        nbytes = batch_bytes(kind, k, n)
                    if mem_used[0] > 0 and mem_used[0] + nbytes > self.mem_budget:
                        break  # wait until running batches release memory
                    batch = [q.popleft() for _ in range(k)]
                    if not q:
                        del pending[key]
                    slot = free_slots.pop()
                    mem_used[0] += nbytes
                    running[0] += 1
                    max_running[0] = max(max_running[0], running[0])
                    sizes.append(k)
                    threading.Thread(target=worker, args=(slot, batch, nbytes), daemon=True).start()
                    launched = True
                if not launched:
                    wait = order[i].t_arrival - (clock() - t0) if i < total else 0.05
                    lock.wait(timeout=max(1e-4, min(wait, 0.05)))
        if errors:
            raise errors[0]
        lat = np.array([(done_t[r.rid] - r.t_arrival) * 1e3 for r in trace])
        makespan = max(done_t.values()) if done_t else 0.0
        arcs = int(sum(self.pool.graphs[r.graph].comp_arcs[r.src] for r in trace))
        return ServeStats(lat, makespan, arcs, len(sizes), float(np.mean(sizes)) if sizes else 0.0,
                          max_running[0], results)


def serve_alone(g2, pool: GraphPool, trace: list[Request]) -> dict:
    """Every request run by itself with plain single-query launches."""
    ex = GpuExecutor(g2, pool, slots=1, keep_results=True)
    out = {}
    for r in trace:
        out.update(ex.execute(0, [r]))
    return out
