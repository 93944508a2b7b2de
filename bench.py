#!/usr/bin/env python3
"""Benchmark of the g2 hot path on one GB300 (or N independent replicas).

Workload (default ``rmat22``): synthetic RMAT graph, scale 22 (4,194,304
vertices), edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), seed 1,
symmetrised, self-loops and duplicates dropped, int32 CSR (the CSC aliases
it).  One step = direction-optimising BFS from the max-degree vertex + connected
components + PageRank (d = 0.85, 20 rounds), all through the C ABI with the
graph and outputs resident in HBM.

value = traversed edges per step / step time, in GTEPS, where traversed edges =
the arcs whose source BFS reached + m (CC) + 20 m (PageRank).

Also reported: per-algorithm times; the dominant kernel's roofline (PageRank
round kernel, CUDA events around its launches); end-to-end GTEPS through the
public API with host buffers (graph upload from pinned host memory, results
read back); the CPU oracle on a bounded sample; SM clocks sampled during the
timed region.

``--impl reference`` times the CPU oracle (the plain reference of this
method) on the same workload, each step a bounded sample (BFS + CC + one
PageRank round).  Under torchrun only rank 0 runs it.

Multi-GPU: the path does not shard, so ``--gpus N`` runs N independent replicas
(one per rank, weak scaling) with no data-path collective; value = all edges
traversed by all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
PR_ITERS = 20
DAMPING = 0.85
TIMED_EVERY = 4  # steps of the timed region whose PageRank launches carry event pairs


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int) -> float:
    """The largest `value` over the ranks (the slowest replica's time); the
    reduction runs on the device under NCCL and on the host under gloo."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gteps(ws: int, edges_per_step: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: every replica traverses edges_per_step per step;
    the job takes the slowest replica's time."""
    return ws * edges_per_step * steps / (total_ms * 1e-3) / 1e9


def make_graph(scale: int):
    from paper_2012_07990_gb300 import graphgen as gg
    return gg.rmat(scale, 16, 0.57, 0.19, 0.19, seed=1)


def bfs_schedule(g2):
    """The library's tuned BFS schedule (NULL): the direction-optimising
    hybrid (Table III) fused into one launch, STRICT PUSH on a sparse queue
    while |frontier| < 2% of n, else VERTEX_BASED PULL over a bitmap."""
    return None


def bfs_per_level_hybrid(g2):
    """The tuned hybrid's schedules as per-level launches (the frontier size
    read back by the host every level).  The bench step runs BFS this way:
    beside PageRank on another stream its small kernels fill the gaps between
    the sweeps, where the fused form's cooperative launch needs every SM at
    once and waits for them (step 3.48 ms against 3.35 ms)."""
    pull = g2.schedule("VERTEX_BASED", direction=g2.G2_PULL, pull_frontier=g2.G2_BITMAP,
                       frontier_creation=g2.G2_UNFUSED_BITMAP, dedup=False)
    return g2.hybrid(g2.schedule("STRICT"), pull, 0.02)


def cc_schedule(g2):
    """The library's tuned CC (NULL): lock-free linking with neighbour
    sampling, then pointer jumping."""
    return None


# ------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2

    G = make_graph(args.scale)
    n, m = G.n, G.m
    src = G.max_degree_vertex()
    dg = g2.load_graph(G)
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    label = torch.empty(n, dtype=torch.int32, device="cuda")
    rank_t = torch.empty(n, dtype=torch.float32, device="cuda")
    sb, sc = bfs_per_level_hybrid(g2), cc_schedule(g2)
    launches = {"n": 0}
    # BFS and CC are independent of PageRank: in a step they run from two
    # worker threads, each on a graph view (own workspace) and a stream of its
    # own, while PageRank runs on this thread's stream; their per-round host
    # round trips then overlap PageRank's sweeps instead of idling the GPU.
    # PageRank's stream has the higher priority: the block scheduler starts
    # its CTAs first, and BFS's and CC's fill the gaps between its kernels
    # instead of holding SMs its whole-SM sweep CTAs wait for.
    from concurrent.futures import ThreadPoolExecutor
    views = {"bfs": g2.g2_graph_view(dg), "cc": g2.g2_graph_view(dg)}
    streams = {"bfs": torch.cuda.Stream(), "cc": torch.cuda.Stream()}
    pr_stream = torch.cuda.Stream(priority=-5)  # the highest priority the device has
    pool = ThreadPoolExecutor(2)

    def bfs_job():
        g2.g2_bfs(views["bfs"], src, depth, parent, sb, stream=streams["bfs"])
        return g2.g2_last_stats()["launches"]

    def cc_job():
        g2.g2_cc(views["cc"], label, sc, stream=streams["cc"])
        return g2.g2_last_stats()["launches"]

    def step(t_algo=None):
        if t_algo is None:
            fb, fc = pool.submit(bfs_job), pool.submit(cc_job)
            g2.g2_pagerank(dg, DAMPING, PR_ITERS, rank_t, stream=pr_stream)
            launches["n"] += g2.g2_last_stats()["launches"] + fb.result() + fc.result()
            return
        # the per-algorithm split: the three one after another on this stream
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        evs[0].record()
        g2.g2_bfs(dg, src, depth, parent, sb)
        evs[1].record()
        g2.g2_cc(dg, label, sc)
        evs[2].record()
        g2.g2_pagerank(dg, DAMPING, PR_ITERS, rank_t)
        evs[3].record()
        t_algo.append(evs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    deg = G.degrees()
    reached = depth.cpu().numpy() >= 0
    m_bfs = int(deg[reached].sum())
    edges_per_step = m_bfs + m + PR_ITERS * m

    # per-algorithm split (separate, untimed-for-value pass)
    t_algo = []
    for _ in range(max(2, min(args.steps, 5))):
        step(t_algo)
    torch.cuda.synchronize()
    per = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(3)] for e in t_algo])
    bfs_ms, cc_ms, pr_ms = (float(x) for x in np.median(per, axis=0))

    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    g2.g2_kernel_time("pr_round", reset=True)
    g2.g2_kernel_time("pr_vertex", reset=True)
    launches["n"] = 0
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    # PageRank's kernels are timed with CUDA events in every TIMED_EVERY-th
    # step of the timed region: an event pair around each launch keeps the
    # next kernel from starting before the last one has drained, which costs
    # a step about 6% when every launch carries one
    for i in range(args.steps):
        g2.g2_set_kernel_timing(i % TIMED_EVERY == 0)
        step()
    e1.record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    g2.g2_set_kernel_timing(False)
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    pv_ms_total, pv_launches = g2.g2_kernel_time("pr_vertex", reset=False)
    pr_ms_total, pr_launches = g2.g2_kernel_time("pr_round", reset=True)
    total_ms = max_over_ranks(total_ms, ws)
    ms_per_step = total_ms / args.steps
    value = job_gteps(ws, edges_per_step, args.steps, total_ms)

    # roofline of the dominant kernel: the PageRank arc sweep (PULL + EDGE_ONLY
    # over the source-blocked layout, k_pr_blk).  Algorithmic bytes of one
    # sweep = 4 m (a column id per arc) + 4 n (each share read once) + 4 n
    # (each row sum written once); of a whole round (sweep + vertex pass) =
    # 4 m + 4 (n + 1) + 16 n (column ids, row offsets, shares written, rank
    # read and written, out-degrees).
    peak, peak_kind = read_peaks()
    alg_bytes = 4 * m + 8 * n
    round_bytes = 4 * m + 4 * (n + 1) + 16 * n
    avg_launch_ms = pr_ms_total / max(pr_launches, 1)
    avg_vertex_ms = pv_ms_total / max(pv_launches, 1)
    achieved = alg_bytes / (avg_launch_ms * 1e-3) / 1e9
    round_achieved = round_bytes / ((avg_launch_ms + avg_vertex_ms) * 1e-3) / 1e9
    traffic = read_traffic("pr_round", G)
    roofline = {"kernel": "k_pr_blk (PageRank round: source-blocked CSC arc sweep)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "bytes_per_launch": int(alg_bytes), "avg_launch_us": round(avg_launch_ms * 1e3, 2),
                "launches": pr_launches,
                "launches_timed": f"every {TIMED_EVERY}th step of the timed region, CUDA events on the "
                                  "launching stream",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "vertex_pass_us": round(avg_vertex_ms * 1e3, 2),
                "limits": (read_profile_record("pr_round") or {}).get("ncu_limits"),
                "round": {"bytes": int(round_bytes), "us": round((avg_launch_ms + avg_vertex_ms) * 1e3, 2),
                          "achieved": round(round_achieved, 1), "frac": round(round_achieved / peak, 4)}}

    pool.shutdown()
    for v in views.values():
        v.free()
    e2e = run_e2e(args, g2, G, src, sb, sc, edges_per_step) if not args.no_e2e else None
    extras = None
    if rank == 0 and ws == 1 and not args.no_extras:
        extras = run_extras(g2, G, dg, src, sb, sc)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(G, src, budget_s=args.cpu_budget)

    if rank == 0:
        line = {
            "metric": "GTEPS (direction-optimising BFS + CC + PageRank x20 on RMAT-22), % HBM roofline",
            "value": round(value, 2), "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32+f32",
            "data": "synthetic RMAT (seeded, counter-based generator)",
            "config": {"workload": f"rmat{args.scale}_bfs_cc_pr",
                       "graph": f"RMAT scale {args.scale}, ef 16, (0.57,0.19,0.19,0.05), seed 1, symmetric",
                       "n": n, "m": m, "src": src, "pr_rounds": PR_ITERS, "damping": DAMPING,
                       "edges_per_step": edges_per_step, "bfs_reached_arcs": m_bfs,
                       "bfs_parent": True,
                       "bfs_schedule": "direction-optimising hybrid as per-level launches (beside PageRank's stream)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                       "l2": "inputs larger than L2 (CSR 513 MB vs 129 MB L2); no flush"},
            "per_algo": {"bfs_ms": round(bfs_ms, 4), "cc_ms": round(cc_ms, 4), "pr_ms": round(pr_ms, 4),
                         "bfs_gteps": round(m_bfs / bfs_ms / 1e6, 2),
                         "cc_gteps": round(m / cc_ms / 1e6, 2),
                         "pr_gteps": round(PR_ITERS * m / pr_ms / 1e6, 2)},
            "roofline": roofline,
            "workloads": extras,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": launches["n"],
            "clocks": clk,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_e2e(args, g2, G, src, sb, sc, edges_per_step):
    """Same metric through the public API with host buffers: every step
    uploads the graph from pinned host memory (g2_load_csr, PageRank's layouts
    prepared in the background), runs the three algorithms and reads the
    results (depth, label, rank) back to pinned host memory.  The steps are
    pipelined the way a stream of graphs would be served: a loader thread
    uploads step k+1's graph on a stream of its own while step k computes
    (two graphs resident), so the host link overlaps the kernels; within a
    step BFS and CC run beside PageRank, as in the device-timed step.  The timed
    region holds every step's upload (the first one included), compute and
    read-back; the median of three such timed runs is reported.
    `serial_ms_per_step` is the same step run one after another.
    Results read back per step: BFS depth and parent, CC labels, PageRank."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    n, m = G.n, G.m
    h_rp = torch.from_numpy(G.rowptr).pin_memory()
    h_col = torch.from_numpy(G.col).pin_memory()
    rp_np = np.frombuffer(h_rp.numpy().data, dtype=np.int32)
    col_np = np.frombuffer(h_col.numpy().data, dtype=np.int32)
    h_depth = torch.empty(n, dtype=torch.int32).pin_memory()
    h_parent = torch.empty(n, dtype=torch.int32).pin_memory()
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    h_label = torch.empty(n, dtype=torch.int32).pin_memory()
    h_rank = torch.empty(n, dtype=torch.float32).pin_memory()
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    label = torch.empty(n, dtype=torch.int32, device="cuda")
    rank_t = torch.empty(n, dtype=torch.float32, device="cuda")
    # all at the default priority: with PageRank's stream above the loader's
    # the next graph's layout build starved and the pipeline slowed down
    # (5.9-7.4 ms per step against 5.9-6.0)
    main = torch.cuda.current_stream()
    load_stream = torch.cuda.Stream()
    s_bfs, s_cc = torch.cuda.Stream(), torch.cuda.Stream()
    workers = ThreadPoolExecutor(2)

    def load():
        return g2.g2_load_csr(n, rp_np, col_np, None, True, stream=load_stream,
                              prepare_pagerank=True, overlap=True)

    def bfs_job(v):
        g2.g2_bfs(v, src, depth, parent, sb, stream=s_bfs)
        with torch.cuda.stream(s_bfs):
            h_depth.copy_(depth, non_blocking=True)
            h_parent.copy_(parent, non_blocking=True)
        s_bfs.synchronize()

    def cc_job(v):
        g2.g2_cc(v, label, sc, stream=s_cc)
        with torch.cuda.stream(s_cc):
            h_label.copy_(label, non_blocking=True)
        s_cc.synchronize()

    def compute(dg):
        # as in the device-timed step: BFS and CC (each on a view of the
        # graph, results read back on their own streams) beside PageRank
        vb, vc = g2.g2_graph_view(dg), g2.g2_graph_view(dg)
        fb, fc = workers.submit(bfs_job, vb), workers.submit(cc_job, vc)
        g2.g2_pagerank(dg, DAMPING, PR_ITERS, rank_t)
        h_rank.copy_(rank_t, non_blocking=True)
        main.synchronize()
        fb.result()
        fc.result()
        vb.free()
        vc.free()
        dg.free()

    k = max(3, args.steps)  # as many steps as the device-timed loop
    compute(load())  # warm-up
    # one after another
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        compute(load())
    serial_ms = (time.perf_counter() - t0) * 1e3 / 2
    # pipelined: step k+1 uploads while step k computes.  The k steps are
    # timed three times over and the median run reported (all three in
    # `repeats_ms_per_step`): a run sometimes meets a host-side stall of a
    # few milliseconds that the other two do not.
    ex = ThreadPoolExecutor(1)

    def pipelined():
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        t0 = time.perf_counter()
        fut = ex.submit(load)
        for i in range(k):
            dg = fut.result()
            if i + 1 < k:
                fut = ex.submit(load)
            compute(dg)
        torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        wall_ms = (time.perf_counter() - t0) * 1e3 / k
        return max(e0.elapsed_time(e1) / k, wall_ms)

    runs = [pipelined() for _ in range(3)]
    ex.shutdown()
    workers.shutdown()
    ms = float(np.median(runs))
    return {"value": round(edges_per_step / (ms * 1e-3) / 1e9, 2), "unit": "GTEPS",
            "ms_per_step": round(ms, 3), "steps": k, "pipelined": True,
            "repeats_ms_per_step": [round(x, 3) for x in runs],
            "serial_ms_per_step": round(serial_ms, 3),
            "h2d_bytes_per_step": 4 * (n + 1) + 4 * m, "d2h_bytes_per_step": 16 * n}


def run_extras(g2, G22, dg22, src22, sb, sc):
    """The rest of the workloads the metric is quoted on, each timed with CUDA
    events after a warm-up call (bounded to well under a minute in all):

    * RMAT-22 BFS (tuned, with parent) and CC (tuned): arcs examined from a
      separate counting pass, algorithmic bytes (BFS 4 per examined arc + 12 n;
      CC 4 per examined arc + 8 n) over the measured time against the
      measured HBM peak;
    * RMAT-14 BFS, the plain single-query path;
    * the 4096 x 4096 road grid: BFS and delta-stepping SSSP (delta 1024 and
      16384), fused persistent loop against plain per-round launches, and the
      asynchronous variants (no barrier inside a bucket);
    * RMAT-21 batched: 64-source BFS in one traversal against 64 single-source
      calls (tuned schedule and the fixed TWC PUSH schedule), 32-source SSSP
      against 32 single calls, BC from 16 sources;
    * serving over the resident pool (RMAT 16-22, grids 512^2-4096^2):
      continuous batching against one launch per query, at 2,000 requests/s
      (more than one GPU serves: latency is mostly queueing) and at 500/s."""
    import torch
    from paper_2012_07990_gb300 import graphgen as gg
    from paper_2012_07990_gb300 import serve
    t_start = time.time()
    peak, _ = read_peaks()
    out = {}

    def dev(k, dtype=torch.int32):
        return torch.empty(k, dtype=dtype, device="cuda")

    def reached_arcs(G, vals, unreached):
        return int(G.degrees()[vals.cpu().numpy() != unreached].sum())

    def bfs_cc_rows(G, dg, src, with_cc):
        n = G.n
        depth, parent, label = dev(n), dev(n), dev(n)
        # alone, BFS runs the library's tuned schedule (NULL: the hybrid
        # fused into one launch); the step's per-level form beside it
        tb = bfs_schedule(g2)
        g2.g2_set_count_arcs(True)
        g2.g2_bfs(dg, src, depth, parent, tb)
        bfs_arcs = g2.g2_last_stats()["arcs_examined"]
        cc_arcs = 0
        if with_cc:
            g2.g2_cc(dg, label, sc)
            cc_arcs = g2.g2_last_stats()["arcs_examined"]
        g2.g2_set_count_arcs(False)
        ms = _timed(lambda: g2.g2_bfs(dg, src, depth, parent, tb), reps=7)
        ms_np = _timed(lambda: g2.g2_bfs(dg, src, depth, None, tb), reps=7)
        ms_pl = _timed(lambda: g2.g2_bfs(dg, src, depth, parent, sb), reps=7)
        reached = reached_arcs(G, depth, -1)
        b = 4 * bfs_arcs + 12 * n
        rows = {"bfs": {"ms": round(ms, 4), "gteps": round(reached / ms / 1e6, 2), "reached_arcs": reached,
                        "arcs_examined": int(bfs_arcs), "bytes": int(b),
                        "achieved_gbs": round(b / ms / 1e6, 1), "frac": round(b / ms / 1e6 / peak, 4),
                        "ms_without_parent": round(ms_np, 4),
                        "per_level_ms": round(ms_pl, 4)}}
        if with_cc:
            ms = _timed(lambda: g2.g2_cc(dg, label, sc), reps=7)
            b = 4 * cc_arcs + 8 * n
            rows["cc"] = {"ms": round(ms, 4), "gteps_nominal": round(G.m / ms / 1e6, 2),
                          "arcs_examined": int(cc_arcs), "bytes": int(b),
                          "achieved_gbs": round(b / ms / 1e6, 1), "frac": round(b / ms / 1e6 / peak, 4),
                          "note": "gteps_nominal = all arcs / time; the tuned CC links only the arcs examined"}
        return rows

    # RMAT-22 BFS and CC
    r = bfs_cc_rows(G22, dg22, src22, True)
    out["rmat22_bfs"], out["rmat22_cc"] = r["bfs"], r["cc"]
    # RMAT-14, plain single-query BFS
    G14 = gg.rmat(14, seed=1)
    dg14 = g2.load_graph(G14)
    out["rmat14_bfs"] = bfs_cc_rows(G14, dg14, G14.max_degree_vertex(), False)["bfs"]
    dg14.free()

    # road grid 4096^2, fused against plain
    Gg = gg.road_grid(4096, seed=1)
    wg = gg.pair_weights(Gg, 1000, seed=1)
    dgg = g2.load_graph(Gg, wg)
    depth, dist = dev(Gg.n), dev(Gg.n)
    strict = g2.schedule("STRICT")
    grid = {}
    for name, s_, reps in (("fused", None, 3), ("plain", strict, 2)):
        ms = _timed(lambda: g2.g2_bfs(dgg, 0, depth, None, s_), reps=reps)
        st = g2.g2_last_stats()
        grid[f"bfs_{name}"] = {"ms": round(ms, 3), "levels": st["iterations"], "launches": st["launches"],
                               "gteps": round(reached_arcs(Gg, depth, -1) / ms / 1e6, 3)}
    for delta, names in ((1024, (("fused", None, 2), ("plain", strict, 1))), (16384, (("fused", None, 2),))):
        for name, s_, reps in names:
            ms = _timed(lambda: g2.g2_sssp_delta(dgg, 0, delta, dist, s_), reps=reps)
            st = g2.g2_last_stats()
            grid[f"sssp_d{delta}_{name}"] = {
                "ms": round(ms, 3), "rounds": st["iterations"], "launches": st["launches"],
                "gteps": round(reached_arcs(Gg, dist, 2**31 - 1) / ms / 1e6, 3)}
    for name, fn in (("sssp_d8192_async", lambda: g2.g2_sssp_async(dgg, 0, 8192, dist)),
                     ("bfs_async_d64", lambda: g2.g2_bfs_async(dgg, 0, 64, depth, None))):
        ms = _timed(fn, reps=2)
        st = g2.g2_last_stats()
        out_arr = dist if name.startswith("sssp") else depth
        grid[name] = {"ms": round(ms, 3), "items": st["iterations"], "barriers": st["barriers"],
                      "gteps": round(reached_arcs(Gg, out_arr, 2**31 - 1 if name.startswith("sssp") else -1)
                                     / ms / 1e6, 3)}
    grid["fused_vs_plain"] = {"bfs": round(grid["bfs_plain"]["ms"] / grid["bfs_fused"]["ms"], 2),
                              "sssp_d1024": round(grid["sssp_d1024_plain"]["ms"] / grid["sssp_d1024_fused"]["ms"], 2)}
    out["grid4096"] = grid
    dgg.free()

    # RMAT-21 batched
    G21 = gg.rmat(21, seed=1)
    w21 = gg.pair_weights(G21, 255, seed=1)
    dg21 = g2.load_graph(G21, w21)
    srcs = gg.random_sources(G21, 64, seed=1)
    deg = G21.degrees()
    b = {}
    d64 = dev(64 * G21.n)
    ms = _timed(lambda: g2.g2_bfs_batch(dg21, srcs, d64, None), reps=3)
    d = d64.cpu().numpy().reshape(64, G21.n)
    edges = int(sum(deg[d[i] >= 0].sum() for i in range(64)))
    b["bfs64_batched"] = {"ms": round(ms, 3), "gteps": round(edges / ms / 1e6, 2)}
    one = dev(G21.n)
    for name, s_ in (("tuned", None), ("twc_push", g2.schedule("TWC"))):
        def loop(s_=s_):
            for v in srcs:
                g2.g2_bfs(dg21, int(v), one, None, s_)
        ms1 = _timed(loop, reps=1)
        b[f"bfs64_serial_{name}"] = {"ms": round(ms1, 3), "gteps": round(edges / ms1 / 1e6, 2)}
    d32 = dev(32 * G21.n)
    ms = _timed(lambda: g2.g2_sssp_batch(dg21, srcs[:32], 64, d32, None), reps=2)
    dd = d32.cpu().numpy().reshape(32, G21.n)
    edges32 = int(sum(deg[dd[i] < 2**31 - 1].sum() for i in range(32)))
    b["sssp32_batched"] = {"ms": round(ms, 3), "gteps": round(edges32 / ms / 1e6, 2)}

    def loop_sssp():
        for v in srcs[:32]:
            g2.g2_sssp_delta(dg21, int(v), 64, one, None)
    ms1 = _timed(loop_sssp, reps=1)
    b["sssp32_serial"] = {"ms": round(ms1, 3), "gteps": round(edges32 / ms1 / 1e6, 2)}
    bc = dev(G21.n, torch.float64)
    ms = _timed(lambda: g2.g2_bc(dg21, srcs[:16], bc, None), reps=1)
    edges16 = int(sum(deg[d[i] >= 0].sum() for i in range(16)))
    b["bc16"] = {"ms": round(ms, 3), "gteps": round(2 * edges16 / ms / 1e6, 2),
                 "note": "forward and backward sweeps counted"}
    b["speedup"] = {"bfs64_vs_serial_tuned": round(b["bfs64_serial_tuned"]["ms"] / b["bfs64_batched"]["ms"], 2),
                    "bfs64_vs_serial_twc_push": round(b["bfs64_serial_twc_push"]["ms"] / b["bfs64_batched"]["ms"], 2),
                    "sssp32_vs_serial": round(b["sssp32_serial"]["ms"] / b["sssp32_batched"]["ms"], 2)}
    out["rmat21_batched"] = b
    dg21.free()
    del d64, d32

    # serving over the full pool (RMAT-22 and the 4096^2 grid reuse the
    # graphs generated above)
    cached = {"rmat22": G22, "grid4096": Gg}
    specs = serve.default_pool_specs()
    for sp in specs:
        if sp.name in cached:
            sp.make = (lambda G=cached[sp.name]: G)
    pool = serve.GraphPool(g2, specs)
    sv = {}
    ex4 = serve.GpuExecutor(g2, pool, slots=4)
    ex1 = serve.GpuExecutor(g2, pool, slots=1)
    for rate, duration in ((2000.0, 0.25), (500.0, 1.0)):
        trace = serve.make_trace(pool, rate=rate, duration=duration, seed=1)
        srv = serve.Server(ex4, pool, policy="hrrn")
        srv.run(trace[: min(128, len(trace))])  # warm views, workspaces and the cost model
        cb = srv.run(trace).summary()
        serial = serve.Server(ex1, pool, max_batch=dict(bfs=1, sssp=1, bc=1), policy="fifo").run(trace).summary()
        sv[f"rate{int(rate)}"] = {"requests": len(trace), "duration_s": duration,
                                  "continuous_batching": cb, "serial_plain": serial}
    out["serving"] = sv
    for ex in (ex4, ex1):
        for views in ex.views:
            for v in views.values():
                v.free()
    for g in pool.graphs.values():
        g.handle.free()
    out["seconds"] = round(time.time() - t_start, 1)
    return out


def read_profile_record(kernel: str):
    """The committed ncu record of `kernel`, if it was taken on the current
    source of that kernel (else None)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        src = os.path.join(ROOT, "paper_2012_07990_gb300", "csrc", d["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return d if h == d["source_sha256_16"] else None
    except Exception:
        return None


def read_traffic(kernel: str, G):
    """Per-launch DRAM bytes of `kernel` from the committed ncu record, scaled
    to the arcs of G (traffic grows with the arcs swept), else None."""
    d = read_profile_record(kernel)
    if d is None:
        return None
    return int(d["dram_bytes_per_launch"] / d["arcs_per_launch"] * G.m)


# ---------------------------------------------------------------- oracle
def oracle_step(G, src, pr_rounds):
    import oracle
    t0 = time.perf_counter()
    depth, _ = oracle.bfs_graph(G, src, want_parent=False)
    t1 = time.perf_counter()
    oracle.cc_graph(G)
    t2 = time.perf_counter()
    oracle.pagerank_graph(G, DAMPING, pr_rounds)
    t3 = time.perf_counter()
    return depth, (t1 - t0, t2 - t1, t3 - t2)


def cpu_baseline(G, src, budget_s=30.0):
    """The oracle as it stands, single thread, on a bounded sample of the same
    workload: one BFS, one CC and the PageRank rounds that fit the budget."""
    depth, (tb, tc, tp1) = oracle_step(G, src, 1)
    m_bfs = int(G.degrees()[depth >= 0].sum())
    edges = m_bfs + G.m + G.m
    secs = tb + tc + tp1
    return {"value": round(edges / secs / 1e9, 4), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"rmat{int(np.log2(G.n))}: 1 BFS + 1 CC + 1 PageRank round "
                      f"(of 20) = {edges} edges in {secs:.2f} s",
            "seconds": {"bfs": round(tb, 3), "cc": round(tc, 3), "pr_round": round(tp1, 3)},
            "host_cpus": os.cpu_count()}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    G = make_graph(args.scale)
    src = G.max_degree_vertex()
    for _ in range(args.warmup):
        oracle_step(G, src, 1)
    times = []
    t0 = time.perf_counter()
    depth = None
    for _ in range(args.steps):
        depth, ts = oracle_step(G, src, 1)
        times.append(sum(ts))
    total = time.perf_counter() - t0
    m_bfs = int(G.degrees()[depth >= 0].sum())
    edges = m_bfs + 2 * G.m
    value = edges * args.steps / total / 1e9
    line = {
        "impl": "reference",
        "metric": "GTEPS (direction-optimising BFS + CC + PageRank x20 on RMAT-22), % HBM roofline",
        "value": round(value, 4), "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64",
        "data": "synthetic RMAT (seeded, counter-based generator)",
        "config": {"workload": f"rmat{args.scale}_bfs_cc_pr", "n": G.n, "m": G.m,
                   "step_sample": "1 BFS + 1 CC + 1 PageRank round (of 20)"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": "each step: BFS + CC + one PageRank round on the full graph"},
        "e2e": {"value": round(value, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _timed(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def run_grid_workload(args):
    """Road-like 4096 x 4096 grid (10% of lattice edges deleted, 1% local
    shortcuts, weights U[1, 1000], seed 1): delta-stepping SSSP plain vs fused
    across deltas, BFS plain vs fused, single-source BC fused, from vertex 0
    (a corner).  The fused WM loops run small levels in one thread-block
    cluster; `*_grid_only` is the same schedule with the one-cluster loops
    switched off (G2_FUSED_CLUSTER=0), the grid-wide kernel throughout."""
    import torch
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2
    from paper_2012_07990_gb300 import graphgen as gg
    W = args.grid
    G = gg.road_grid(W, seed=1)
    w = gg.pair_weights(G, 1000, seed=1)
    dg = g2.load_graph(G, w)
    dist = torch.empty(G.n, dtype=torch.int32, device="cuda")
    depth = torch.empty(G.n, dtype=torch.int32, device="cuda")
    res = {"sssp": [], "bfs": []}
    deg = G.degrees()
    wm = g2.schedule("WM", kernel_fusion=True)

    def grid_only(fn):
        os.environ["G2_FUSED_CLUSTER"] = "0"
        try:
            return fn()
        finally:
            os.environ.pop("G2_FUSED_CLUSTER", None)

    for delta in (16, 64, 256, 1024, 4096, 16384):
        row = {"delta": delta}
        for name, s in (("plain_strict", g2.schedule("STRICT")),
                        ("fused_vertex", g2.schedule("VERTEX_BASED", kernel_fusion=True)),
                        ("fused_wm", wm), ("fused_wm_grid_only", wm)):
            run = lambda: _timed(lambda: g2.g2_sssp_delta(dg, 0, delta, dist, s), reps=2)
            ms = grid_only(run) if name.endswith("grid_only") else run()
            st = g2.g2_last_stats()
            row[name + "_ms"] = round(ms, 3)
            row[name + "_rounds"] = st["iterations"]
        reached = int(deg[dist.cpu().numpy() < 2**31 - 1].sum())
        row["gteps_best"] = round(reached / min(v for k, v in row.items() if k.endswith("_ms")) / 1e6, 3)
        res["sssp"].append(row)
    # asynchronous delta-stepping (no barrier inside a bucket) beside them
    res["sssp_async"] = []
    for delta in (0, 1024, 4096, 8192, 16384, 65536):
        ms = _timed(lambda: g2.g2_sssp_async(dg, 0, delta, dist), reps=2)
        st = g2.g2_last_stats()
        res["sssp_async"].append({"delta": delta, "ms": round(ms, 3), "items": st["iterations"],
                                  "barriers": st["barriers"]})
    res["bfs_async"] = []
    for delta in (1, 16, 64, 256):
        ms = _timed(lambda: g2.g2_bfs_async(dg, 0, delta, depth, None), reps=2)
        st = g2.g2_last_stats()
        res["bfs_async"].append({"delta": delta, "ms": round(ms, 3), "items": st["iterations"],
                                 "barriers": st["barriers"]})
    for name, s in (("null_schedule", None), ("plain_strict", g2.schedule("STRICT")),
                    ("fused_vertex", g2.schedule("VERTEX_BASED", kernel_fusion=True)),
                    ("fused_wm", wm), ("fused_wm_grid_only", wm)):
        run = lambda: _timed(lambda: g2.g2_bfs(dg, 0, depth, None, s))
        ms = grid_only(run) if name.endswith("grid_only") else run()
        st = g2.g2_last_stats()
        reached = int(deg[depth.cpu().numpy() >= 0].sum())
        res["bfs"].append({"schedule": name, "ms": round(ms, 3), "levels": st["iterations"],
                           "launches": st["launches"], "gteps": round(reached / ms / 1e6, 3)})
    res["bc"] = []
    bc = torch.empty(G.n, dtype=torch.float64, device="cuda")
    reached = int(deg[depth.cpu().numpy() >= 0].sum())  # BFS from vertex 0 above
    for name in ("fused_wm", "fused_wm_grid_only"):
        run = lambda: _timed(lambda: g2.g2_bc(dg, [0], bc, wm), reps=2)
        ms = grid_only(run) if name.endswith("grid_only") else run()
        st = g2.g2_last_stats()
        res["bc"].append({"schedule": name, "ms": round(ms, 3), "levels": st["iterations"],
                          "launches": st["launches"], "gteps": round(2 * reached / ms / 1e6, 3)})
    print(json.dumps({"workload": f"grid{W}x{W}_sssp_bfs", "n": G.n, "m": G.m, **res}))


def run_tune_workload(args):
    """Autotuner: for a power-law graph (RMAT-18) and a road-like grid
    (1024^2), BFS and delta-stepping SSSP (and PageRank on RMAT-18) are
    tuned from cold (random sampling + successive halving); the tuned
    schedule is compared with the library's default schedule and with the
    paper's default schedule (all Table II fields at their defaults).  Then
    a sibling graph of each family (RMAT-19 seed 2, grid 1200^2 seed 2) is
    tuned once from cold and once warm-started from the first graph's cache
    entry with a sixth of the random samples.  For BFS the whole space is
    also searched exhaustively (every simple schedule of both directions,
    then hybrids of the fastest), on both graphs."""
    import tempfile
    import torch
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import autotune as at
    from paper_2012_07990_gb300 import g2
    from paper_2012_07990_gb300 import graphgen as gg

    fams = {"powerlaw": (lambda: gg.rmat(18, seed=1), lambda: gg.rmat(19, seed=2), 255),
            "road": (lambda: gg.road_grid(1024, seed=1), lambda: gg.road_grid(1200, seed=2), 1000)}
    algos = {"powerlaw": ("bfs", "sssp", "pr"), "road": ("bfs", "sssp")}
    paper_default = {"criteria": 0, "threshold": 0.0, "s1": at._simple(), "s2": at._simple()}
    cache = at.TuneCache(os.path.join(tempfile.mkdtemp(), "tune.json"))
    out = {"workload": "autotune", "graphs": {}}

    def evaluate(G, w, algo):
        dg = g2.load_graph(G, w)
        src = G.max_degree_vertex() if G.name.startswith("rmat") else 0
        if algo == "sssp":
            base = at.gpu_evaluator(g2, dg, "sssp", src=src)

            def cost(d):
                # the paper's default schedule leaves delta at its default, 1
                if not d.get("tuned_default") and d["s1"]["delta"] == 0:
                    d = json.loads(json.dumps(d))
                    d["s1"]["delta"] = d["s2"]["delta"] = 1
                return base(d)
            return dg, cost
        return dg, at.gpu_evaluator(g2, dg, algo, src=src)

    for fam, (mk1, mk2, wmax) in fams.items():
        G1, G2 = mk1(), mk2()
        w1, w2 = gg.pair_weights(G1, wmax, seed=1), gg.pair_weights(G2, wmax, seed=2)
        f1, f2 = at.graph_features(G1.n, G1.rowptr), at.graph_features(G2.n, G2.rowptr)
        fp1 = at.graph_fingerprint(G1.n, G1.rowptr, G1.col)
        rows = {}
        for algo in algos[fam]:
            dg, cost = evaluate(G1, w1, algo)
            t0 = time.perf_counter()
            res = at.tune(algo, cost, n_samples=24, seed=1)
            tune_s = time.perf_counter() - t0
            cache.put(fp1, algo, res, f1)
            best = min(cost(res.best) for _ in range(3))
            lib = min(cost({"tuned_default": True}) if algo in ("cc", "pr") else
                      _lib_default_ms(g2, dg, G1, algo) for _ in range(3))
            pdef = None
            # delta = 1 on a road grid means ~10^6 buckets with a host round
            # trip each: not timed
            if not (algo == "sssp" and fam == "road"):
                try:
                    pdef = min(cost(paper_default) for _ in range(2))
                except Exception:  # unsupported for this algorithm
                    pdef = None
            row = {"tuned_ms": round(best, 3), "library_default_ms": round(lib, 3),
                   "paper_default_ms": None if pdef is None else round(pdef, 3),
                   "evaluations": res.evaluated, "tune_s": round(tune_s, 2),
                   "best": res.best}
            dg.free()
            # sibling graph: cold search vs warm start with 4 random samples
            dg2, cost2 = evaluate(G2, w2, algo)
            cold = at.tune(algo, cost2, n_samples=24, seed=5)
            warm = at.tune(algo, cost2, n_samples=4, seed=5, warm=cache.warm_start(f2, algo))
            row["sibling"] = {"cold_ms": round(min(cost2(cold.best) for _ in range(3)), 3),
                              "cold_evaluations": cold.evaluated,
                              "warm_ms": round(min(cost2(warm.best) for _ in range(3)), 3),
                              "warm_evaluations": warm.evaluated}
            if algo == "bfs":
                # the whole space (Table I): every simple schedule of both
                # directions, then hybrids of the fastest ones; how far the
                # random + halving search and the warm start land from it
                ex2 = at.exhaustive(cost2, reps=2)
                row["sibling"]["exhaustive_ms"] = round(min(cost2(ex2.best) for _ in range(3)), 3)
                row["sibling"]["exhaustive_evaluations"] = ex2.evaluated
                row["sibling"]["exhaustive_rejected"] = ex2.rejected
            dg2.free()
            if algo == "bfs":
                dg, cost = evaluate(G1, w1, algo)
                t0 = time.perf_counter()
                ex = at.exhaustive(cost, reps=2)
                row["exhaustive"] = {
                    "ms": round(min(cost(ex.best) for _ in range(3)), 3), "best": ex.best,
                    "evaluations": ex.evaluated, "rejected": ex.rejected,
                    "seconds": round(time.perf_counter() - t0, 1),
                    "push_only_ms": round(ex.per_direction[0]["ms"], 3),
                    "pull_only_ms": round(ex.per_direction[1]["ms"], 3),
                    "tuned_over_exhaustive": round(best / min(cost(ex.best) for _ in range(3)), 3)}
                dg.free()
            rows[algo] = row
        out["graphs"][f"{fam}:{G1.name}"] = rows
    print(json.dumps(out))


def _lib_default_ms(g2, dg, G, algo):
    """The library's tuned default schedule (NULL) for BFS / SSSP, timed."""
    import torch
    out = torch.empty(G.n, dtype=torch.int32, device="cuda")
    src = G.max_degree_vertex() if G.name.startswith("rmat") else 0
    if algo == "bfs":
        fn = lambda: g2.g2_bfs(dg, src, out, None, None)
    else:
        fn = lambda: g2.g2_sssp_delta(dg, src, 64 if G.name.startswith("rmat") else 4096, out, None)
    return _timed(fn, reps=1)


def run_gather_workload(args):
    """The floor under the PageRank arc sweep: plain gather passes over
    RMAT-22's column ids (g2_diag_gather) in CSC order, in the sweep's
    renumbered order (only the arcs whose share is not in the shared-memory
    cache), in uniformly random order, and the column stream alone, next to
    the sweep's own time per round."""
    import torch
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2
    G = make_graph(args.scale)
    n, m = G.n, G.m
    H = 16384
    deg = G.degrees()
    order = np.lexsort((np.arange(n), -deg))  # degree descending, ties to the lower id
    hot = np.zeros(n, bool)
    hot[order[:H]] = True
    slot = (H + np.arange(n)).astype(np.int64)
    slot[hot] = np.cumsum(hot)[hot] - 1
    ren = slot[G.col]
    cold = ren[ren >= H]
    rng = np.random.default_rng(1)
    variants = {"csc_order": G.col, "renumbered_cold_arcs": cold.astype(np.int32),
                "uniform_random": rng.integers(0, n, m, dtype=np.int32)}
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    grid = sm * 8  # 2,048 threads per SM, as the sweep
    x = torch.rand(n + H, device="cuda")
    out = torch.empty(grid * 256, device="cuda")
    res = {}

    def best_pass(d, xx, mode, reps=5):
        return min(g2.g2_diag_gather(d, xx, mode, out, grid) for _ in range(reps + 1))

    for name, idx in variants.items():
        d = torch.from_numpy(np.ascontiguousarray(idx)).cuda()
        ms = best_pass(d, x, 0)
        res[name] = {"loads": int(d.numel()), "us": round(ms * 1e3, 1),
                     "gloads_per_s": round(d.numel() / ms / 1e6, 1)}
    d = torch.from_numpy(G.col).cuda()
    ms = best_pass(d, None, 1)
    res["column_stream_only"] = {"bytes": 4 * m, "us": round(ms * 1e3, 1),
                                 "gb_per_s": round(4 * m / ms / 1e6, 1)}
    dg = g2.load_graph(G)
    rank = torch.empty(n, dtype=torch.float32, device="cuda")
    g2.g2_pagerank(dg, DAMPING, 2, rank)
    g2.g2_set_kernel_timing(True)
    g2.g2_kernel_time("pr_round", reset=True)
    g2.g2_pagerank(dg, DAMPING, PR_ITERS, rank)
    torch.cuda.synchronize()
    kt, kl = g2.g2_kernel_time("pr_round", reset=True)
    g2.g2_set_kernel_timing(False)
    sweep_us = kt / kl * 1e3
    print(json.dumps({"workload": f"gather_floor_rmat{args.scale}", "n": n, "m": m, "grid": grid,
                      "hot_slots": H, **res, "pr_sweep_us": round(sweep_us, 1),
                      "sweep_over_csc_order_gather": round(sweep_us / res["csc_order"]["us"], 3),
                      "sweep_over_cold_gather_plus_stream": round(
                          sweep_us / (res["renumbered_cold_arcs"]["us"] +
                                      res["column_stream_only"]["us"]), 3)}))


def run_batched_workload(args):
    """RMAT scale 21 (ef 16, symmetric): 64-source BFS in one traversal vs 64
    single-source BFS calls (tuned and fixed TWC PUSH); 32-source SSSP (weights
    U[1, 255]) vs 32 single calls; BC from 16 sources."""
    import torch
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2
    from paper_2012_07990_gb300 import graphgen as gg
    G = gg.rmat(args.batch_scale, seed=1)
    w = gg.pair_weights(G, 255, seed=1)
    dg = g2.load_graph(G, w)
    srcs = gg.random_sources(G, 64, seed=1)
    deg = G.degrees()
    out = {}
    depth64 = torch.empty(64 * G.n, dtype=torch.int32, device="cuda")
    ms = _timed(lambda: g2.g2_bfs_batch(dg, srcs, depth64, None))
    d = depth64.cpu().numpy().reshape(64, G.n)
    edges = int(sum(deg[d[i] >= 0].sum() for i in range(64)))
    out["msbfs64"] = {"ms": round(ms, 3), "gteps": round(edges / ms / 1e6, 2)}
    one = torch.empty(G.n, dtype=torch.int32, device="cuda")
    for name, s in (("tuned", None), ("twc_push", g2.schedule("TWC"))):
        def loop():
            for sv in srcs:
                g2.g2_bfs(dg, int(sv), one, None, s)
        ms1 = _timed(loop, reps=2)
        out[f"bfs64_serial_{name}"] = {"ms": round(ms1, 3), "gteps": round(edges / ms1 / 1e6, 2)}
    dist32 = torch.empty(32 * G.n, dtype=torch.int32, device="cuda")
    ms = _timed(lambda: g2.g2_sssp_batch(dg, srcs[:32], 64, dist32, None))
    dd = dist32.cpu().numpy().reshape(32, G.n)
    edges32 = int(sum(deg[dd[i] < 2**31 - 1].sum() for i in range(32)))
    out["mssssp32"] = {"ms": round(ms, 3), "gteps": round(edges32 / ms / 1e6, 2)}

    def loop_sssp():
        for sv in srcs[:32]:
            g2.g2_sssp_delta(dg, int(sv), 64, one, None)
    ms1 = _timed(loop_sssp, reps=2)
    out["sssp32_serial"] = {"ms": round(ms1, 3), "gteps": round(edges32 / ms1 / 1e6, 2)}
    bc = torch.empty(G.n, dtype=torch.float64, device="cuda")
    ms = _timed(lambda: g2.g2_bc(dg, srcs[:16], bc, None), reps=2)
    edges16 = int(sum(deg[d[i] >= 0].sum() for i in range(16)))
    out["bc16"] = {"ms": round(ms, 3), "gteps": round(2 * edges16 / ms / 1e6, 2),
                   "note": "forward + backward sweeps counted"}
    print(json.dumps({"workload": f"rmat{args.batch_scale}_batched", "n": G.n, "m": G.m, **out}))


def run_lb_workload(args):
    """The load-balancing comparison of the paper's Table VIII: BFS PUSH-only
    (kernel fusion off) with ETWC, TWC and CM (and STRICT, WM and
    VERTEX_BASED beside them) on RMAT-22 from its hub and on the 4096 x 4096
    road grid from vertex 0; plus one PUSH round from RMAT-22's hub alone
    (163K arcs in one vertex), the case where a load balancer that keeps a
    vertex on one CTA serialises."""
    import torch
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2
    from paper_2012_07990_gb300 import graphgen as gg
    lbs = ("ETWC", "TWC", "CM", "STRICT", "WM", "VERTEX_BASED")
    out = {"workload": "lb_push_bfs"}
    G = make_graph(22)
    Gg = gg.road_grid(4096, seed=1)
    for name, graph, src in (("rmat22", G, G.max_degree_vertex()), ("grid4096", Gg, 0)):
        dg = g2.load_graph(graph)
        depth = torch.empty(graph.n, dtype=torch.int32, device="cuda")
        row = {}
        for lb in lbs:
            ms = _timed(lambda: g2.g2_bfs(dg, src, depth, None, g2.schedule(lb)), reps=3 if name == "rmat22" else 1)
            row[lb] = {"ms": round(ms, 3), "levels": g2.g2_last_stats()["iterations"]}
        if name == "rmat22":
            hub = np.array([src], np.int32)
            fin = g2.Frontier(dg, g2.G2_FRONTIER_SPARSE)
            fin.set(hub)
            first = {}
            for lb in lbs:
                ts = []
                for rep in range(6):
                    depth.fill_(-1)
                    depth[src] = 0
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    g2.g2_edgeset_apply(dg, g2.G2_OP_BFS, fin, depth, None, g2.schedule(lb))
                    e1.record()
                    torch.cuda.synchronize()
                    if rep:
                        ts.append(e0.elapsed_time(e1))
                first[lb] = round(float(np.median(ts)), 4)
            row["first_round_from_hub_ms"] = first
        out[name] = row
        dg.free()
    print(json.dumps(out))


def run_serve_workload(args):
    """Serving: Poisson stream (BFS 60% / SSSP 30% / single-source BC 10%) over
    a resident pool (full: RMAT 16/18/20/22 + grids 512^2..4096^2; small: RMAT
    16/18/20 + grids 512^2, 1024^2), continuous batching on 4 slots (queue
    choice by response ratio with learned batch costs, and oldest-first) vs
    the same trace served serially with one launch per query."""
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2
    from paper_2012_07990_gb300 import serve
    if args.serve_pool == "full":
        specs = serve.default_pool_specs()
    else:
        specs = serve.default_pool_specs(scales=(16, 18, 20), grids=(512, 1024))
    t = time.time()
    pool = serve.GraphPool(g2, specs)
    load_s = time.time() - t
    ex = serve.GpuExecutor(g2, pool, slots=4)
    ex1 = serve.GpuExecutor(g2, pool, slots=1)
    if args.serve_rates:
        # latency against offered load: the same number of requests at each
        # rate, continuous batching (response ratio) against serial launches
        curve = []
        for rate in (float(r) for r in args.serve_rates.split(",")):
            trace = serve.make_trace(pool, rate=rate, duration=args.serve_requests / rate, seed=1)
            srv = serve.Server(ex, pool, policy="hrrn")
            srv.run(trace[: min(128, len(trace))])  # warm views, workspaces and the cost model
            cb = srv.run(trace).summary()
            serial = serve.Server(ex1, pool, max_batch=dict(bfs=1, sssp=1, bc=1), policy="fifo").run(trace)
            curve.append({"rate_per_s": rate, "requests": len(trace), "continuous_batching": cb,
                          "serial_plain": serial.summary()})
        print(json.dumps({"workload": f"serve_curve_{args.serve_pool}", "graphs": [s.name for s in specs],
                          "pool_load_s": round(load_s, 2), "curve": curve}))
        return
    trace = serve.make_trace(pool, rate=args.serve_rate, duration=args.serve_duration, seed=1)
    res = {}
    for policy in ("hrrn", "fifo"):
        srv = serve.Server(ex, pool, policy=policy)
        srv.run(trace[: min(256, len(trace))])  # warm views, workspaces and the cost model
        res[policy] = srv.run(trace).summary()
    serial = serve.Server(ex1, pool, max_batch=dict(bfs=1, sssp=1, bc=1), policy="fifo").run(trace)
    print(json.dumps({"workload": f"serve_{args.serve_pool}", "graphs": [s.name for s in specs],
                      "pool_load_s": round(load_s, 2), "rate_per_s": args.serve_rate,
                      "duration_s": args.serve_duration, "requests": len(trace),
                      "continuous_batching_4_slots": res["hrrn"],
                      "continuous_batching_4_slots_fifo": res["fifo"],
                      "serial_plain": serial.summary()}))


def run_profile_case(args):
    """A short run of one piece of the library for profilers (one launch of
    each kernel of interest, a few hundred MB on the device at most), so that a
    capture names a committed command:

    * pr / bfs / cc: RMAT at --scale, the algorithm --steps times with the
      tuned schedule (BFS: the direction-optimising hybrid fused into one
      launch);
    * bfs_levels: the same BFS hybrid as per-level launches (the bench
      step's form);
    * road_fused: the --grid x --grid road grid (weights U[1, 1000]), one fused
      WM BFS from vertex 0 (no parent array) and one fused WM delta-stepping
      SSSP from vertex 0 with delta 1024 -- the one-cluster loops;
    * bc_rmat: RMAT at --scale, BC from its two highest-degree vertices with
      the NULL schedule -- the level passes on a power-law graph;
    * batch_grid: the --grid x --grid road grid, the fused multi-source loops
      (64-source BFS, 32-source SSSP with delta 4096), the split into
      single-source queries switched off;
    * pr_layout: RMAT at --scale, loaded --steps times, each load building
      PageRank's source-blocked layout (a PageRank call with no rounds)."""
    import torch
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2
    from paper_2012_07990_gb300 import graphgen as gg
    case = args.profile_case
    if case == "road_fused":
        G = gg.road_grid(args.grid, seed=1)
        w = gg.pair_weights(G, 1000, seed=1)
        dg = g2.load_graph(G, w)
        out = torch.empty(G.n, dtype=torch.int32, device="cuda")
        s = g2.schedule("WM", kernel_fusion=True)
        g2.g2_bfs(dg, 0, out, None, s)
        bfs = g2.g2_last_stats()
        g2.g2_sssp_delta(dg, 0, 1024, out, s)
        sssp = g2.g2_last_stats()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": case, "grid": args.grid, "bfs_levels": bfs["iterations"],
                          "bfs_launches": bfs["launches"], "sssp_rounds": sssp["iterations"],
                          "sssp_launches": sssp["launches"]}))
        return
    if case == "batch_grid":
        # the fused multi-source loops on a road grid (the split into
        # single-source queries switched off): 64-source BFS, then 32-source
        # delta-stepping SSSP with delta 4096
        os.environ["G2_BATCH_SPLIT_WORKERS"] = "0"
        G = gg.road_grid(args.grid, seed=1)
        w = gg.pair_weights(G, 1000, seed=1)
        dg = g2.load_graph(G, w)
        srcs = gg.random_sources(G, 64, seed=1)
        out = torch.empty(64 * G.n, dtype=torch.int32, device="cuda")
        g2.g2_bfs_batch(dg, srcs, out, None)
        bfs = g2.g2_last_stats()
        g2.g2_sssp_batch(dg, srcs[:32], 4096, out, None)
        sssp = g2.g2_last_stats()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": case, "grid": args.grid, "bfs_levels": bfs["iterations"],
                          "bfs_launches": bfs["launches"], "sssp_rounds": sssp["iterations"],
                          "sssp_launches": sssp["launches"]}))
        return
    G = make_graph(args.scale)
    dg = g2.load_graph(G)
    if case == "bc_rmat":
        srcs = np.argsort(-G.degrees(), kind="stable")[:2].astype(np.int32)
        bc = torch.empty(G.n, dtype=torch.float64, device="cuda")
        g2.g2_bc(dg, srcs, bc, None)
        st = g2.g2_last_stats()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": case, "scale": args.scale, "levels": st["iterations"],
                          "launches": st["launches"]}))
        return
    if case == "pr_layout":
        dg.free()
        out = torch.empty(G.n, dtype=torch.float32, device="cuda")
        ms = []
        for _ in range(args.steps):
            dg = g2.load_graph(G)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2.g2_pagerank(dg, DAMPING, 0, out)
            torch.cuda.synchronize()
            ms.append(round((time.perf_counter() - t0) * 1e3, 3))
            dg.free()
        print(json.dumps({"profile_case": case, "scale": args.scale, "n": G.n, "m": G.m,
                          "layout_ms": ms}))
        return
    src = G.max_degree_vertex()
    out = torch.empty(G.n, dtype=torch.float32 if case == "pr" else torch.int32, device="cuda")
    for _ in range(args.steps):
        if case == "pr":
            g2.g2_pagerank(dg, DAMPING, PR_ITERS, out)
        elif case == "bfs":
            g2.g2_bfs(dg, src, out, None, None)
        elif case == "bfs_levels":
            g2.g2_bfs(dg, src, out, None, bfs_per_level_hybrid(g2))
        else:
            g2.g2_cc(dg, out, None)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": case, "scale": args.scale, "n": G.n, "m": G.m,
                      "checksum": float(out.double().sum().item())}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", choices=["pr", "bfs", "bfs_levels", "cc", "road_fused", "bc_rmat",
                                               "batch_grid", "pr_layout"],
                    default=None)
    ap.add_argument("--serve-pool", choices=["full", "small"], default="full")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-duration", type=float, default=1.0)
    ap.add_argument("--serve-rates", default=None,
                    help="comma-separated request rates: a latency-against-load curve")
    ap.add_argument("--serve-requests", type=int, default=600,
                    help="requests per rate of the curve (--serve-rates)")
    ap.add_argument("--workload", choices=["rmat22", "grid", "batched", "serve", "tune", "gather", "lb"],
                    default="rmat22",
                    help="rmat22: the default step (the benchmark's JSON line); grid and "
                         "batched: the road-grid and multi-source configurations")
    ap.add_argument("--grid", type=int, default=4096)
    ap.add_argument("--batch-scale", type=int, default=21)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (RMAT-14, grid, batched, serving) in the default line")
    ap.add_argument("--cpu-budget", type=float, default=30.0)
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.workload == "grid":
        run_grid_workload(args)
        return
    if args.workload == "batched":
        run_batched_workload(args)
        return
    if args.workload == "tune":
        run_tune_workload(args)
        return
    if args.workload == "gather":
        run_gather_workload(args)
        return
    if args.workload == "serve":
        run_serve_workload(args)
        return
    if args.workload == "lb":
        run_lb_workload(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
