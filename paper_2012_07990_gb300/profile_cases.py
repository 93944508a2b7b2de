"""Small, fixed invocations of the library's kernels for profiler captures
(one launch of each kernel of interest, a few hundred MB on the device at
most), so that a capture names a committed command.

    python -m paper_2012_07990_gb300.profile_cases road_fused --grid 1024

road_fused: a road-like W x W grid (graphgen.road_grid(W, seed=1), weights
pair_weights(G, 1000, seed=1)), one fused WM BFS from vertex 0 (no parent
array) and one fused WM delta-stepping SSSP from vertex 0 with delta 1024 —
the one-cluster loops (k_bfs_cluster, k_sssp_cluster) on this grid size.

bc_rmat: RMAT-S (graphgen.rmat(S, seed=1)), betweenness centrality from the
two highest-degree vertices with the library's NULL schedule — the level
passes k_bc_level<true/false> on a power-law graph.
"""
from __future__ import annotations

import argparse


def road_fused(grid: int) -> None:
    import torch

    from . import build_native
    build_native.build()
    from . import g2
    from . import graphgen as gg
    G = gg.road_grid(grid, seed=1)
    w = gg.pair_weights(G, 1000, seed=1)
    dg = g2.load_graph(G, w)
    out = torch.empty(G.n, dtype=torch.int32, device="cuda")
    s = g2.schedule("WM", kernel_fusion=True)
    g2.g2_bfs(dg, 0, out, None, s)
    bfs = g2.g2_last_stats()
    g2.g2_sssp_delta(dg, 0, 1024, out, s)
    sssp = g2.g2_last_stats()
    torch.cuda.synchronize()
    print(f"road_fused grid {grid}: bfs levels {bfs['iterations']} launches {bfs['launches']}; "
          f"sssp rounds {sssp['iterations']} launches {sssp['launches']}")
    dg.free()


def bc_rmat(scale: int) -> None:
    import numpy as np
    import torch

    from . import build_native
    build_native.build()
    from . import g2
    from . import graphgen as gg
    G = gg.rmat(scale, seed=1)
    dg = g2.load_graph(G)
    srcs = np.argsort(-G.degrees(), kind="stable")[:2].astype(np.int32)
    bc = torch.empty(G.n, dtype=torch.float64, device="cuda")
    g2.g2_bc(dg, srcs, bc, None)
    st = g2.g2_last_stats()
    torch.cuda.synchronize()
    print(f"bc_rmat scale {scale}: levels {st['iterations']} launches {st['launches']}")
    dg.free()


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=["road_fused", "bc_rmat"])
    ap.add_argument("--grid", type=int, default=1024)
    ap.add_argument("--scale", type=int, default=21)
    args = ap.parse_args()
    if args.case == "road_fused":
        road_fused(args.grid)
    else:
        bc_rmat(args.scale)


if __name__ == "__main__":
    main()
