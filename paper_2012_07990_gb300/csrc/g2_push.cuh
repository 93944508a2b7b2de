// g2_push.cuh — __global__ wrappers of the PUSH load-balancing routines and
// the dispatcher that runs one PUSH round of any update function under a
// schedule's load balancing.  Shared by every translation unit that defines
// update functions (the single-source ops and the multi-source ones).
#pragma once
#include "g2_host.h"
#include "g2_lb.cuh"

namespace g2 {

// ---------------------------------------------------------- kernel wrappers
template <class Op>
__global__ void __launch_bounds__(kCta) k_push_vertex(DevGraph g, FrontierIn fin, int32_t fsize,
                                                      Op op, OutCtx out, unsigned long long *ctr) {
    lb_vertex(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_push_warp(DevGraph g, FrontierIn fin, int32_t fsize,
                                                    Op op, OutCtx out, unsigned long long *ctr) {
    lb_warp(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_push_cta(DevGraph g, FrontierIn fin, int32_t fsize,
                                                   Op op, OutCtx out, unsigned long long *ctr) {
    lb_cta(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_push_etwc(DevGraph g, FrontierIn fin, int32_t fsize,
                                                    Op op, OutCtx out, unsigned long long *ctr,
                                                    EtwcSpill<typename Op::S> spill) {
    lb_etwc(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr, spill);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_push_etwc_spill(DevGraph g,
                                                          const EtwcEntry<typename Op::S> *q,
                                                          const int32_t *cnt, Op op, OutCtx out) {
    lb_etwc_spill(g, q, cnt, op, out, blockIdx.x, gridDim.x);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_push_strict(DevGraph g, FrontierIn fin, int32_t fsize,
                                                      const int32_t *scan, Op op, OutCtx out,
                                                      unsigned long long *ctr) {
    lb_strict(g, fin, fsize, scan, op, out, blockIdx.x, gridDim.x, ctr);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_twc_classify(DevGraph g, FrontierIn fin, int32_t fsize,
                                                       Op op, int32_t *qs, int32_t *qm,
                                                       int32_t *ql, int32_t *counts) {
    lb_twc_classify(g, fin, fsize, op, qs, qm, ql, counts, blockIdx.x, gridDim.x);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_twc_process(DevGraph g, const int32_t *qs,
                                                      const int32_t *qm, const int32_t *ql,
                                                      const int32_t *counts, Op op, OutCtx out,
                                                      unsigned long long *ctr) {
    lb_twc_process(g, qs, qm, ql, counts, op, out, blockIdx.x, gridDim.x, ctr);
}
template <class Op>
__global__ void __launch_bounds__(kCta) k_push_edges(const int32_t *src, const int32_t *dst,
                                                     int64_t e0, int64_t e1, Op op, OutCtx out,
                                                     unsigned long long *ctr) {
    lb_edges(src, dst, e0, e1, op, out, blockIdx.x, gridDim.x, ctr);
}
// degrees of the active vertices (0 for skipped ones), for the STRICT scan
template <class Op>
__global__ void k_frontier_degrees(DevGraph g, FrontierIn fin, int32_t fsize, Op op,
                                   int32_t *deg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < fsize;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = fin.vertex((int32_t)i);
        deg[i] = op.skip(op.load(u)) ? 0 : g.rowptr[u + 1] - g.rowptr[u];
    }
}

// ------------------------------------------------------------ push dispatch
template <class Op>
inline g2_status push_round(g2_graph *g, const g2_schedule &s, const Op &op, const VSet &in,
                            const OutCtx &out, unsigned long long *ctr, cudaStream_t st) {
    Topology *t = g->topo;
    const DevGraph dg = t->view();
    FrontierIn fin{in.rep == -1 ? nullptr : in.q, in.size, nullptr};
    const int32_t fsize = in.rep == -1 ? t->n : in.size;
    if (fsize == 0 && s.load_balance != G2_LB_EDGE_ONLY) return G2_OK;
    switch (s.load_balance) {
        case G2_LB_VERTEX_BASED:
            k_push_vertex<<<grid_for(g, fsize, kCta), kCta, 0, st>>>(dg, fin, fsize, op, out, ctr);
            break;
        case G2_LB_WM:
            k_push_warp<<<grid_for(g, fsize, kCta), kCta, 0, st>>>(dg, fin, fsize, op, out, ctr);
            break;
        case G2_LB_CM:
            k_push_cta<<<grid_for(g, fsize, kCta), kCta, 0, st>>>(dg, fin, fsize, op, out, ctr);
            break;
        case G2_LB_ETWC: {
            // entries of kEtwcSpill arcs or more are handed to a second pass
            // over the whole grid, where the graph has such vertices
            int32_t maxdeg = 0;
            G2_TRY(max_out_degree(g, st, &maxdeg));
            EtwcSpill<typename Op::S> spill{nullptr, nullptr};
            if (maxdeg >= kEtwcSpill) {
                int32_t *ctrs;
                G2_TRY(ws(g, B_CTR, 64, &ctrs));
                spill.cnt = ctrs + 45;
                G2_TRY(ws(g, B_TWC_L, (size_t)fsize, &spill.q));
                G2_CK(cudaMemsetAsync(spill.cnt, 0, sizeof(int32_t), st));
            }
            k_push_etwc<<<grid_for(g, fsize, kCta), kCta, 0, st>>>(dg, fin, fsize, op, out, ctr, spill);
            if (spill.q) {
                k_push_etwc_spill<<<t->sm_count * 8, kCta, 0, st>>>(dg, spill.q, spill.cnt, op, out);
                stats().launches += 1;
            }
            break;
        }
        case G2_LB_STRICT: {
            int32_t *deg, *scan;
            G2_TRY(ws(g, B_I1, (size_t)fsize + 1, &deg));
            G2_TRY(ws(g, B_SCAN, (size_t)fsize + 1, &scan));
            k_frontier_degrees<<<grid_for(g, fsize, kCta), kCta, 0, st>>>(dg, fin, fsize, op, deg);
            G2_TRY(exclusive_scan_i32(g, deg, scan, fsize, st));
            // one tile per kCta*4 arcs; the arc total is on the device, so size
            // the grid for the resident CTAs and stride
            k_push_strict<<<t->sm_count * 8, kCta, 0, st>>>(dg, fin, fsize, scan, op, out, ctr);
            stats().launches += 1;
            break;
        }
        case G2_LB_TWC: {
            int32_t *qs, *qm, *ql, *ctrs;
            G2_TRY(ws(g, B_TWC_S, (size_t)fsize, &qs));
            G2_TRY(ws(g, B_TWC_M, (size_t)fsize, &qm));
            G2_TRY(ws(g, B_TWC_L, (size_t)fsize, &ql));
            G2_TRY(ws(g, B_CTR, 64, &ctrs));
            G2_CK(cudaMemsetAsync(ctrs + 40, 0, 3 * sizeof(int32_t), st));
            k_twc_classify<<<grid_for(g, fsize, kCta), kCta, 0, st>>>(dg, fin, fsize, op, qs, qm,
                                                                    ql, ctrs + 40);
            k_twc_process<<<grid_for(g, fsize, kCta), kCta, 0, st>>>(dg, qs, qm, ql, ctrs + 40, op,
                                                                   out, ctr);
            stats().launches += 1;
            break;
        }
        case G2_LB_EDGE_ONLY: {
            if (in.rep != -1) return fail(G2_EINVAL, "EDGE_ONLY needs the all-vertices frontier");
            if (t->m == 0) return G2_OK;
            if (s.edge_blocking) {
                // Algorithm 2: segment by segment, one launch per segment so that
                // the destination range of a segment stays in L2
                G2_TRY(ensure_edge_block(g, s.blocking_size, st));
                int64_t prev = 0;
                for (int32_t seg = 0; seg < t->eb_nseg; ++seg) {
                    int64_t e1 = t->h_eb_seg[seg];
                    if (e1 > prev)
                        k_push_edges<<<grid_for(g, e1 - prev, kCta), kCta, 0, st>>>(
                            t->eb_src, t->eb_dst, prev, e1, op, out, ctr);
                    stats().launches += 1;
                    prev = e1;
                }
                stats().launches -= 1;
            } else {
                G2_TRY(ensure_coo(g, st));
                k_push_edges<<<grid_for(g, t->m, kCta), kCta, 0, st>>>(t->coo_src, t->col, 0, t->m,
                                                                     op, out, ctr);
            }
            break;
        }
        default: return fail(G2_EINVAL, "unknown load_balance");
    }
    stats().launches += 1;
    G2_CK(cudaGetLastError());
    return G2_OK;
}

}  // namespace g2
