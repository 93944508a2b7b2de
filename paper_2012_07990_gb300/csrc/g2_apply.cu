// g2_apply.cu — one round of edgeset.apply / applyModified (Sec. IV) under a
// SimpleGPUSchedule (Table II): load balancing x direction x frontier
// creation x deduplication, and the hybrid choice between two schedules
// (Table III).  Also the public g2_edgeset_apply.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "g2_host.h"
#include "g2_lb.cuh"
#include "g2_push.cuh"

namespace g2 {

// ---------------------------------------------------------- kernel wrappers
template <class P, int G>
__global__ void __launch_bounds__(kCta) k_pull(DevGraph g, const int32_t *cand, int32_t ncand,
                                               Member mem, P op, OutCtx out,
                                               unsigned long long *ctr) {
    lb_pull<P, G>(g, cand, ncand, mem, op, out, blockIdx.x, gridDim.x, ctr);
}

template <class P>
static g2_status pull_round(g2_graph *g, const g2_schedule &s, const P &op, const VSet &in,
                            const OutCtx &out, unsigned long long *ctr, cudaStream_t st) {
    Topology *t = g->topo;
    const DevGraph dg = t->view();
    Member mem{MEM_ALL, nullptr, nullptr};
    if (in.rep == OUT_BITMAP) mem = Member{MEM_BITMAP, in.bitmap, nullptr};
    else if (in.rep == OUT_BOOLMAP) mem = Member{MEM_BOOLMAP, nullptr, in.boolmap};
    else if (in.rep != -1) return fail(G2_EINVAL, "PULL needs a bitmap/boolmap input frontier");
    const int32_t n = t->n;
    if (n == 0) return G2_OK;
    switch (s.load_balance) {
        case G2_LB_VERTEX_BASED:
            k_pull<P, 1><<<grid_for(g, n, kCta), kCta, 0, st>>>(dg, nullptr, n, mem, op, out, ctr);
            break;
        case G2_LB_WM:
            k_pull<P, 32><<<grid_for(g, (int64_t)n * 32, kCta), kCta, 0, st>>>(dg, nullptr, n, mem,
                                                                              op, out, ctr);
            break;
        case G2_LB_CM:
            k_pull<P, kCta><<<grid_for(g, (int64_t)n * kCta, kCta), kCta, 0, st>>>(dg, nullptr, n,
                                                                                  mem, op, out, ctr);
            break;
        default:
            return fail(G2_EUNSUPPORTED, "PULL supports VERTEX_BASED, WM and CM load balancing");
    }
    stats().launches += 1;
    G2_CK(cudaGetLastError());
    return G2_OK;
}

g2_status check_schedule(const g2_graph *g, const g2_schedule &s, OpKind op, bool all_vertices) {
    (void)g;
    if (s.load_balance < 0 || s.load_balance > G2_LB_TWC) return fail(G2_EINVAL, "bad load_balance");
    if (s.direction != G2_PUSH && s.direction != G2_PULL) return fail(G2_EINVAL, "bad direction");
    if (s.pull_frontier != G2_BOOLMAP && s.pull_frontier != G2_BITMAP)
        return fail(G2_EINVAL, "bad pull frontier representation");
    if (s.frontier_creation < G2_FUSED || s.frontier_creation > G2_UNFUSED_BITMAP)
        return fail(G2_EINVAL, "bad frontier_creation");
    if (s.dedup != G2_DEDUP_ENABLED && s.dedup != G2_DEDUP_DISABLED)
        return fail(G2_EINVAL, "bad dedup");
    if (s.dedup_type < G2_DEDUP_MONOTONIC_COUNTERS || s.dedup_type > G2_DEDUP_BOOLMAP)
        return fail(G2_EINVAL, "bad dedup_type");
    if (s.delta < 0 || s.blocking_size < 0) return fail(G2_EINVAL, "negative delta/blocking_size");
    if (s.edge_blocking && s.load_balance != G2_LB_EDGE_ONLY)
        return fail(G2_EUNSUPPORTED, "EdgeBlocking applies to EDGE_ONLY full sweeps only");
    if (s.direction == G2_PULL) {
        if (s.load_balance != G2_LB_VERTEX_BASED && s.load_balance != G2_LB_WM &&
            s.load_balance != G2_LB_CM)
            return fail(G2_EUNSUPPORTED, "PULL supports VERTEX_BASED, WM and CM load balancing");
        if (op == K_HOOK) return fail(G2_EUNSUPPORTED, "hooking is a PUSH update");
    } else {
        if (s.load_balance == G2_LB_EDGE_ONLY && !all_vertices)
            return fail(G2_EUNSUPPORTED, "EDGE_ONLY needs the all-vertices frontier");
    }
    return G2_OK;
}

g2_hybrid default_hybrid() {
    g2_hybrid h;
    memset(&h, 0, sizeof(h));
    return h;
}

const g2_schedule &pick_schedule(const g2_hybrid &h, int32_t size, int32_t n) {
    if (h.criteria != G2_INPUT_VERTEXSET_SIZE) return h.s1;
    return (double)size < (double)h.threshold * (double)n ? h.s1 : h.s2;
}

// --------------------------------------------------------------- apply_round
g2_status apply_round(g2_graph *g, const g2_schedule &s, const OpArgs &a, const VSet &in,
                      const OutArgs &o, cudaStream_t st) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = o.rep;
    out.q = o.q;
    out.cnt = o.cnt;
    out.cap = o.qcap;
    out.bitmap = o.bitmap;
    out.boolmap = o.boolmap;
    out.err = a.err;
    out.dedup = DD_NONE;
    if (o.rep == OUT_SPARSE && o.dedup != DD_NONE) {
        out.dedup = o.dedup;
        if (o.dedup == DD_STAMP) {
            G2_TRY(ws(g, B_STAMP, (size_t)std::max(n, 1), &out.stamp));
            if (g->round == 0 || g->round == 0x7fffffff) {
                G2_CK(cudaMemsetAsync(out.stamp, 0, (size_t)std::max(n, 1) * 4, st));
                g->round = 0;
            }
            out.round = ++g->round;
        } else if (o.dedup == DD_BITMAP) {
            size_t words = (size_t)(n + 31) / 32 + 1;
            G2_TRY(ws(g, B_DDBM, words, &out.dd_bitmap));
            G2_CK(cudaMemsetAsync(out.dd_bitmap, 0, words * 4, st));
        } else if (o.dedup == DD_BOOLMAP) {
            G2_TRY(ws(g, B_DDBOOL, (size_t)std::max(n, 1), &out.dd_boolmap));
            G2_CK(cudaMemsetAsync(out.dd_boolmap, 0, (size_t)std::max(n, 1), st));
        }
    }
    if (o.q2) {
        out.q2 = o.q2;
        out.cnt2 = o.cnt2;
        out.cap2 = o.q2cap;
        out.stamp2 = o.stamp2;
        out.round2 = o.round2;
    }
    unsigned long long *ctr = nullptr;
    if (count_arcs_enabled()) G2_TRY(ws(g, B_ARCS, 2, &ctr));
    const DevGraph dg = t->view();
    static const char *push_names[] = {"bfs_push", "sssp_relax", "label_push", "pr_push",
                                       "sigma_push", "cc_hook", "delta_push"};
    static const char *pull_names[] = {"bfs_pull", "relax_pull", "label_pull", "pr_pull",
                                       "sigma_pull", "hook_pull", "delta_pull"};
    KTime kt;
    ktime_begin(kt, s.direction == G2_PUSH ? push_names[a.kind] : pull_names[a.kind], st);
    g2_status r = G2_OK;
    if (s.direction == G2_PUSH) {
        switch (a.kind) {
            case K_BFS: r = push_round(g, s, OpBFS{a.i0, a.i1}, in, out, ctr, st); break;
            case K_RELAX:
                r = push_round(g, s, OpRelaxMin{a.i0, dg.w, a.err, a.threshold}, in, out, ctr, st);
                break;
            case K_LABEL: r = push_round(g, s, OpLabelMin{a.i0}, in, out, ctr, st); break;
            case K_PR: r = push_round(g, s, OpPRAdd{a.f0, a.f1}, in, out, ctr, st); break;
            case K_SIGMA: r = push_round(g, s, OpBCSigma{a.i0, a.d0}, in, out, ctr, st); break;
            case K_HOOK: r = push_round(g, s, OpHook{a.i0}, in, out, ctr, st); break;
            case K_DELTA:
                r = push_round(g, s, OpBCDelta{a.i0, a.d0, a.d0 + g->topo->n}, in, out, ctr, st);
                break;
        }
    } else {
        switch (a.kind) {
            case K_BFS: r = pull_round(g, s, PullBFS{a.i0, a.i1}, in, out, ctr, st); break;
            case K_RELAX: r = pull_round(g, s, PullRelaxMin{a.i0, dg.cw, a.err}, in, out, ctr, st); break;
            case K_LABEL: r = pull_round(g, s, PullLabelMin{a.i0}, in, out, ctr, st); break;
            case K_PR: r = pull_round(g, s, PullPRAdd{a.f0, a.f1}, in, out, ctr, st); break;
            case K_SIGMA: r = pull_round(g, s, PullBCSigma{a.i0, a.d0}, in, out, ctr, st); break;
            case K_HOOK: r = fail(G2_EUNSUPPORTED, "hooking is a PUSH update"); break;
            case K_DELTA:
                r = pull_round(g, s, PullBCDelta{a.i0, a.d0, a.d0 + g->topo->n}, in, out, ctr, st);
                break;
        }
    }
    ktime_end(kt, st);
    return r;
}

}  // namespace g2

using namespace g2;

// ====================================================================== C ABI
extern "C" g2_status g2_edgeset_apply(g2_graph *g, g2_op op, g2_frontier *in, void *vdata,
                                      void *vdata2, const g2_hybrid *sched, g2_frontier *outf,
                                      int32_t *out_size, void *stream) {
    if (!g) return fail(G2_EINVAL, "null graph");
    if (!vdata) return fail(G2_EINVAL, "null vdata");
    if ((in && in->g->topo != g->topo) || (outf && outf->g->topo != g->topo))
        return fail(G2_EINVAL, "frontier belongs to another graph");
    OpKind kind;
    switch (op) {
        case G2_OP_BFS: kind = K_BFS; break;
        case G2_OP_RELAX_MIN: kind = K_RELAX; break;
        case G2_OP_LABEL_MIN: kind = K_LABEL; break;
        case G2_OP_PR_ADD: kind = K_PR; break;
        case G2_OP_BC_SIGMA: kind = K_SIGMA; break;
        case G2_OP_BC_DELTA: kind = K_DELTA; break;
        default: return fail(G2_EINVAL, "unknown op");
    }
    const bool no_out = kind == K_PR || kind == K_SIGMA || kind == K_DELTA;
    if (no_out && !vdata2) return fail(G2_EINVAL, "op needs vdata2");
    if (no_out && outf)
        return fail(G2_EINVAL, "this op produces no output vertexset (out must be NULL)");
    if (kind == K_DELTA && !g->topo->symmetric)
        return fail(G2_EINVAL, "BC_DELTA needs a symmetric graph");
    if (kind == K_RELAX && !g->topo->w) return fail(G2_EINVAL, "RELAX_MIN needs arc weights");
    Topology *t = g->topo;
    const int32_t n = t->n;
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : default_hybrid();
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    int32_t *ctrs = d_err - 62;

    // input vertexset and its size
    VSet vin{-1, nullptr, 0, nullptr, nullptr, nullptr, n};
    if (in) {
        int32_t sz = 0;
        G2_TRY(g2_frontier_size(in, &sz, stream));
        vin.size = sz;
        if (in->format == G2_FRONTIER_SPARSE) {
            vin.rep = OUT_SPARSE; vin.q = in->q; vin.qcap = in->cap; vin.cnt = in->cnt;
        } else if (in->format == G2_FRONTIER_BITMAP) {
            vin.rep = OUT_BITMAP; vin.bitmap = in->bitmap;
        } else {
            vin.rep = OUT_BOOLMAP; vin.boolmap = in->boolmap;
        }
    }
    const g2_schedule &s = pick_schedule(h, vin.size, n);
    G2_TRY(check_schedule(g, s, kind, in == nullptr));
    if (s.kernel_fusion) return fail(G2_EUNSUPPORTED, "kernel fusion applies to whole loops (g2_bfs, g2_sssp_delta)");

    // bring the input to the representation the direction needs
    VSet use = vin;
    if (in) {
        if (s.direction == G2_PUSH && vin.rep != OUT_SPARSE) {
            VSet tmp{OUT_SPARSE, nullptr, std::max(n, 1), ctrs + 60, nullptr, nullptr, 0};
            G2_TRY(ws(g, B_Q2, (size_t)std::max(n, 1), &tmp.q));
            G2_TRY(vset_convert(g, vin, OUT_SPARSE, tmp, st));
            use = tmp;
        } else if (s.direction == G2_PULL) {
            int want = s.pull_frontier == G2_BITMAP ? OUT_BITMAP : OUT_BOOLMAP;
            if (vin.rep != want) {
                VSet tmp{want, nullptr, 0, nullptr, nullptr, nullptr, vin.size};
                if (want == OUT_BITMAP) G2_TRY(ws(g, B_BM0, (size_t)(n + 31) / 32 + 1, &tmp.bitmap));
                else G2_TRY(ws(g, B_BOOL0, (size_t)std::max(n, 1), &tmp.boolmap));
                G2_TRY(vset_convert(g, vin, want, tmp, st));
                use = tmp;
            }
        }
    }

    // output per frontier_creation, into workspace, then into the caller's frontier
    OutArgs o;
    memset(&o, 0, sizeof(o));
    o.rep = OUT_NONE;
    VSet produced{OUT_NONE, nullptr, 0, nullptr, nullptr, nullptr, 0};
    if (outf) {
        if (s.frontier_creation == G2_FUSED) {
            bool dedup = s.dedup == G2_DEDUP_ENABLED;
            size_t cap = dedup ? (size_t)std::max(n, 1) : (size_t)t->m + (size_t)n + 1;
            G2_TRY(ws(g, dedup ? B_Q3 : B_BIG, cap, &o.q));
            o.rep = OUT_SPARSE;
            o.qcap = (int32_t)std::min<size_t>(cap, 2147483647u);
            o.cnt = ctrs + 61;
            G2_CK(cudaMemsetAsync(o.cnt, 0, sizeof(int32_t), st));
            o.dedup = !dedup ? DD_NONE
                      : s.dedup_type == G2_DEDUP_BITMAP ? DD_BITMAP
                      : s.dedup_type == G2_DEDUP_BOOLMAP ? DD_BOOLMAP
                                                         : DD_STAMP;
            produced = VSet{OUT_SPARSE, o.q, o.qcap, o.cnt, nullptr, nullptr, 0};
        } else if (s.frontier_creation == G2_UNFUSED_BITMAP) {
            size_t words = (size_t)(n + 31) / 32 + 1;
            G2_TRY(ws(g, B_BM1, words, &o.bitmap));
            G2_CK(cudaMemsetAsync(o.bitmap, 0, words * 4, st));
            o.rep = OUT_BITMAP;
            produced = VSet{OUT_BITMAP, nullptr, 0, nullptr, o.bitmap, nullptr, 0};
        } else {
            G2_TRY(ws(g, B_BOOL1, (size_t)std::max(n, 1), &o.boolmap));
            G2_CK(cudaMemsetAsync(o.boolmap, 0, (size_t)std::max(n, 1), st));
            o.rep = OUT_BOOLMAP;
            produced = VSet{OUT_BOOLMAP, nullptr, 0, nullptr, nullptr, o.boolmap, 0};
        }
    }
    OpArgs a;
    memset(&a, 0, sizeof(a));
    a.kind = kind;
    a.err = d_err;
    a.threshold = G2_INF32;
    switch (kind) {
        case K_BFS: a.i0 = (int32_t *)vdata; a.i1 = (int32_t *)vdata2; break;
        case K_RELAX: case K_LABEL: a.i0 = (int32_t *)vdata; break;
        case K_PR: a.f0 = (const float *)vdata; a.f1 = (float *)vdata2; break;
        case K_SIGMA: case K_DELTA: a.i0 = (int32_t *)vdata; a.d0 = (double *)vdata2; break;
        default: break;
    }
    G2_TRY(apply_round(g, s, a, use, o, st));
    s.direction == G2_PUSH ? stats().push_rounds++ : stats().pull_rounds++;
    stats().iterations = 1;

    int32_t size = 0;
    if (outf) {
        // produced -> caller's representation
        if (produced.rep == OUT_SPARSE) {
            G2_CK(cudaMemcpyAsync(g->h_ctr, o.cnt, 4, cudaMemcpyDeviceToHost, st));
            G2_TRY(sync_and_check(g, st, d_err));
            size = g->h_ctr[0];
        } else {
            G2_TRY(vset_count(g, produced, ctrs + 59, st));
            G2_CK(cudaMemcpyAsync(g->h_ctr, ctrs + 59, 4, cudaMemcpyDeviceToHost, st));
            G2_TRY(sync_and_check(g, st, d_err));
            size = g->h_ctr[0];
        }
        produced.size = size;
        if (outf->format == G2_FRONTIER_SPARSE) {
            if (size > outf->cap) {
                dfree(outf->q, st);
                outf->q = nullptr;
                G2_CK(dmalloc(&outf->q, (size_t)size * 4, st));
                outf->cap = size;
            }
            if (produced.rep == OUT_SPARSE) {
                if (size > 0)
                    G2_CK(cudaMemcpyAsync(outf->q, produced.q, (size_t)size * 4,
                                          cudaMemcpyDeviceToDevice, st));
            } else {
                VSet d{OUT_SPARSE, outf->q, outf->cap, outf->cnt, nullptr, nullptr, 0};
                G2_TRY(vset_convert(g, produced, OUT_SPARSE, d, st));
            }
            G2_CK(cudaMemcpyAsync(outf->cnt, o.rep == OUT_SPARSE ? o.cnt : &size, 4,
                                  o.rep == OUT_SPARSE ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyHostToDevice,
                                  st));
        } else {
            int want = outf->format == G2_FRONTIER_BITMAP ? OUT_BITMAP : OUT_BOOLMAP;
            VSet d{want, nullptr, 0, nullptr, outf->bitmap, outf->boolmap, 0};
            if (produced.rep == want) {
                if (want == OUT_BITMAP)
                    G2_CK(cudaMemcpyAsync(outf->bitmap, produced.bitmap, ((size_t)(n + 31) / 32) * 4,
                                          cudaMemcpyDeviceToDevice, st));
                else
                    G2_CK(cudaMemcpyAsync(outf->boolmap, produced.boolmap, (size_t)n,
                                          cudaMemcpyDeviceToDevice, st));
            } else {
                G2_TRY(vset_convert(g, produced, want, d, st));
            }
        }
    }
    G2_TRY(end_call(g, st, d_err));
    if (out_size) *out_size = size;
    return G2_OK;
}
