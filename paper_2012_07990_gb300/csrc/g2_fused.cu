// g2_fused.cu — kernel fusion (Sec. III and VI-C, Fig. 5 middle): the whole
// while loop of BFS or delta-stepping SSSP runs inside one persistent
// cooperative kernel.  Loop state lives in device memory, every resident CTA
// does the work of many virtual CTAs through the load-balancing library's
// device routines, and a grid barrier separates the rounds.  Each barrier
// wait is bounded in time; when it runs out the kernel records G2_ETIMEOUT
// and returns, and the host reports the status.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "g2_host.h"
#include "g2_lb.cuh"

namespace g2 {

template <int LB, class Op>
__device__ __forceinline__ void run_lb(const DevGraph &g, const FrontierIn &fin, int32_t size,
                                       const Op &op, const OutCtx &out,
                                       unsigned long long *ctr) {
    if (LB == G2_LB_WM) lb_warp(g, fin, size, op, out, blockIdx.x, gridDim.x, ctr);
    else if (LB == G2_LB_CM) lb_cta(g, fin, size, op, out, blockIdx.x, gridDim.x, ctr);
    else if (LB == G2_LB_ETWC) lb_etwc(g, fin, size, op, out, blockIdx.x, gridDim.x, ctr);
    else lb_vertex(g, fin, size, op, out, blockIdx.x, gridDim.x, ctr);
}

struct FusedBfsArgs {
    DevGraph g;
    int32_t *depth;
    int32_t *parent;
    int32_t *q[2];
    int32_t *cnt;      // [3] rotating list lengths; cnt[0] = 1 at launch
    int32_t *result;   // [0] rounds
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;
    unsigned long long *ctr;
};

// One launch for the whole BFS.  Round d reads list d&1 (length cnt[d%3]) and
// appends to list (d+1)&1 (length cnt[(d+1)%3]); cnt[(d+2)%3], read in round
// d-1 only, is cleared for round d+1.  One barrier per round.
template <int LB>
__global__ void __launch_bounds__(kCta) k_bfs_fused(FusedBfsArgs a) {
    OpBFS op{a.depth, a.parent};
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = OUT_SPARSE;
    out.dedup = DD_NONE;  // the compare-and-swap on depth admits each vertex once
    out.cap = a.g.n;
    out.err = a.err;
    int d = 0;
    for (;; ++d) {
        int32_t size = ld_relaxed_i32(a.cnt + d % 3);
        if (size == 0) break;
        FrontierIn fin{a.q[d & 1], size, nullptr};
        out.q = a.q[(d + 1) & 1];
        out.cnt = a.cnt + (d + 1) % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[(d + 2) % 3] = 0;
        run_lb<LB>(a.g, fin, size, op, out, a.ctr);
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.result[0] = d;
}

struct FusedSsspArgs {
    DevGraph g;
    int32_t *dist;
    int32_t delta;
    int32_t *nq[2];
    int32_t *fq[2];
    int32_t *ncnt;     // [3] rotating near-list lengths; ncnt[0] = 1 at launch
    int32_t *fcnt;     // [2] far-pile lengths (zero at launch)
    int32_t *dmin;     // [2] far minimum per epoch parity (G2_INF32 at launch)
    int32_t *stamp;    // near dedup stamps
    int32_t round0;    // first near stamp
    int32_t *stamp2;   // far dedup stamps
    int32_t epoch0;    // first far stamp
    int32_t *result;   // [0] near rounds, [1] buckets
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;
    unsigned long long *ctr;
};

// Delta-stepping with the near/far two-bucket queue in one launch.  Near
// rounds relax the current bucket until it empties (improvements below the
// threshold go to the next near list, the rest to the far pile); then the
// smallest live far distance picks the next bucket and the far pile is split
// (stale entries, already settled, are dropped).
template <int LB>
__global__ void __launch_bounds__(kCta) k_sssp_fused(FusedSsspArgs a) {
    const int32_t n = a.g.n;
    int64_t T = a.delta;
    int d = 0, fp = 0, epoch = 0, buckets = 0;
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = OUT_SPARSE;
    out.dedup = DD_STAMP;
    out.stamp = a.stamp;
    out.cap = n;
    out.err = a.err;
    out.cap2 = n;
    out.stamp2 = a.stamp2;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int32_t size = ld_relaxed_i32(a.ncnt + d % 3);
        if (size > 0) {
            OpRelaxMin op{a.dist, a.g.w, a.err, (int32_t)(T < G2_INF32 ? T : G2_INF32)};
            FrontierIn fin{a.nq[d & 1], size, nullptr};
            out.q = a.nq[(d + 1) & 1];
            out.cnt = a.ncnt + (d + 1) % 3;
            out.round = a.round0 + d;
            out.q2 = a.fq[fp];
            out.cnt2 = a.fcnt + fp;
            out.round2 = a.epoch0 + epoch;
            if (blockIdx.x == 0 && threadIdx.x == 0) a.ncnt[(d + 2) % 3] = 0;
            run_lb<LB>(a.g, fin, size, op, out, a.ctr);
            if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
            ++d;
            continue;
        }
        // near list empty: next bucket from the far pile
        const int32_t nfar = ld_relaxed_i32(a.fcnt + fp);
        if (nfar == 0) break;
        const int32_t Told = (int32_t)(T < G2_INF32 ? T : G2_INF32);
        int32_t *dm = a.dmin + (epoch & 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.fcnt[1 - fp] = 0;
            a.dmin[1 - (epoch & 1)] = G2_INF32;
        }
        {
            int32_t best = G2_INF32;
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nfar;
                 i += (int64_t)gridDim.x * blockDim.x) {
                int32_t dv = a.dist[a.fq[fp][i]];
                if (dv >= Told && dv < best) best = dv;
            }
            best = (int32_t)__reduce_min_sync(G2_FULL, (unsigned)best);
            if (lane == 0 && best != G2_INF32) atomicMin(dm, best);
        }
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
        const int32_t dmin = ld_relaxed_i32(dm);
        if (dmin == G2_INF32) break;
        const int64_t Tnew = ((int64_t)dmin / a.delta + 1) * (int64_t)a.delta;
        const int32_t Tn = (int32_t)(Tnew < G2_INF32 ? Tnew : G2_INF32);
        const int32_t newepoch = a.epoch0 + epoch + 1;
        // split: near list d&1 (its length ncnt[d%3] is zero), far pile 1-fp
        for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nfar;
             base += (int64_t)gridDim.x * blockDim.x) {
            int64_t i = base + lane;
            int32_t v = 0, dv = G2_INF32;
            bool ok = i < nfar;
            if (ok) {
                v = a.fq[fp][i];
                dv = a.dist[v];
            }
            bool to_near = ok && dv >= Told && dv < Tn;
            bool to_far = ok && dv >= Tn;
            if (to_far) a.stamp2[v] = newepoch;
            warp_append(a.nq[d & 1], a.ncnt + d % 3, n, a.err, v, to_near);
            warp_append(a.fq[1 - fp], a.fcnt + 1 - fp, n, a.err, v, to_far);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ncnt[(d + 1) % 3] = 0;
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
        fp = 1 - fp;
        ++epoch;
        ++buckets;
        T = Tnew;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.result[0] = d;
        a.result[1] = buckets;
    }
}

__global__ void k_fill_dist(int32_t *a, int32_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        a[v] = G2_INF32;
}

static g2_status check_fused_lb(const g2_schedule &s) {
    if (s.direction != G2_PUSH)
        return fail(G2_EUNSUPPORTED, "fused loops run PUSH rounds");
    switch (s.load_balance) {
        case G2_LB_VERTEX_BASED: case G2_LB_WM: case G2_LB_CM: case G2_LB_ETWC: return G2_OK;
        default:
            return fail(G2_EUNSUPPORTED,
                        "fused loops support VERTEX_BASED, WM, CM and ETWC load balancing");
    }
}

g2_status bfs_fused(g2_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                    const g2_schedule &s, cudaStream_t st, int32_t *d_err) {
    G2_TRY(check_fused_lb(s));
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    FusedBfsArgs a;
    a.g = t->view();
    a.depth = depth;
    a.parent = parent;
    G2_TRY(ws(g, B_Q0, (size_t)std::max(n, 1), &a.q[0]));
    G2_TRY(ws(g, B_Q1, (size_t)std::max(n, 1), &a.q[1]));
    a.cnt = ctrs + 20;
    a.result = ctrs + 24;
    a.bar = GridBarrier{reinterpret_cast<unsigned long long *>(ctrs + 28)};
    a.err = d_err;
    a.limit_ns = barrier_limit_ns();
    a.ctr = nullptr;
    if (count_arcs_enabled()) G2_TRY(ws(g, B_ARCS, 2, &a.ctr));
    // depth/parent init and the source in list 0
    if (parent) G2_CK(cudaMemsetAsync(parent, 0xFF, (size_t)n * 4, st));
    G2_CK(cudaMemsetAsync(depth, 0xFF, (size_t)n * 4, st));
    int32_t zero = 0, one = 1;
    G2_CK(cudaMemcpyAsync(depth + src, &zero, 4, cudaMemcpyHostToDevice, st));
    if (parent) G2_CK(cudaMemcpyAsync(parent + src, &src, 4, cudaMemcpyHostToDevice, st));
    G2_CK(cudaMemcpyAsync(a.q[0], &src, 4, cudaMemcpyHostToDevice, st));
    G2_CK(cudaMemcpyAsync(a.cnt, &one, 4, cudaMemcpyHostToDevice, st));
    switch (s.load_balance) {
        case G2_LB_WM: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_WM>, a, st)); break;
        case G2_LB_CM: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_CM>, a, st)); break;
        case G2_LB_ETWC: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_ETWC>, a, st)); break;
        default: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_VERTEX_BASED>, a, st)); break;
    }
    G2_TRY(read_counters(g, ctrs + 24, 1, st, d_err));
    stats().iterations = g->h_ctr[0];
    stats().push_rounds = g->h_ctr[0];
    stats().barriers = g->h_ctr[0];
    return G2_OK;
}

g2_status sssp_fused(g2_graph *g, int32_t src, int32_t delta, int32_t *dist,
                     const g2_schedule &s, cudaStream_t st, int32_t *d_err) {
    G2_TRY(check_fused_lb(s));
    if (s.frontier_creation != G2_FUSED || s.dedup != G2_DEDUP_ENABLED)
        return fail(G2_EUNSUPPORTED, "the fused near/far queue uses FUSED lists with deduplication");
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    FusedSsspArgs a;
    a.g = t->view();
    a.dist = dist;
    a.delta = delta;
    G2_TRY(ws(g, B_Q0, (size_t)std::max(n, 1), &a.nq[0]));
    G2_TRY(ws(g, B_Q1, (size_t)std::max(n, 1), &a.nq[1]));
    G2_TRY(ws(g, B_Q2, (size_t)std::max(n, 1), &a.fq[0]));
    G2_TRY(ws(g, B_Q3, (size_t)std::max(n, 1), &a.fq[1]));
    G2_TRY(ws(g, B_STAMP, (size_t)std::max(n, 1), &a.stamp));
    G2_TRY(ws(g, B_STAMP2, (size_t)std::max(n, 1), &a.stamp2));
    // stamps only grow; restart them well before int32 runs out
    if (g->round == 0 || g->round > (1 << 29)) {
        G2_CK(cudaMemsetAsync(a.stamp, 0, (size_t)std::max(n, 1) * 4, st));
        g->round = 0;
    }
    if (g->round2 == 0 || g->round2 > (1 << 29)) {
        G2_CK(cudaMemsetAsync(a.stamp2, 0, (size_t)std::max(n, 1) * 4, st));
        g->round2 = 0;
    }
    a.round0 = g->round + 1;
    a.epoch0 = g->round2 + 1;
    a.ncnt = ctrs + 20;
    a.fcnt = ctrs + 23;
    a.dmin = ctrs + 25;
    a.result = ctrs + 30;
    a.bar = GridBarrier{reinterpret_cast<unsigned long long *>(ctrs + 28)};
    a.err = d_err;
    a.limit_ns = barrier_limit_ns();
    a.ctr = nullptr;
    if (count_arcs_enabled()) G2_TRY(ws(g, B_ARCS, 2, &a.ctr));
    int32_t init[8] = {1, 0, 0, 0, 0, G2_INF32, G2_INF32, 0};  // ncnt[3], fcnt[2], dmin[2]
    G2_CK(cudaMemcpyAsync(ctrs + 20, init, 7 * 4, cudaMemcpyHostToDevice, st));
    k_fill_dist<<<grid_for(g, n, kCta), kCta, 0, st>>>(dist, n);
    int32_t zero = 0;
    G2_CK(cudaMemcpyAsync(dist + src, &zero, 4, cudaMemcpyHostToDevice, st));
    G2_CK(cudaMemcpyAsync(a.nq[0], &src, 4, cudaMemcpyHostToDevice, st));
    switch (s.load_balance) {
        case G2_LB_WM: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_WM>, a, st)); break;
        case G2_LB_CM: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_CM>, a, st)); break;
        case G2_LB_ETWC: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_ETWC>, a, st)); break;
        default: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_VERTEX_BASED>, a, st)); break;
    }
    G2_TRY(read_counters(g, ctrs + 30, 2, st, d_err));
    stats().iterations = g->h_ctr[0];
    stats().push_rounds = g->h_ctr[0];
    stats().barriers = g->h_ctr[0] + 2 * g->h_ctr[1];
    g->round += g->h_ctr[0] + 1;
    g->round2 += g->h_ctr[1] + 1;
    return G2_OK;
}

}  // namespace g2
