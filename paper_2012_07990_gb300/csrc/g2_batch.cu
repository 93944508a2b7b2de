// g2_batch.cu — multi-source traversals: up to 64 BFS sources share one
// frontier loop with one bit per source in per-vertex 64-bit masks, and up to
// 32 SSSP sources relax stacked distance arrays together, so the topology is
// read once per round for all of them.  Both reuse the load-balancing library
// (PUSH) and its PULL routine with mask-valued update functions.
#include <cuda_runtime.h>

#include <string>
#include <thread>
#include <vector>

#include <algorithm>
#include <cstring>
#include <vector>

#include "g2_host.h"
#include "g2_lb.cuh"
#include "g2_push.cuh"

namespace g2 {

typedef unsigned long long u64;

// ------------------------------------------------------- multi-source BFS
// PUSH: the bits of u's frontier mask not yet visited at v are ORed into v's
// next mask; the first arc to touch v lists it.
struct OpMsBfs {
    const u64 *visit;
    const u64 *fcur;
    u64 *fnext;
    typedef u64 S;
    __device__ __forceinline__ S load(int32_t u) const { return fcur[u]; }
    __device__ __forceinline__ bool skip(S m) const { return m == 0; }
    __device__ __forceinline__ int relax(int32_t, S fm, int32_t v, int32_t) const {
        u64 m = fm & ~visit[v];
        if (m == 0) return 0;
        if ((fnext[v] & m) == m) return 0;
        u64 old = atomicOr(&fnext[v], m);
        return old == 0 ? 1 : 0;
    }
};

// PULL: v ORs the frontier masks of its in-neighbours, stops once every
// source has reached it.
struct PullMsBfs {
    u64 *visit;
    const u64 *fcur;
    u64 *fnext;
    int32_t *depth;
    int32_t n;
    int32_t level;  // depth assigned this round
    u64 full;
    typedef u64 Ctx;
    typedef u64 Acc;
    __device__ __forceinline__ Ctx ctx(int32_t v) const { return visit[v]; }
    __device__ __forceinline__ bool filter(Ctx c) const { return c != full; }
    __device__ __forceinline__ Acc identity() const { return 0ull; }
    __device__ __forceinline__ Acc edge(Ctx, int32_t u, int32_t) const { return fcur[u]; }
    __device__ __forceinline__ Acc combine(Acc a, Acc b) const { return a | b; }
    __device__ __forceinline__ bool stop(Acc a) const { return (a & full) == full; }
    __device__ __forceinline__ int finish(int32_t v, Ctx c, Acc a) const {
        u64 nm = a & ~c & full;
        if (!nm) return 0;
        fnext[v] = nm;
        visit[v] = c | nm;
        while (nm) {
            int i = __ffsll((long long)nm) - 1;
            nm &= nm - 1;
            depth[(int64_t)i * n + v] = level;
        }
        return 1;
    }
};

// after a PUSH round: newly reached bits become visited, depths written
__global__ void k_ms_commit(const int32_t *touched, int32_t cnt, u64 *visit, const u64 *fnext,
                            int32_t *depth, int32_t n, int32_t level) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = touched[i];
        u64 nm = fnext[v];
        visit[v] |= nm;
        while (nm) {
            int b = __ffsll((long long)nm) - 1;
            nm &= nm - 1;
            depth[(int64_t)b * n + v] = level;
        }
    }
}

__global__ void k_ms_clear(const int32_t *list, int32_t cnt, u64 *f) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        f[list[i]] = 0ull;
}

__global__ void k_ms_seed(const int32_t *srcs, int32_t k, u64 *visit, u64 *fcur, int32_t *depth,
                          int32_t n, int32_t *list, int32_t *cnt) {
    int i = threadIdx.x;
    if (i < k) {
        int32_t s = srcs[i];
        atomicOr(&visit[s], 1ull << i);
        u64 old = atomicOr(&fcur[s], 1ull << i);
        depth[(int64_t)i * n + s] = 0;
        if (old == 0) list[atomicAdd(cnt, 1)] = s;
    }
}

template <class Op>
__global__ void __launch_bounds__(kCta) k_ms_push(DevGraph g, FrontierIn fin, int32_t fsize, Op op,
                                                  OutCtx out, int lb, unsigned long long *ctr) {
    switch (lb) {
        case G2_LB_WM: lb_warp(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr); break;
        case G2_LB_CM: lb_cta(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr); break;
        case G2_LB_ETWC: lb_etwc(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr); break;
        default: lb_vertex(g, fin, fsize, op, out, blockIdx.x, gridDim.x, ctr); break;
    }
}

template <class P, int G>
__global__ void __launch_bounds__(kCta) k_ms_pull(DevGraph g, P op, OutCtx out,
                                                  unsigned long long *ctr) {
    Member all{MEM_ALL, nullptr, nullptr};
    lb_pull<P, G>(g, nullptr, g.n, all, op, out, blockIdx.x, gridDim.x, ctr);
}

// ------------------------------------------- multi-source BFS, fused
// The whole multi-source loop in one cooperative kernel (kernel fusion for
// the batch): per level a WM PUSH over the list of vertices whose frontier
// mask is non-zero, a grid barrier, the commit of the newly reached bits
// (visit masks, depths) together with clearing the spent frontier masks, and
// a second barrier.  Counters rotate over three words so that a level's
// count is read after the barrier that completed it and reset two levels
// ahead.
struct MsBfsFusedArgs {
    DevGraph g;
    u64 *visit;
    u64 *F[2];
    int32_t *list[2];
    int32_t *cnt;     // [3] rotating list lengths; cnt[0] = seeded sources
    int32_t *depth;   // [k][n]
    int32_t *levels;  // out
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;
};

__global__ void __launch_bounds__(kCta) k_ms_bfs_fused(MsBfsFusedArgs a) {
    const int32_t n = a.g.n;
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = OUT_SPARSE;
    out.dedup = DD_NONE;  // the first arc that turns a mask non-zero lists the vertex
    out.cap = n;
    out.err = a.err;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    int level = 1;
    for (;; ++level) {
        const int p = (level - 1) & 1, q = level & 1;
        const int32_t size = ld_relaxed_i32(a.cnt + (level - 1) % 3);
        if (size == 0) break;
        FrontierIn fin{a.list[p], size, nullptr};
        out.q = a.list[q];
        out.cnt = a.cnt + level % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[(level + 1) % 3] = 0;
        lb_warp(a.g, fin, size, OpMsBfs{a.visit, a.F[p], a.F[q]}, out, blockIdx.x, gridDim.x,
                nullptr);
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
        const int32_t nt_new = ld_relaxed_i32(a.cnt + level % 3);
        for (int64_t i = tid; i < nt_new; i += nt) {
            const int32_t v = a.list[q][i];
            u64 nm = a.F[q][v];
            a.visit[v] |= nm;
            while (nm) {
                const int b = __ffsll((long long)nm) - 1;
                nm &= nm - 1;
                a.depth[(int64_t)b * n + v] = level;
            }
        }
        for (int64_t i = tid; i < size; i += nt) a.F[p][a.list[p][i]] = 0ull;
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
    }
    if (tid == 0) *a.levels = level - 1;
}

static g2_status batch_lb(const g2_schedule &s) {
    if (s.load_balance < G2_LB_VERTEX_BASED || s.load_balance > G2_LB_TWC)
        return fail(G2_EINVAL, "bad load_balance");
    if (s.load_balance == G2_LB_EDGE_ONLY)
        return fail(G2_EUNSUPPORTED, "multi-source traversals are frontier-driven (no EDGE_ONLY)");
    if (s.direction == G2_PULL && s.load_balance != G2_LB_VERTEX_BASED &&
        s.load_balance != G2_LB_WM)
        return fail(G2_EUNSUPPORTED, "multi-source PULL supports VERTEX_BASED and WM");
    return G2_OK;
}

static g2_status bfs_batch_fused(g2_graph *g, const int32_t *srcs, int32_t k, int32_t *depth,
                                 const g2_schedule &sc, cudaStream_t st, int32_t *d_err) {
    if (sc.direction != G2_PUSH || sc.load_balance != G2_LB_WM)
        return fail(G2_EUNSUPPORTED, "the fused multi-source BFS runs WM PUSH rounds");
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    MsBfsFusedArgs a;
    a.g = t->view();
    int32_t *dsrc;
    G2_TRY(ws(g, B_MS0, (size_t)std::max(n, 1), &a.visit));
    G2_TRY(ws(g, B_MS1, (size_t)std::max(n, 1), &a.F[0]));
    G2_TRY(ws(g, B_MS2, (size_t)std::max(n, 1), &a.F[1]));
    G2_TRY(ws(g, B_Q0, (size_t)std::max(n, 1), &a.list[0]));
    G2_TRY(ws(g, B_Q1, (size_t)std::max(n, 1), &a.list[1]));
    G2_TRY(ws(g, B_I1, 64, &dsrc));
    G2_CK(cudaMemsetAsync(a.visit, 0, (size_t)n * 8, st));
    G2_CK(cudaMemsetAsync(a.F[0], 0, (size_t)n * 8, st));
    G2_CK(cudaMemsetAsync(a.F[1], 0, (size_t)n * 8, st));
    G2_CK(cudaMemsetAsync(depth, 0xFF, (size_t)k * n * 4, st));
    G2_TRY(put_array(dsrc, srcs, k, st));
    a.cnt = ctrs + 20;  // [20..22]; zero from begin_call
    a.levels = ctrs + 24;
    k_ms_seed<<<1, 64, 0, st>>>(dsrc, k, a.visit, a.F[0], depth, n, a.list[0], a.cnt);
    a.depth = depth;
    a.bar = GridBarrier{reinterpret_cast<unsigned long long *>(ctrs + 28)};
    a.err = d_err;
    a.limit_ns = barrier_limit_ns();
    stats().launches += 1;
    G2_TRY(launch_coop(g, k_ms_bfs_fused, a, st));
    G2_TRY(read_counters(g, ctrs + 24, 1, st, d_err));
    stats().iterations = g->h_ctr[0];
    stats().push_rounds = g->h_ctr[0];
    stats().barriers = 2 * g->h_ctr[0];
    return G2_OK;
}

g2_status bfs_batch_run(g2_graph *g, const int32_t *srcs, int32_t k, int32_t *depth,
                        const g2_hybrid &h, cudaStream_t st, int32_t *d_err) {
    if (h.s1.kernel_fusion) {
        if (h.criteria != G2_CRITERIA_NONE && !h.s2.kernel_fusion)
            return fail(G2_EUNSUPPORTED, "kernel fusion must be set on both hybrid schedules");
        return bfs_batch_fused(g, srcs, k, depth, h.s1, st, d_err);
    }
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    u64 *visit, *F[2];
    int32_t *list[2], *dsrc;
    G2_TRY(ws(g, B_MS0, (size_t)std::max(n, 1), &visit));
    G2_TRY(ws(g, B_MS1, (size_t)std::max(n, 1), &F[0]));
    G2_TRY(ws(g, B_MS2, (size_t)std::max(n, 1), &F[1]));
    G2_TRY(ws(g, B_Q0, (size_t)std::max(n, 1), &list[0]));
    G2_TRY(ws(g, B_Q1, (size_t)std::max(n, 1), &list[1]));
    G2_TRY(ws(g, B_I1, 64, &dsrc));
    G2_CK(cudaMemsetAsync(visit, 0, (size_t)n * 8, st));
    G2_CK(cudaMemsetAsync(F[0], 0, (size_t)n * 8, st));
    G2_CK(cudaMemsetAsync(F[1], 0, (size_t)n * 8, st));
    G2_CK(cudaMemsetAsync(depth, 0xFF, (size_t)k * n * 4, st));
    G2_TRY(put_array(dsrc, srcs, k, st));
    k_ms_seed<<<1, 64, 0, st>>>(dsrc, k, visit, F[0], depth, n, list[0], ctrs + 0);
    stats().launches += 1;
    G2_TRY(read_counters(g, ctrs, 4, st, d_err));
    int32_t size = g->h_ctr[0];
    const u64 full = k == 64 ? ~0ull : ((1ull << k) - 1);
    unsigned long long *ctr = nullptr;
    if (count_arcs_enabled()) G2_TRY(ws(g, B_ARCS, 2, &ctr));
    const DevGraph dg = t->view();
    int p = 0;
    for (int level = 1; size > 0; ++level) {
        const g2_schedule &s = pick_schedule(h, size, n);
        G2_TRY(batch_lb(s));
        int q = 1 - p;
        OutCtx out;
        memset(&out, 0, sizeof(out));
        out.mode = OUT_SPARSE;
        out.q = list[q];
        out.cnt = ctrs + q;
        out.cap = n;
        out.err = d_err;
        G2_CK(cudaMemsetAsync(ctrs + q, 0, 4, st));
        if (s.direction == G2_PUSH) {
            VSet in{OUT_SPARSE, list[p], n, ctrs + p, nullptr, nullptr, size};
            G2_TRY(push_round(g, s, OpMsBfs{visit, F[p], F[q]}, in, out, ctr, st));
            G2_TRY(read_counters(g, ctrs, 4, st, d_err));
            int32_t nt = g->h_ctr[q];
            if (nt > 0)
                k_ms_commit<<<grid_for(g, nt, kCta), kCta, 0, st>>>(list[q], nt, visit, F[q], depth,
                                                                   n, level);
            stats().push_rounds++;
            stats().launches += 2;
        } else {
            PullMsBfs op{visit, F[p], F[q], depth, n, level, full};
            if (s.load_balance == G2_LB_WM)
                k_ms_pull<PullMsBfs, 32><<<grid_for(g, (int64_t)n * 32, kCta), kCta, 0, st>>>(
                    dg, op, out, ctr);
            else
                k_ms_pull<PullMsBfs, 1><<<grid_for(g, n, kCta), kCta, 0, st>>>(dg, op, out, ctr);
            stats().pull_rounds++;
            stats().launches += 1;
        }
        // the current frontier masks become the (all-zero) next-next array
        k_ms_clear<<<grid_for(g, size, kCta), kCta, 0, st>>>(list[p], size, F[p]);
        stats().launches += 1;
        G2_TRY(read_counters(g, ctrs, 4, st, d_err));
        size = g->h_ctr[q];
        p = q;
        stats().iterations++;
    }
    return G2_OK;
}

// ------------------------------------------------------ multi-source SSSP
// Masks: M[p][v] = sources whose dist at v improved below the bucket
// threshold and wait to be relaxed; Far[v] = sources improved to a value at
// or above it.  Lists hold each vertex once (the first arc that turns its
// mask non-zero lists it).
struct OpMsRelax {
    int32_t *dist;  // [k][n]
    const int32_t *w;
    const unsigned *mcur;
    unsigned *mnext;
    unsigned *far;
    int32_t n;
    int32_t T;
    int32_t *err;
    typedef unsigned S;
    __device__ __forceinline__ S load(int32_t u) const { return mcur[u]; }
    __device__ __forceinline__ bool skip(S m) const { return m == 0; }
    __device__ __forceinline__ int relax(int32_t u, S mu, int32_t v, int32_t e) const {
        const int32_t wt = w[e];
        unsigned nb = 0, fb = 0;
        while (mu) {
            int i = __ffs(mu) - 1;
            mu &= mu - 1;
            int32_t du = dist[(int64_t)i * n + u];
            int64_t nd = (int64_t)du + wt;
            if (nd >= G2_INF32) {
                set_error(err, G2_EOVERFLOW);
                continue;
            }
            int32_t *dv = dist + (int64_t)i * n + v;
            if ((int32_t)nd < *dv) {
                int32_t old = atomicMin(dv, (int32_t)nd);
                if ((int32_t)nd < old) {
                    if ((int32_t)nd < T) nb |= 1u << i;
                    else fb |= 1u << i;
                }
            }
        }
        int code = 0;
        if (nb && atomicOr(&mnext[v], nb) == 0) code |= 1;
        if (fb && atomicOr(&far[v], fb) == 0) code |= 2;
        return code;
    }
};

__global__ void k_msr_far_min(const int32_t *flist, int32_t cnt, const unsigned *far,
                              const int32_t *dist, int32_t n, int32_t Told, int32_t *out) {
    int32_t best = G2_INF32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = flist[i];
        unsigned m = far[v];
        while (m) {
            int b = __ffs(m) - 1;
            m &= m - 1;
            int32_t d = dist[(int64_t)b * n + v];
            if (d >= Told && d < best) best = d;
        }
    }
    best = (int32_t)__reduce_min_sync(G2_FULL, (unsigned)best);
    if ((threadIdx.x & 31) == 0 && best != G2_INF32) atomicMin(out, best);
}

__global__ void k_msr_far_split(const int32_t *flist, int32_t cnt, unsigned *far,
                                const int32_t *dist, int32_t n, int32_t Told, int32_t Tnew,
                                unsigned *mnear, int32_t *nlist, int32_t *ncnt, int32_t *flist2,
                                int32_t *fcnt2, int32_t *err) {
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < cnt;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + (threadIdx.x & 31);
        int32_t v = 0;
        unsigned nb = 0, fb = 0;
        if (i < cnt) {
            v = flist[i];
            unsigned m = far[v];
            while (m) {
                int b = __ffs(m) - 1;
                m &= m - 1;
                int32_t d = dist[(int64_t)b * n + v];
                if (d < Told) continue;  // settled in an earlier bucket
                if (d < Tnew) nb |= 1u << b;
                else fb |= 1u << b;
            }
            far[v] = fb;
            if (nb) mnear[v] = nb;
        }
        warp_append(nlist, ncnt, n, err, v, nb != 0);
        warp_append(flist2, fcnt2, n, err, v, fb != 0);
    }
}

// ------------------------------------------ multi-source SSSP, fused
// The near/far loop of the multi-source relaxation in one cooperative kernel.
// Near round r pushes from list NL[r % 3] with masks M[r % 3] into
// NL[(r + 1) % 3] / M[(r + 1) % 3] (and the far pile), while the masks of
// round r - 1's input (M[(r + 2) % 3], listed in NL[(r + 2) % 3]) are
// cleared: three rotating buffers make one grid barrier per round enough.
// When a round produces nothing, the smallest far distance at or above the
// threshold picks the next bucket and the far pile is split as in the plain
// loop (two barriers per bucket).
struct MsSsspFusedArgs {
    DevGraph g;
    int32_t *dist;  // [k][n]
    unsigned *M[3];
    unsigned *far;
    int32_t *NL[3];
    int32_t *FL[2];
    int32_t *ncnt;    // [3]; ncnt[0] = seeded sources
    int32_t *fcnt;    // [2]
    int32_t *dmin;    // [2]; dmin[0] = G2_INF32 at launch
    int32_t *result;  // [0] near rounds, [1] buckets
    int32_t delta;    // 0: one bucket
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;
};

__global__ void __launch_bounds__(kCta) k_msr_fused(MsSsspFusedArgs a) {
    const int32_t n = a.g.n;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    const bool bucketed = a.delta > 0;
    int64_t T = bucketed ? a.delta : (int64_t)G2_INF32;
    int r = 0, fp = 0, epoch = 0;
    int32_t prev_size = 0;
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = OUT_SPARSE;
    out.dedup = DD_NONE;  // a vertex is listed when its mask turns non-zero
    out.cap = n;
    out.cap2 = n;
    out.err = a.err;
    for (;;) {
        for (;;) {
            const int ia = r % 3, ib = (r + 1) % 3, ic = (r + 2) % 3;
            const int32_t size = ld_relaxed_i32(a.ncnt + ia);
            if (size == 0) break;
            out.q = a.NL[ib];
            out.cnt = a.ncnt + ib;
            out.q2 = a.FL[fp];
            out.cnt2 = a.fcnt + fp;
            if (tid == 0) a.ncnt[ic] = 0;  // round r + 1's output count
            for (int64_t i = tid; i < prev_size; i += nt) a.M[ic][a.NL[ic][i]] = 0u;
            FrontierIn fin{a.NL[ia], size, nullptr};
            OpMsRelax op{a.dist, a.g.w, a.M[ia], a.M[ib], a.far, n,
                         (int32_t)(T < G2_INF32 ? T : G2_INF32), a.err};
            lb_warp(a.g, fin, size, op, out, blockIdx.x, gridDim.x, nullptr);
            if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
            prev_size = size;
            ++r;
        }
        const int32_t nfar = ld_relaxed_i32(a.fcnt + fp);
        if (!bucketed || nfar == 0) break;
        const int32_t Told = (int32_t)(T < G2_INF32 ? T : G2_INF32);
        // phase A: the smallest live far distance
        {
            int32_t best = G2_INF32;
            for (int64_t i = tid; i < nfar; i += nt) {
                const int32_t v = a.FL[fp][i];
                unsigned m = a.far[v];
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const int32_t d = a.dist[(int64_t)b * n + v];
                    if (d >= Told && d < best) best = d;
                }
            }
            best = (int32_t)__reduce_min_sync(G2_FULL, (unsigned)best);
            if ((threadIdx.x & 31) == 0 && best != G2_INF32) atomicMin(a.dmin + (epoch & 1), best);
            if (tid == 0) {
                a.fcnt[1 - fp] = 0;                 // the far pile of the next epoch
                a.dmin[(epoch + 1) & 1] = G2_INF32;  // its minimum
            }
        }
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
        const int32_t dmin = ld_relaxed_i32(a.dmin + (epoch & 1));
        if (dmin == G2_INF32) break;
        const int64_t Tnew = ((int64_t)dmin / a.delta + 1) * (int64_t)a.delta;
        const int32_t Tn = (int32_t)(Tnew < G2_INF32 ? Tnew : G2_INF32);
        // phase B: split the far pile into round r's near list and the next pile
        {
            const int ia = r % 3;
            for (int64_t base = tid & ~31LL; base < nfar; base += nt) {
                const int64_t i = base + (threadIdx.x & 31);
                int32_t v = 0;
                unsigned nb = 0, fb = 0;
                if (i < nfar) {
                    v = a.FL[fp][i];
                    unsigned m = a.far[v];
                    while (m) {
                        const int b = __ffs(m) - 1;
                        m &= m - 1;
                        const int32_t d = a.dist[(int64_t)b * n + v];
                        if (d < Told) continue;  // settled in an earlier bucket
                        if (d < Tn) nb |= 1u << b;
                        else fb |= 1u << b;
                    }
                    a.far[v] = fb;
                    if (nb) a.M[ia][v] = nb;
                }
                warp_append(a.NL[ia], a.ncnt + ia, n, a.err, v, nb != 0);
                warp_append(a.FL[1 - fp], a.fcnt + 1 - fp, n, a.err, v, fb != 0);
            }
        }
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
        fp = 1 - fp;
        T = Tnew;
        ++epoch;
    }
    if (tid == 0) {
        a.result[0] = r;
        a.result[1] = epoch;
    }
}

__global__ void k_msr_seed(const int32_t *srcs, int32_t k, int32_t *dist, int32_t n, unsigned *m,
                           int32_t *list, int32_t *cnt) {
    int i = threadIdx.x;
    if (i < k) {
        int32_t s = srcs[i];
        dist[(int64_t)i * n + s] = 0;
        if (atomicOr(&m[s], 1u << i) == 0) list[atomicAdd(cnt, 1)] = s;
    }
}

__global__ void k_msr_clear(const int32_t *list, int32_t cnt, unsigned *m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        m[list[i]] = 0u;
}

__global__ void k_fill_i32_b(int32_t *a, int64_t n, int32_t val) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        a[v] = val;
}

static g2_status sssp_batch_fused(g2_graph *g, const int32_t *srcs, int32_t k, int32_t delta,
                                  int32_t *dist, const g2_schedule &sc, cudaStream_t st,
                                  int32_t *d_err) {
    if (sc.direction != G2_PUSH || sc.load_balance != G2_LB_WM)
        return fail(G2_EUNSUPPORTED, "the fused multi-source SSSP runs WM PUSH rounds");
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    MsSsspFusedArgs a;
    a.g = t->view();
    a.dist = dist;
    int32_t *dsrc;
    int32_t *m2;
    G2_TRY(ws(g, B_F0, (size_t)std::max(n, 1), &a.M[0]));
    G2_TRY(ws(g, B_F1, (size_t)std::max(n, 1), &a.M[1]));
    G2_TRY(ws(g, B_STAMP, (size_t)std::max(n, 1), &m2));
    a.M[2] = reinterpret_cast<unsigned *>(m2);
    G2_TRY(ws(g, B_F2, (size_t)std::max(n, 1), &a.far));
    G2_TRY(ws(g, B_Q0, (size_t)std::max(n, 1), &a.NL[0]));
    G2_TRY(ws(g, B_Q1, (size_t)std::max(n, 1), &a.NL[1]));
    G2_TRY(ws(g, B_Q2, (size_t)std::max(n, 1), &a.NL[2]));
    G2_TRY(ws(g, B_Q3, (size_t)std::max(n, 1), &a.FL[0]));
    G2_TRY(ws(g, B_STAMP2, (size_t)std::max(n, 1), &a.FL[1]));
    G2_TRY(ws(g, B_I1, 64, &dsrc));
    for (int i = 0; i < 3; ++i) G2_CK(cudaMemsetAsync(a.M[i], 0, (size_t)n * 4, st));
    G2_CK(cudaMemsetAsync(a.far, 0, (size_t)n * 4, st));
    k_fill_i32_b<<<grid_for(g, (int64_t)k * n, kCta), kCta, 0, st>>>(dist, (int64_t)k * n, G2_INF32);
    G2_TRY(put_array(dsrc, srcs, k, st));
    a.ncnt = ctrs + 36;   // [36..38], zero from begin_call
    a.fcnt = ctrs + 39;   // [39..40]
    a.dmin = ctrs + 41;   // [41..42]
    a.result = ctrs + 43; // [43..44]
    const int32_t inf = G2_INF32;
    G2_TRY(put_i32(st, {{a.dmin, inf}}));
    k_msr_seed<<<1, 32, 0, st>>>(dsrc, k, dist, n, a.M[0], a.NL[0], a.ncnt);
    a.delta = delta;
    a.bar = GridBarrier{reinterpret_cast<unsigned long long *>(ctrs + 28)};
    a.err = d_err;
    a.limit_ns = barrier_limit_ns();
    stats().launches += 2;
    G2_TRY(launch_coop(g, k_msr_fused, a, st));
    G2_TRY(read_counters(g, ctrs + 43, 2, st, d_err));
    stats().iterations = g->h_ctr[0];
    stats().push_rounds = g->h_ctr[0];
    stats().barriers = g->h_ctr[0] + 2 * g->h_ctr[1];
    return G2_OK;
}

g2_status sssp_batch_run(g2_graph *g, const int32_t *srcs, int32_t k, int32_t delta, int32_t *dist,
                         const g2_hybrid &h, cudaStream_t st, int32_t *d_err) {
    if (h.s1.kernel_fusion) {
        if (h.criteria != G2_CRITERIA_NONE && !h.s2.kernel_fusion)
            return fail(G2_EUNSUPPORTED, "kernel fusion must be set on both hybrid schedules");
        return sssp_batch_fused(g, srcs, k, delta, dist, h.s1, st, d_err);
    }
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    unsigned *M[2], *far;
    int32_t *nl[2], *fl[2], *dsrc;
    G2_TRY(ws(g, B_F0, (size_t)std::max(n, 1), &M[0]));
    G2_TRY(ws(g, B_F1, (size_t)std::max(n, 1), &M[1]));
    G2_TRY(ws(g, B_F2, (size_t)std::max(n, 1), &far));
    G2_TRY(ws(g, B_Q0, (size_t)std::max(n, 1), &nl[0]));
    G2_TRY(ws(g, B_Q1, (size_t)std::max(n, 1), &nl[1]));
    G2_TRY(ws(g, B_Q2, (size_t)std::max(n, 1), &fl[0]));
    G2_TRY(ws(g, B_Q3, (size_t)std::max(n, 1), &fl[1]));
    G2_TRY(ws(g, B_I1, 64, &dsrc));
    G2_CK(cudaMemsetAsync(M[0], 0, (size_t)n * 4, st));
    G2_CK(cudaMemsetAsync(M[1], 0, (size_t)n * 4, st));
    G2_CK(cudaMemsetAsync(far, 0, (size_t)n * 4, st));
    k_fill_i32_b<<<grid_for(g, (int64_t)k * n, kCta), kCta, 0, st>>>(dist, (int64_t)k * n, G2_INF32);
    G2_TRY(put_array(dsrc, srcs, k, st));
    k_msr_seed<<<1, 32, 0, st>>>(dsrc, k, dist, n, M[0], nl[0], ctrs + 0);
    stats().launches += 2;
    G2_TRY(read_counters(g, ctrs, 8, st, d_err));
    int32_t size = g->h_ctr[0];
    unsigned long long *ctr = nullptr;
    if (count_arcs_enabled()) G2_TRY(ws(g, B_ARCS, 2, &ctr));
    const DevGraph dg = t->view();
    const bool bucketed = delta > 0;
    int64_t T = bucketed ? delta : (int64_t)G2_INF32;
    int p = 0, fp = 0;
    G2_CK(cudaMemsetAsync(ctrs + 4, 0, 8, st));
    for (;;) {
        while (size > 0) {
            const g2_schedule &s = pick_schedule(h, size, n);
            G2_TRY(batch_lb(s));
            if (s.direction != G2_PUSH)
                return fail(G2_EUNSUPPORTED, "multi-source SSSP relaxes in the PUSH direction");
            int q = 1 - p;
            OutCtx out;
            memset(&out, 0, sizeof(out));
            out.mode = OUT_SPARSE;
            out.q = nl[q];
            out.cnt = ctrs + q;
            out.cap = n;
            out.q2 = fl[fp];
            out.cnt2 = ctrs + 4 + fp;
            out.cap2 = n;
            out.err = d_err;
            G2_CK(cudaMemsetAsync(ctrs + q, 0, 4, st));
            VSet in{OUT_SPARSE, nl[p], n, ctrs + p, nullptr, nullptr, size};
            OpMsRelax op{dist, t->w, M[p], M[q], far, n, (int32_t)std::min<int64_t>(T, G2_INF32),
                         d_err};
            G2_TRY(push_round(g, s, op, in, out, ctr, st));
            k_msr_clear<<<grid_for(g, size, kCta), kCta, 0, st>>>(nl[p], size, M[p]);
            stats().launches += 2;
            stats().push_rounds++;
            stats().iterations++;
            G2_TRY(read_counters(g, ctrs, 8, st, d_err));
            size = g->h_ctr[q];
            p = q;
        }
        int32_t nfar = g->h_ctr[4 + fp];
        if (!bucketed || nfar == 0) break;
        int32_t Told = (int32_t)std::min<int64_t>(T, G2_INF32);
        int32_t inf = G2_INF32;
        G2_TRY(put_i32(st, {{ctrs + 6, inf}}));
        k_msr_far_min<<<grid_for(g, nfar, kCta), kCta, 0, st>>>(fl[fp], nfar, far, dist, n, Told,
                                                               ctrs + 6);
        G2_TRY(read_counters(g, ctrs, 8, st, d_err));
        int32_t dmin = g->h_ctr[6];
        if (dmin == G2_INF32) break;
        int64_t Tnew = ((int64_t)dmin / delta + 1) * (int64_t)delta;
        int nf = 1 - fp;
        G2_CK(cudaMemsetAsync(ctrs + p, 0, 4, st));
        G2_CK(cudaMemsetAsync(ctrs + 4 + nf, 0, 4, st));
        k_msr_far_split<<<grid_for(g, nfar, kCta), kCta, 0, st>>>(
            fl[fp], nfar, far, dist, n, Told, (int32_t)std::min<int64_t>(Tnew, G2_INF32), M[p],
            nl[p], ctrs + p, fl[nf], ctrs + 4 + nf, d_err);
        stats().launches += 2;
        G2_TRY(read_counters(g, ctrs, 8, st, d_err));
        size = g->h_ctr[p];
        fp = nf;
        T = Tnew;
        stats().barriers++;
    }
    return G2_OK;
}

}  // namespace g2

using namespace g2;

// Tuned schedules when the caller passes none: multi-source BFS switches from
// STRICT PUSH to VERTEX_BASED PULL once the union frontier holds 2% of the
// vertices; multi-source SSSP relaxes with STRICT PUSH.
// Tuned multi-source BFS: the direction-optimising hybrid (STRICT PUSH below
// 2% of n, VERTEX_BASED PULL); on a bounded-degree graph the fused WM PUSH
// loop (thousands of small levels: launches and host round trips dominate).
static g2_hybrid tuned_batch_bfs(g2_graph *g, cudaStream_t st) {
    int32_t dmax = 0;
    if (max_out_degree(g, st, &dmax) == G2_OK && dmax <= kBoundedDegree) {
        g2_hybrid h = default_hybrid();
        h.s1.load_balance = G2_LB_WM;
        h.s1.kernel_fusion = 1;
        h.s2 = h.s1;
        return h;
    }
    g2_hybrid h = default_hybrid();
    h.criteria = G2_INPUT_VERTEXSET_SIZE;
    h.threshold = 0.02f;
    h.s1.load_balance = G2_LB_STRICT;
    h.s2.load_balance = G2_LB_VERTEX_BASED;
    h.s2.direction = G2_PULL;
    return h;
}

// Tuned multi-source SSSP: STRICT PUSH; the fused WM PUSH loop on a
// bounded-degree graph.
static g2_hybrid tuned_batch_sssp(g2_graph *g, cudaStream_t st) {
    int32_t dmax = 0;
    if (max_out_degree(g, st, &dmax) == G2_OK && dmax <= kBoundedDegree) {
        g2_hybrid h = default_hybrid();
        h.s1.load_balance = G2_LB_WM;
        h.s1.kernel_fusion = 1;
        h.s2 = h.s1;
        return h;
    }
    g2_hybrid h = default_hybrid();
    h.s1.load_balance = G2_LB_STRICT;
    return h;
}

extern "C" {

g2_status g2_bfs_batch(g2_graph *g, const int32_t *srcs, int32_t k, int32_t *depth,
                       const g2_hybrid *sched, void *stream);
g2_status g2_sssp_batch(g2_graph *g, const int32_t *srcs, int32_t k, int32_t delta, int32_t *dist,
                        const g2_hybrid *sched, void *stream);

}  // extern "C"

namespace g2 {

// Split mode for the NULL schedule on a bounded-degree graph: the sources run
// as single-source fused queries, `workers` at a time, each on a view of the
// graph (its own workspace) and a stream of its own, driven by a host thread.
// A single-source fused loop keeps most levels of a road graph inside one
// 16-CTA thread-block cluster, so about nine of them fit on the GPU at once;
// on the 4096^2 road grid 64 BFS sources take 178 ms this way against 475 ms
// in one multi-source traversal (whose 64 wavefronts rarely meet, so it does
// the same vertex work with wider masks), and 32 SSSP sources 447 ms against
// 512 ms.  Outputs are row i of the caller's k x n array, as in the batched
// traversal.
static int split_workers(g2_graph *g, int32_t k, int per_sm_default) {
    int w = std::max(1, g->topo->sm_count / per_sm_default);
    if (const char *e = getenv("G2_BATCH_SPLIT_WORKERS")) w = atoi(e);
    return std::min(w, (int)k);
}

static g2_status split_run(g2_graph *g, const int32_t *srcs, int32_t k, int32_t delta, int32_t *out,
                           int workers, cudaStream_t st) {
    Topology *t = g->topo;
    const int64_t n = t->n;
    G2_CK(cudaStreamSynchronize(st));  // the caller's earlier work on its stream comes first
    std::vector<g2_graph *> views(workers, nullptr);
    std::vector<cudaStream_t> streams(workers, nullptr);
    g2_status made = G2_OK;
    for (int i = 0; i < workers && made == G2_OK; ++i) {
        made = g2_graph_view(g, &views[i]);
        if (made == G2_OK && cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess)
            made = fail(G2_ECUDA, "stream for a split batch");
    }
    struct Res {
        g2_status s = G2_OK;
        std::string msg;
        int64_t launches = 0, iterations = 0, barriers = 0;
    };
    std::vector<Res> res(workers);
    if (made == G2_OK) {
        const int dev = t->device;
        std::vector<std::thread> th;
        for (int w = 0; w < workers; ++w)
            th.emplace_back([&, w]() {
                cudaSetDevice(dev);
                for (int32_t i = w; i < k && res[w].s == G2_OK; i += workers) {
                    g2_status r = delta > 0
                                      ? g2_sssp_delta(views[w], srcs[i], delta, out + i * n, nullptr,
                                                      streams[w])
                                      : g2_bfs(views[w], srcs[i], out + i * n, nullptr, nullptr,
                                               streams[w]);
                    g2_stats st_w;
                    g2_last_stats(&st_w);
                    res[w].launches += st_w.launches;
                    res[w].iterations += st_w.iterations;
                    res[w].barriers += st_w.barriers;
                    if (r != G2_OK) {
                        res[w].s = r;
                        res[w].msg = g2_last_error();
                    }
                }
            });
        for (auto &x : th) x.join();
    }
    for (int i = 0; i < workers; ++i) {
        if (streams[i]) cudaStreamDestroy(streams[i]);
        if (views[i]) g2_free_graph(views[i]);
    }
    G2_TRY(made);
    for (const Res &r : res) {
        stats().launches += (int32_t)r.launches;
        stats().iterations += (int32_t)r.iterations;
        stats().barriers += (int32_t)r.barriers;
    }
    for (const Res &r : res)
        if (r.s != G2_OK) return fail(r.s, "split batch: " + r.msg);
    return G2_OK;
}

}  // namespace g2

extern "C" {

g2_status g2_bfs_batch(g2_graph *g, const int32_t *srcs, int32_t k, int32_t *depth,
                       const g2_hybrid *sched, void *stream) {
    if (!g || !depth || !srcs || k < 1 || k > 64) return fail(G2_EINVAL, "need 1 <= k <= 64 sources");
    for (int32_t i = 0; i < k; ++i)
        if (srcs[i] < 0 || srcs[i] >= g->topo->n) return fail(G2_EINVAL, "source out of range");
    if ((int64_t)k * g->topo->n >= (int64_t)1 << 40) return fail(G2_EINVAL, "output too large");
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : tuned_batch_bfs(g, st);
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    if (!sched && h.s1.kernel_fusion && k >= 2) {
        const int workers = split_workers(g, k, 12);
        if (workers >= 2) {
            G2_TRY(split_run(g, srcs, k, 0, depth, workers, st));
            return end_call(g, st, d_err);
        }
    }
    G2_TRY(bfs_batch_run(g, srcs, k, depth, h, st, d_err));
    return end_call(g, st, d_err);
}

g2_status g2_sssp_batch(g2_graph *g, const int32_t *srcs, int32_t k, int32_t delta, int32_t *dist,
                        const g2_hybrid *sched, void *stream) {
    if (!g || !dist || !srcs || k < 1 || k > 32) return fail(G2_EINVAL, "need 1 <= k <= 32 sources");
    if (!g->topo->w) return fail(G2_EINVAL, "SSSP needs arc weights");
    for (int32_t i = 0; i < k; ++i)
        if (srcs[i] < 0 || srcs[i] >= g->topo->n) return fail(G2_EINVAL, "source out of range");
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : tuned_batch_sssp(g, st);
    if (delta <= 0 && h.s1.delta > 0) delta = h.s1.delta;
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    if (!sched && h.s1.kernel_fusion && k >= 2) {
        const int workers = split_workers(g, k, 19);
        if (workers >= 2) {
            G2_TRY(split_run(g, srcs, k, delta > 0 ? delta : 1, dist, workers, st));
            return end_call(g, st, d_err);
        }
    }
    G2_TRY(sssp_batch_run(g, srcs, k, delta, dist, h, st, d_err));
    return end_call(g, st, d_err);
}

}  // extern "C"
