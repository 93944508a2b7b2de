// g2_async.cu — asynchronous SSSP and BFS for high-diameter graphs.
//
// Sec. VII-A and Table VII: on road graphs the GPU's delta-stepping loses to
// a 24-core CPU, because every bucket, and every near round inside it, ends
// at a barrier while the frontier holds a few thousand vertices.  Here the
// relaxations inside a bucket run without any barrier: one persistent kernel
// relaxes the out-arcs of the vertices in a shared worklist until nothing is
// pending; only the step to the next bucket synchronises the grid.  A bucket
// width of INT32_MAX (delta <= 0 from the caller) leaves one bucket: fully
// asynchronous relaxation.
//
//  * Worklist: a linear array of slots (-1 = not written yet) with a claim
//    counter (head) and an append counter (tail).  A warp claims 32
//    consecutive slots with one atomic; each lane waits (bounded in time)
//    until its slot is written, then relaxes that vertex's out-arcs with
//    atomicMin on the distances.  Claims may run ahead of the appends; when
//    a bucket ends, the claim counter is set back to the append counter, so
//    the slots claimed but never written serve the next bucket.
//  * A vertex is in the worklist at most once at a time (a bit per vertex,
//    set when it is appended, cleared when it is taken, before its distance
//    is read): an improvement that arrives while it waits is picked up when
//    it is processed, one that arrives after appends it again.
//  * Improvements at or beyond the bucket's threshold T go to a far pile
//    (once per pile, by stamps).  When the bucket is done, the smallest live
//    far distance picks the next threshold and the pile is split: entries
//    below it are appended to the worklist, the rest form the next pile,
//    entries already settled are dropped.
//  * Quiescence of a bucket: `pending` counts appended items whose processing
//    has not finished (an item's own appends are counted before its
//    decrement).  It reaches zero exactly when no item of the bucket is
//    queued or being processed; every waiting lane then leaves.
//  * Every wait is bounded (G2_ETIMEOUT after the limit); appends beyond the
//    worklist's capacity record G2_EOVERFLOW and the host runs the kernel
//    again with four times the capacity.
//
// Distances are unique, so the result is independent of the order in which
// the relaxations happen; BFS is the same kernel with unit weights, and its
// canonical parent (the smallest in-neighbour one level up) is taken by a
// pull pass over the final depths.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "g2_host.h"

namespace g2 {
namespace {

struct AsyncArgs {
    DevGraph g;
    int32_t *dist;              // distances (depths for BFS)
    uint32_t *inq;              // a bit per vertex: in the worklist
    int32_t *wl;                // worklist slots
    int64_t cap;                // appends allowed (slots beyond are for claims)
    unsigned long long *ctr;    // [0] head (claimed), [1] tail (appended), [2] pending,
                                // [3] items processed, [4] buckets
    int32_t *fq[2];             // far piles (n entries each)
    int32_t *fcnt;              // [2] far pile lengths
    int32_t *dmin;              // [2] smallest live far distance per epoch parity
    int32_t *stamp;             // far pile stamp per vertex (the epoch it was added in)
    int32_t delta;              // bucket width (G2_INF32: one bucket)
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;          // longest wait for one slot or barrier
    int unit;                   // 1: unit weights (BFS)
    unsigned nap_max;           // longest sleep of an idle warp between polls (ns)
};

__device__ __forceinline__ void st_release_i32(int32_t *p, int32_t v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_acquire_i32(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void k_async_init(int32_t *dist, uint32_t *inq, int32_t *wl, int64_t slots, int32_t n,
                             int32_t src, unsigned long long *ctr, int32_t *stamp, int32_t *fcnt,
                             int32_t *dmin, unsigned long long *bar) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t v = i0; v < n; v += stride) {
        dist[v] = v == src ? 0 : G2_INF32;
        stamp[v] = -1;
    }
    for (int64_t w = i0; w < ((int64_t)n + 31) / 32; w += stride)
        inq[w] = w == (src >> 5) ? 1u << (src & 31) : 0u;
    for (int64_t i = i0; i < slots; i += stride) wl[i] = i == 0 ? src : -1;
    if (i0 == 0) {
        ctr[0] = 0;  // head
        ctr[1] = 1;  // tail: the source is appended
        ctr[2] = 1;  // pending
        ctr[3] = 0;  // processed
        ctr[4] = 0;  // buckets
        fcnt[0] = fcnt[1] = 0;
        dmin[0] = dmin[1] = G2_INF32;
        *bar = 0;
    }
}

// Append the lanes' vertices u (where `push`, their bits already set) to the
// worklist: one reservation for the warp, counted as pending first, so that
// the count never reaches zero while an append is under way.  Every lane of
// the warp calls it.
__device__ __forceinline__ void async_append_warp(const AsyncArgs &a, bool push, int32_t u) {
    const unsigned pm = __ballot_sync(G2_FULL, push);
    if (!pm) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) {
        atomicAdd(a.ctr + 2, (unsigned long long)__popc(pm));
        base = atomicAdd(a.ctr + 1, (unsigned long long)__popc(pm));
    }
    base = __shfl_sync(G2_FULL, base, 0);
    if (push) {
        const unsigned long long p = base + __popc(pm & lanemask_lt());
        if ((int64_t)p < a.cap) st_release_i32(a.wl + p, u);
        else set_error(a.err, G2_EOVERFLOW);
    }
}

// Append to far pile fp, one reservation for the warp.  Every lane calls it.
__device__ __forceinline__ void async_far_warp(const AsyncArgs &a, bool far, int32_t u, int32_t fp) {
    const unsigned fm = __ballot_sync(G2_FULL, far);
    if (!fm) return;
    const int lane = threadIdx.x & 31;
    int32_t base = 0;
    if (lane == 0) base = atomicAdd(a.fcnt + fp, __popc(fm));
    base = __shfl_sync(G2_FULL, base, 0);
    if (far) {
        const int32_t p = base + __popc(fm & lanemask_lt());
        if (p < a.g.n) a.fq[fp][p] = u;
        else set_error(a.err, G2_EOVERFLOW);
    }
}

// Relax arc k (where `act`) from a vertex at distance dv: a lowered distance
// below T queues the head (once), one at or beyond T puts it on the far pile
// (once per epoch).  Every lane of the warp calls it.
__device__ __forceinline__ void async_relax_arc(const AsyncArgs &a, bool act, int32_t k, int32_t dv,
                                                int32_t T, int32_t fp, int32_t epoch) {
    int code = 0;  // 1: queue, 2: far pile
    int32_t u = 0;
    if (act) {
        u = a.g.col[k];
        const int32_t w = a.unit ? 1 : a.g.w[k];
        if (dv > G2_INF32 - 1 - w) {
            set_error(a.err, G2_EOVERFLOW);  // a distance would reach INT32_MAX
        } else {
            const int32_t nd = dv + w;
            if (nd < ld_relaxed_i32(a.dist + u) && nd < atomicMin(a.dist + u, nd))
                code = nd >= T ? 2 : 1;
        }
    }
    async_far_warp(a, code == 2 && atomicExch(a.stamp + u, epoch) != epoch, u, fp);
    if (__any_sync(G2_FULL, code == 1)) {
        __threadfence();  // the lowered distances are visible before their vertices are queued
        const uint32_t bit = 1u << (u & 31);
        async_append_warp(a, code == 1 && !(atomicOr(&a.inq[u >> 5], bit) & bit), u);
    }
}

// Process the lanes' items v (where `have`): clear each bit, read the
// distance, relax the out-arcs -- lists of up to 32 arcs with a lane each in
// lock step, longer ones by the whole warp -- then retire the items.
// Every lane of the warp calls it.
__device__ __forceinline__ void async_process_warp(const AsyncArgs &a, bool have, int32_t v,
                                                   int32_t T, int32_t fp, int32_t epoch) {
    const int lane = threadIdx.x & 31;
    if (have) atomicAnd(&a.inq[v >> 5], ~(1u << (v & 31)));
    __threadfence();  // the bits are clear before the distances are read
    int32_t dv = 0, b = 0, e = 0;
    if (have) {
        dv = ld_relaxed_i32(a.dist + v);
        b = a.g.rowptr[v];
        e = a.g.rowptr[v + 1];
    }
    const int32_t deg = e - b;
    const bool small = have && deg <= 32;
    const int32_t kmax = (int32_t)__reduce_max_sync(G2_FULL, small ? (unsigned)deg : 0u);
    for (int32_t k = 0; k < kmax; ++k)
        async_relax_arc(a, small && k < deg, b + k, dv, T, fp, epoch);
    unsigned big = __ballot_sync(G2_FULL, have && deg > 32);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const int32_t vb = __shfl_sync(G2_FULL, b, src), ve = __shfl_sync(G2_FULL, e, src);
        const int32_t vd = __shfl_sync(G2_FULL, dv, src);
        for (int32_t k0 = vb; k0 < ve; k0 += 32)
            async_relax_arc(a, k0 + lane < ve, k0 + lane, vd, T, fp, epoch);
    }
    __threadfence();  // the items' appends are counted before they retire
    const unsigned hm = __ballot_sync(G2_FULL, have);
    if (lane == 0 && hm) atomicAdd(a.ctr + 2, (unsigned long long)(0ull - __popc(hm)));
}

// One bucket: the warp claims 32 slots, processes them as they are written
// (lane 0 watches the append counter for the warp), claims again; it leaves
// once nothing is pending (or on an error).
__device__ __forceinline__ void async_bucket(const AsyncArgs &a, int32_t T, int32_t fp,
                                             int32_t epoch, unsigned &processed) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.ctr, 32ull);
        base = __shfl_sync(G2_FULL, base, 0);
        const unsigned long long idx = base + lane;
        bool done = false;  // this lane's slot has been processed
        unsigned nap = 32;
        uint64_t t0 = 0;
        for (;;) {
            unsigned long long tl = 0;
            if (lane == 0) tl = ld_relaxed_u64(a.ctr + 1);
            tl = __shfl_sync(G2_FULL, tl, 0);
            int32_t v = -1;
            if (!done && idx < tl) {
                // reserved: its write follows the reservation closely
                for (unsigned spins = 0; (v = ld_acquire_i32(a.wl + idx)) < 0; ++spins) {
                    if (spins > (1u << 20)) {
                        set_error(a.err, G2_ETIMEOUT);
                        break;
                    }
                }
            }
            const bool have = v >= 0;
            if (__any_sync(G2_FULL, have)) {
                async_process_warp(a, have, v, T, fp, epoch);
                processed += have;
                done |= have;
                nap = 32;
                t0 = 0;
                if (__all_sync(G2_FULL, done)) break;
                continue;
            }
            // nothing new for this warp: leave if nothing is pending, else wait
            int stop = 0;
            if (lane == 0) {
                if (ld_relaxed_u64(a.ctr + 2) == 0ull || ld_relaxed_i32(a.err) != 0) {
                    stop = 1;
                } else {
                    const uint64_t now = globaltimer_ns();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > a.limit_ns) {
                        set_error(a.err, G2_ETIMEOUT);
                        stop = 1;
                    }
                }
            }
            if (__shfl_sync(G2_FULL, stop, 0)) return;
            __nanosleep(nap);
            nap = nap < a.nap_max ? nap * 2 : a.nap_max;
        }
    }
}

__global__ void __launch_bounds__(kCta) k_async_relax(AsyncArgs a) {
    const int lane = threadIdx.x & 31;
    unsigned processed = 0;
    int32_t T = a.delta, fp = 0, epoch = 0, buckets = 0;
    for (;;) {
        async_bucket(a, T, fp, epoch, processed);
        if (!grid_sync(a.bar, a.err, a.limit_ns)) break;
        // the bucket is done: nothing is queued, every bit is clear
        const int32_t nfar = ld_relaxed_i32(a.fcnt + fp);
        if (nfar == 0) break;
        const int32_t Told = T;
        int32_t *dm = a.dmin + (epoch & 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            // claims past the last append were never written: serve the next bucket
            a.ctr[0] = a.ctr[1];
            a.fcnt[1 - fp] = 0;
            a.dmin[1 - (epoch & 1)] = G2_INF32;
        }
        {
            int32_t best = G2_INF32;
            for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nfar;
                 i += (int64_t)gridDim.x * blockDim.x) {
                const int32_t dv = a.dist[a.fq[fp][i]];
                if (dv >= Told && dv < best) best = dv;
            }
            best = (int32_t)__reduce_min_sync(G2_FULL, (unsigned)best);
            if (lane == 0 && best != G2_INF32) atomicMin(dm, best);
        }
        if (!grid_sync(a.bar, a.err, a.limit_ns)) break;
        const int32_t dmin = ld_relaxed_i32(dm);
        if (dmin == G2_INF32) break;
        const int64_t Tnew = ((int64_t)dmin / a.delta + 1) * (int64_t)a.delta;
        const int32_t Tn = (int32_t)(Tnew < G2_INF32 ? Tnew : G2_INF32);
        // split the pile: [Told, Tn) to the worklist, the rest to the next
        // pile (a warp at a time, so the appends are aggregated)
        for (int64_t b0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; b0 < nfar;
             b0 += (int64_t)gridDim.x * blockDim.x) {
            const int64_t i = b0 + lane;
            int32_t v = 0, dv = G2_INF32;
            if (i < nfar) {
                v = a.fq[fp][i];
                dv = a.dist[v];
            }
            const bool to_near = i < nfar && dv >= Told && dv < Tn;
            const bool to_far = i < nfar && dv >= Tn;
            if (to_near) atomicOr(&a.inq[v >> 5], 1u << (v & 31));
            if (to_far) a.stamp[v] = epoch + 1;
            async_append_warp(a, to_near, v);
            async_far_warp(a, to_far, v, 1 - fp);
        }
        if (!grid_sync(a.bar, a.err, a.limit_ns)) break;
        fp = 1 - fp;
        ++epoch;
        ++buckets;
        T = Tn;
    }
    processed = __reduce_add_sync(G2_FULL, processed);
    if (lane == 0 && processed) atomicAdd(a.ctr + 3, (unsigned long long)processed);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctr[4] = (unsigned long long)buckets + 1;
}

// parent[v] = the smallest in-neighbour u with depth[u] == depth[v] - 1
// (parent[src] = src, -1 unreached); CSC lists are ascending, so the first hit
__global__ void k_async_parent(const int32_t *crowptr, const int32_t *ccol, const int32_t *depth,
                               int32_t n, int32_t src, int32_t *parent) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t dv = depth[v];
        int32_t p = -1;
        if (v == src) {
            p = src;
        } else if (dv > 0) {
            for (int32_t k = crowptr[v]; k < crowptr[v + 1]; ++k)
                if (depth[ccol[k]] == dv - 1) {
                    p = ccol[k];
                    break;
                }
        }
        parent[v] = p;
    }
}

__global__ void k_async_unreached(int32_t *depth, int32_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (depth[v] == G2_INF32) depth[v] = -1;
}

// The whole asynchronous loop; dist as SSSP leaves it (INT32_MAX unreached).
g2_status async_run(g2_graph *g, int32_t src, int32_t delta, int32_t *dist, bool unit,
                    cudaStream_t st, int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    int per_sm = 0;
    G2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_async_relax, kCta, 0));
    if (per_sm < 1) return fail(G2_EUNSUPPORTED, "asynchronous kernel does not fit on an SM");
    // Fewer warps wait better: every idle warp holds a claim and polls, and
    // on the 4096^2 road grid half the SMs with one CTA each measured best
    // (delta 8192: 81 ms against 88 ms on every SM, 128 ms with two CTAs per
    // SM, 212 ms with four).  G2_ASYNC_CTAS / G2_ASYNC_CTAS_PER_SM override.
    int want = 1;
    if (const char *e = getenv("G2_ASYNC_CTAS_PER_SM")) want = std::max(1, atoi(e));
    per_sm = std::min(per_sm, want);
    int grid = std::max(1, per_sm * t->sm_count / (want == 1 ? 2 : 1));
    if (const char *e = getenv("G2_ASYNC_CTAS"))
        grid = std::max(1, std::min(per_sm * t->sm_count, atoi(e)));
    const int64_t warps = (int64_t)grid * (kCta / 32);
    uint32_t *inq;
    int32_t *small, *stamp, *fq0, *fq1;
    G2_TRY(ws(g, B_DDBM, ((size_t)n + 31) / 32 + 1, &inq));
    G2_TRY(ws(g, B_SCAN, 32, &small));  // counters (5 x u64), far lengths, minima, barrier
    G2_TRY(ws(g, B_STAMP2, (size_t)n, &stamp));
    G2_TRY(ws(g, B_Q0, (size_t)n, &fq0));
    G2_TRY(ws(g, B_Q1, (size_t)n, &fq1));
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(small);
    int32_t *fcnt = small + 12, *dmin = small + 14;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(small + 16);
    int64_t factor = 4;
    if (const char *e = getenv("G2_ASYNC_CAP")) factor = std::max(1, atoi(e));
    for (;;) {
        // appends allowed, plus one claim of 32 slots per warp beyond them
        const int64_t cap = factor * (int64_t)n + 1024;
        const int64_t slots = cap + 32 * warps + 32;
        int32_t *wl;
        G2_TRY(ws(g, B_BIG, (size_t)slots, &wl));
        G2_CK(cudaMemsetAsync(d_err, 0, sizeof(int32_t), st));
        k_async_init<<<grid_for(g, std::max<int64_t>(slots, n), kCta), kCta, 0, st>>>(
            dist, inq, wl, slots, n, src, ctr, stamp, fcnt, dmin, bar);
        AsyncArgs a;
        a.g = t->view();
        a.dist = dist;
        a.inq = inq;
        a.wl = wl;
        a.cap = cap;
        a.ctr = ctr;
        a.fq[0] = fq0;
        a.fq[1] = fq1;
        a.fcnt = fcnt;
        a.dmin = dmin;
        a.stamp = stamp;
        a.delta = delta;
        a.bar = GridBarrier{bar};
        a.err = d_err;
        a.limit_ns = barrier_limit_ns();
        a.unit = unit ? 1 : 0;
        a.nap_max = 1024;
        if (const char *e = getenv("G2_ASYNC_NAP_NS")) a.nap_max = (unsigned)std::max(32, atoi(e));
        void *params[] = {&a};
        G2_CK(cudaLaunchCooperativeKernel((const void *)k_async_relax, dim3(grid), dim3(kCta),
                                          params, 0, st));
        stats().launches += 2;
        unsigned long long h[5];
        G2_CK(cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st));
        G2_CK(cudaMemcpyAsync(g->h_ctr, d_err, 4, cudaMemcpyDeviceToHost, st));
        G2_CK(cudaStreamSynchronize(st));
        stats().iterations = (int32_t)std::min<unsigned long long>(h[3], 2147483647ull);
        stats().barriers = (int32_t)std::min<unsigned long long>(3 * h[4], 2147483647ull);
        if (g->h_ctr[0] == G2_EOVERFLOW && (int64_t)h[1] > cap && factor < 256) {
            factor *= 4;  // the worklist ran out: again with more room
            continue;
        }
        return G2_OK;  // other device errors are reported by end_call
    }
}

g2_status check_async_args(g2_graph *g, int32_t src, const void *out) {
    if (!g || !out) return fail(G2_EINVAL, "null graph or output");
    if (src < 0 || src >= g->topo->n) return fail(G2_EINVAL, "source out of range");
    return G2_OK;
}

}  // namespace
}  // namespace g2

using namespace g2;

extern "C" g2_status g2_sssp_async(g2_graph *g, int32_t src, int32_t delta, int32_t *dist,
                                   void *stream) {
    G2_TRY(check_async_args(g, src, dist));
    if (!g->topo->w) return fail(G2_EINVAL, "SSSP needs arc weights");
    cudaStream_t st = as_stream(stream);
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    G2_TRY(async_run(g, src, delta > 0 ? delta : G2_INF32, dist, false, st, d_err));
    return end_call(g, st, d_err);
}

extern "C" g2_status g2_bfs_async(g2_graph *g, int32_t src, int32_t delta, int32_t *depth,
                                  int32_t *parent, void *stream) {
    G2_TRY(check_async_args(g, src, depth));
    cudaStream_t st = as_stream(stream);
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    G2_TRY(async_run(g, src, delta > 0 ? delta : G2_INF32, depth, true, st, d_err));
    Topology *t = g->topo;
    const int grid = grid_for(g, t->n, kCta);
    if (parent) {
        k_async_parent<<<grid, kCta, 0, st>>>(t->crowptr, t->ccol, depth, t->n, src, parent);
        stats().launches += 1;
    }
    k_async_unreached<<<grid, kCta, 0, st>>>(depth, t->n);
    stats().launches += 1;
    G2_CK(cudaGetLastError());
    return end_call(g, st, d_err);
}
