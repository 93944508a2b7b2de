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

#include "g2_cluster.cuh"
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
    int32_t *cnt;      // [3] rotating list lengths; cnt[d0 % 3] > 0 at launch
    int32_t d0;        // first round (its frontier is list d0 & 1)
    int32_t lo;        // after the first round, stop before a level with fewer vertices
    int32_t *result;   // [0] level reached, [1] 1 if stopped for the cluster loop
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;
    unsigned long long *ctr;
};

// One launch for the BFS rounds from d0 on.  Round d reads list d&1 (length
// cnt[d%3]) and appends to list (d+1)&1 (length cnt[(d+1)%3]); cnt[(d+2)%3],
// read in round d-1 only, is cleared for round d+1.  One barrier per round.
// Every CTA reads the same length after the barrier, so all stop together:
// at an empty level (the search is done) or, after the first round, at a
// level smaller than `lo` (the one-cluster loop takes it over).
template <int LB>
__global__ void __launch_bounds__(kCta) k_bfs_fused(FusedBfsArgs a) {
    OpBFS op{a.depth, a.parent};
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = OUT_SPARSE;
    out.dedup = DD_NONE;  // the compare-and-swap on depth admits each vertex once
    out.cap = a.g.n;
    out.err = a.err;
    int d = a.d0;
    int handover = 0;
    for (;; ++d) {
        int32_t size = ld_relaxed_i32(a.cnt + d % 3);
        if (size == 0) break;
        if (size < a.lo && d > a.d0) {
            handover = 1;
            break;
        }
        FrontierIn fin{a.q[d & 1], size, nullptr};
        out.q = a.q[(d + 1) & 1];
        out.cnt = a.cnt + (d + 1) % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt[(d + 2) % 3] = 0;
        run_lb<LB>(a.g, fin, size, op, out, a.ctr);
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.result[0] = d;
        a.result[1] = handover;
    }
}

// ------------------------------------------------- fused direction-optimising BFS
// The hybrid of Table III inside one launch (kernel fusion, Sec. VI-C, over a
// direction-optimising schedule): a level below `push_below` vertices runs
// PUSH with load balancing LB from a sparse list, a larger one runs PULL
// (VERTEX_BASED, a thread per vertex scanning its ascending in-list until the
// first in-frontier neighbour, the canonical parent) over a bitmap of the
// frontier.  A PUSH level's output is a list, a PULL level's a bitmap (each
// word stored by the one warp that owns its 32 vertices, so it needs no
// clearing) with its population; the representation is converted where the
// direction changes.  Rotating counters as in k_bfs_fused: at the start of
// level d, cnt[(d+1)%3] and bcnt[(d+1)%3] are zero and cnt[(d+2)%3],
// bcnt[(d+2)%3] are cleared for level d+1.  Every CTA reads the same counts
// after a barrier, so all take the same branches.
struct FusedDoBfsArgs {
    DevGraph g;
    int32_t *depth;
    int32_t *parent;
    int32_t *q[2];
    int32_t *cnt;        // [3] list lengths; cnt[0] = 1 (the source) at launch, the rest 0
    uint32_t *bm[2];     // frontier bitmaps, (n + 31) / 32 words each
    int32_t *bcnt;       // [3] bitmap populations, 0 at launch
    int32_t push_below;  // PUSH while the frontier holds fewer vertices
    int32_t *scan;       // STRICT: prefix sums of a PUSH level's degrees (n + 1) ...
    int32_t *ctasum;     // ... and the slice totals of the CTAs (one per CTA)
    EtwcEntry<int32_t> *spq;  // ETWC: a level's entries of kEtwcSpill arcs or more ...
    int32_t *spcnt;           // ... and their counts per level parity, 0 at launch
    int32_t *result;     // [0] levels, [1] PULL levels
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;
    unsigned long long *ctr;
};

// STRICT inside a fused loop: scan[i] = the degrees of list entries before i
// and scan[size] = their sum, over the whole grid in two phases separated by
// barriers (each CTA scans an equal slice of the list and leaves its total,
// then adds the totals of the slices before its own).  False: a barrier
// wait gave up (the error word says why).
__device__ bool fused_strict_scan(const DevGraph &g, const int32_t *q, int32_t size,
                                  int32_t *scan, int32_t *ctasum, const GridBarrier &bar,
                                  int32_t *err, uint64_t limit_ns) {
    __shared__ int s_warp[kWarps];
    __shared__ int s_part[kWarps];
    const int bid = blockIdx.x, nb = gridDim.x;
    const int32_t i0 = (int32_t)((int64_t)size * bid / nb);
    const int32_t i1 = (int32_t)((int64_t)size * (bid + 1) / nb);
    int run = 0;
    for (int32_t t = i0; t < i1; t += kCta) {
        const int32_t i = t + (int32_t)threadIdx.x;
        int dg = 0;
        if (i < i1) {
            const int32_t u = q[i];
            dg = g.rowptr[u + 1] - g.rowptr[u];
        }
        int tot;
        const int incl = block_incl_scan(dg, s_warp, &tot);
        if (i < i1) scan[i] = run + incl - dg;
        run += tot;
        __syncthreads();  // s_warp is read above before the next tile writes it
    }
    if (threadIdx.x == 0) ctasum[bid] = run;
    if (!grid_sync(bar, err, limit_ns)) return false;
    int part = 0;
    for (int j = threadIdx.x; j < bid; j += kCta) part += ctasum[j];
    part = __reduce_add_sync(G2_FULL, (unsigned)part);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = part;
    __syncthreads();
    int off = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) off += s_part[w];
    for (int32_t i = i0 + (int32_t)threadIdx.x; i < i1; i += kCta) scan[i] += off;
    if (bid == nb - 1 && threadIdx.x == 0) scan[size] = off + run;
    return grid_sync(bar, err, limit_ns);
}

template <int LB>
__global__ void __launch_bounds__(kCta) k_bfs_fused_do(FusedDoBfsArgs a) {
    OpBFS op{a.depth, a.parent};
    PullBFS pop{a.depth, a.parent};
    const int lane = threadIdx.x & 31;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = gt >> 5, nwarps = nt >> 5;
    const int32_t n = a.g.n;
    const int32_t words = (n + 31) / 32;
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = OUT_SPARSE;
    out.dedup = DD_NONE;  // the compare-and-swap on depth admits each vertex once
    out.cap = n;
    out.err = a.err;
    bool sparse = true;  // level d's frontier is a list (else a bitmap)
    int d = 0, pulls = 0;
    for (;; ++d) {
        int32_t size = sparse ? ld_relaxed_i32(a.cnt + d % 3) : ld_relaxed_i32(a.bcnt + d % 3);
        if (size == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.cnt[(d + 2) % 3] = 0;
            a.bcnt[(d + 2) % 3] = 0;
            if (a.spcnt) a.spcnt[(d + 1) & 1] = 0;
        }
        if (size < a.push_below) {
            if (!sparse) {
                // bitmap -> list d & 1 (cnt[d % 3] is zero: cleared two levels ago)
                const uint32_t *bm = a.bm[d & 1];
                for (int64_t base = gwarp * 32; base < words; base += nwarps * 32) {
                    const int64_t w = base + lane;
                    const uint32_t bits = w < words ? bm[w] : 0u;
                    const int c = __popc(bits);
                    int incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(G2_FULL, incl, o);
                        if (lane >= o) incl += t;
                    }
                    const int tot = __shfl_sync(G2_FULL, incl, 31);
                    int32_t pos = 0;
                    if (lane == 31 && tot) pos = atomicAdd(a.cnt + d % 3, tot);
                    pos = __shfl_sync(G2_FULL, pos, 31) + incl - c;
                    uint32_t b = bits;
                    while (b) {
                        const int j = __ffs(b) - 1;
                        b &= b - 1;
                        if (pos < n) a.q[d & 1][pos] = (int32_t)(w * 32 + j);
                        ++pos;
                    }
                }
                if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
                size = ld_relaxed_i32(a.cnt + d % 3);
                sparse = true;
            }
            FrontierIn fin{a.q[d & 1], size, nullptr};
            out.q = a.q[(d + 1) & 1];
            out.cnt = a.cnt + (d + 1) % 3;
            if (LB == G2_LB_ETWC && a.spcnt) {
                // Algorithm 3 with the CTA-stage entries of kEtwcSpill arcs or
                // more handed to a grid-wide pass after the barrier (a hub
                // would otherwise keep one CTA busy while the rest wait)
                int32_t *spc = a.spcnt + (d & 1);
                lb_etwc(a.g, fin, size, op, out, blockIdx.x, gridDim.x, a.ctr,
                        EtwcSpill<int32_t>{a.spq, spc});
                if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
                if (ld_relaxed_i32(spc) > 0) {
                    lb_etwc_spill(a.g, a.spq, spc, op, out, blockIdx.x, gridDim.x);
                    if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
                }
            } else if (LB == G2_LB_STRICT) {
                // the same number of arcs for every thread of the grid
                if (!fused_strict_scan(a.g, a.q[d & 1], size, a.scan, a.ctasum, a.bar, a.err,
                                       a.limit_ns))
                    return;
                lb_strict(a.g, fin, size, a.scan, op, out, blockIdx.x, gridDim.x, a.ctr);
                if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
            } else {
                run_lb<LB>(a.g, fin, size, op, out, a.ctr);
                if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
            }
        } else {
            uint32_t *cur = a.bm[d & 1];
            if (sparse) {
                // list d & 1 -> bitmap: clear it, then set the list's bits
                for (int64_t w = gt; w < words; w += nt) cur[w] = 0u;
                if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
                const int32_t *q = a.q[d & 1];
                for (int64_t i = gt; i < size; i += nt) {
                    const int32_t v = q[i];
                    atomicOr(&cur[v >> 5], 1u << (v & 31));
                }
                if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
            }
            // bottom-up over every vertex; the next level as a bitmap
            Member mem{MEM_BITMAP, cur, nullptr};
            uint32_t *next = a.bm[(d + 1) & 1];
            int32_t found = 0;
            for (int64_t base = gwarp * 32; base < n; base += nwarps * 32) {
                const int64_t v = base + lane;
                int code = 0, scanned = 0;
                if (v < n) {
                    const int32_t c = pop.ctx((int32_t)v);
                    if (pop.filter(c)) {
                        int32_t acc = pop.identity();
                        const int32_t e1 = a.g.crowptr[v + 1];
                        for (int32_t e = a.g.crowptr[v]; e < e1; ++e) {
                            const int32_t u = a.g.ccol[e];
                            ++scanned;
                            if (mem.has(u)) {
                                acc = u;  // ascending in-list: the first hit is the smallest
                                break;
                            }
                        }
                        code = pop.finish((int32_t)v, c, acc);
                    }
                }
                count_arcs(a.ctr, scanned);
                const unsigned mask = __ballot_sync(G2_FULL, code & 1);
                if (lane == 0) {
                    next[base >> 5] = mask;
                    found += __popc(mask);
                }
            }
            if (lane == 0 && found) atomicAdd(a.bcnt + (d + 1) % 3, found);
            if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
            sparse = false;
            ++pulls;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.result[0] = d;
        a.result[1] = pulls;
    }
}

struct FusedSsspArgs {
    DevGraph g;
    int32_t *dist;
    int32_t delta;
    int32_t *nq[2];
    int32_t *fq[2];
    int32_t *ncnt;     // [3] rotating near-list lengths (list 0: ncnt[0] at launch)
    int32_t *fcnt;     // [2] far-pile lengths (pile 0: fcnt[0] at launch, fcnt[1] = 0)
    int32_t *dmin;     // [2] far minimum per epoch parity (G2_INF32 at launch)
    int32_t *stamp;    // near dedup stamps
    int32_t round0;    // first near stamp
    int32_t *stamp2;   // far dedup stamps
    int32_t epoch0;    // far stamp of pile 0 at launch
    int32_t T0;        // threshold of the bucket at launch (clamped to G2_INF32)
    int32_t lo_far;    // after a near round, stop at a bucket boundary whose
                       // pile holds at most this many entries (0: never)
    int32_t *result;   // [0] near rounds, [1] buckets, [2] 1 if stopped for the
                       // cluster loop, [3] threshold, [4] live pile, [5] epochs
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
    int64_t T = a.T0;
    int d = 0, fp = 0, epoch = 0, buckets = 0, handover = 0;
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
        if (nfar <= a.lo_far && d > 0) {  // no CTA appends now: the same length everywhere
            handover = 1;
            break;
        }
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
        a.result[2] = handover;
        a.result[3] = (int32_t)(T < G2_INF32 ? T : G2_INF32);
        a.result[4] = fp;
        a.result[5] = epoch;
    }
}

__global__ void k_fill_dist(int32_t *a, int32_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        a[v] = G2_INF32;
}

// ---------------------------------------------------- BFS in one cluster
// Fused BFS rounds while the frontier is small (bounded degree, high
// diameter): the loop runs inside one thread-block cluster of CL CTAs, so a
// level boundary is the cluster's hardware barrier instead of a grid barrier
// over global counters.  Each CTA appends the vertices it discovers to a
// queue in its own shared memory; after the barrier every CTA reads the CL
// queue lengths through distributed shared memory and takes an equal slice of
// their concatenation, reading the vertices from the owners' shared memory.
// Within a CTA a warp takes 32 frontier vertices and spreads their arcs over
// its lanes (a warp-wide scan of the degrees and a shuffle search for each
// arc's source), four arcs per lane in flight, so a level costs one chain of
// dependent accesses: queue entry, row offsets, column ids, compare-and-swap.
// Every CTA reads the same lengths and takes the same decisions, so all
// threads pass the same sequence of cluster barriers.
//
// The loop and the grid-wide loop (k_bfs_fused) hand the search to each other
// at a level boundary: the cluster stops when a level holds more than `hi`
// vertices (its frontier is copied to the global list of that level), the
// grid loop stops when a level holds fewer than `lo`.  Each launch runs at
// least one level.  A level that outgrows a CTA's queue (appends past the
// capacity are counted, not stored) also stops the cluster; its vertices are
// all labelled, so the host rebuilds that frontier from the depths.
constexpr int kClQcap = 28672;    // queue entries per CTA and buffer (2 buffers: 224 KiB)
constexpr int kClArcs = 4;        // arcs per lane in flight

struct ClusterBfsArgs {
    DevGraph g;
    int32_t *depth;
    int32_t *parent;  // may be null
    int32_t *q[2];    // global lists: level d's frontier is q[d & 1] ...
    int32_t *cnt;     // ... with length cnt[d % 3]
    int32_t d0;       // first level (its frontier is in the global list)
    int32_t hi;       // stop before a level with more vertices
    int32_t *result;  // out: [0] level reached, [1] CL_DONE / CL_TO_GRID / CL_OVERFLOW
    unsigned long long *ctr;  // arcs examined, or null
};

template <int CL>
__global__ void __launch_bounds__(kClCta, 1) k_bfs_cluster(ClusterBfsArgs a) {
    extern __shared__ int32_t s_q[];    // [2][kClQcap]
    __shared__ int32_t s_cnt[2];        // entries appended to queue buffer 0 / 1
    __shared__ int32_t s_off[CL + 1];   // prefix of the cluster's queue lengths
    __shared__ int32_t s_over;
    const uint32_t rank = cl_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t *__restrict__ rowptr = a.g.rowptr;
    const int32_t *__restrict__ col = a.g.col;
    if (threadIdx.x == 0) {
        s_cnt[0] = 0;
        s_cnt[1] = 0;
    }
    const int32_t *qg = (a.d0 & 1) ? a.q[1] : a.q[0];
    int32_t total = ld_relaxed_i32(a.cnt + a.d0 % 3);
    int reason = CL_DONE;
    unsigned long long arcs = 0;
    cl_barrier();
    int d = a.d0;
    for (;; ++d) {
        const int cb = d & 1, nb = cb ^ 1;
        const bool first = d == a.d0;
        if (!first) {
            if (warp == 0) {
                int32_t c = lane < CL ? cl_read(&s_cnt[cb], lane) : 0;
                const bool over = __any_sync(G2_FULL, c > kClQcap);
#pragma unroll
                for (int o = 1; o < CL; o <<= 1) {
                    const int32_t t = __shfl_up_sync(G2_FULL, c, o);
                    if (lane >= o) c += t;
                }
                if (lane < CL) s_off[lane + 1] = c;
                if (lane == 0) {
                    s_off[0] = 0;
                    s_over = over;
                    s_cnt[nb] = 0;
                }
            }
            __syncthreads();
            total = s_off[CL];
            if (total == 0) break;
            if (s_over) {
                reason = CL_OVERFLOW;
                break;
            }
            if (total > a.hi) {
                // hand the level to the grid loop: this CTA's part of the list
                int32_t *dst = (cb ? a.q[1] : a.q[0]) + s_off[rank];
                const int32_t mine = s_off[rank + 1] - s_off[rank];
                for (int32_t j = threadIdx.x; j < mine; j += kClCta) dst[j] = s_q[cb * kClQcap + j];
                reason = CL_TO_GRID;
                break;
            }
        }
        const int32_t *cur = s_q + cb * kClQcap;
        int32_t *nxt = s_q + nb * kClQcap;
        const int32_t lo = (int32_t)((int64_t)total * rank / CL);
        const int32_t hi = (int32_t)((int64_t)total * (rank + 1) / CL);
        for (int32_t base = lo + warp * 32; base < hi; base += kClCta) {
            const int32_t i = base + lane;
            int32_t u = 0, beg = 0, deg = 0;
            if (i < hi) {
                if (first) {
                    u = qg[i];
                } else {
                    const int r = cl_owner<CL>(s_off, i);
                    u = cl_read(cur + (i - s_off[r]), (uint32_t)r);
                }
                beg = __ldg(rowptr + u);
                deg = __ldg(rowptr + u + 1) - beg;
            }
            int32_t incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t t = __shfl_up_sync(G2_FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const int32_t tot = __shfl_sync(G2_FULL, incl, 31);
            const int32_t excl = incl - deg;
            arcs += (unsigned)tot;
            for (int32_t k0 = 0; k0 < tot; k0 += 32 * kClArcs) {
                int32_t v[kClArcs], ou[kClArcs], dv[kClArcs];
#pragma unroll
                for (int j = 0; j < kClArcs; ++j) {
                    const int32_t k = k0 + 32 * j + lane;
                    // arc k belongs to the last lane whose first arc is <= k
                    int own = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int32_t ex = __shfl_sync(G2_FULL, excl, own + step);
                        if (ex <= k) own += step;
                    }
                    ou[j] = __shfl_sync(G2_FULL, u, own);
                    const int32_t ob = __shfl_sync(G2_FULL, beg, own);
                    const int32_t oe = __shfl_sync(G2_FULL, excl, own);
                    v[j] = k < tot ? __ldg(col + ob + (k - oe)) : -1;
                }
#pragma unroll
                for (int j = 0; j < kClArcs; ++j)
                    dv[j] = v[j] >= 0 ? atomicCAS(a.depth + v[j], -1, d + 1) : 0;
#pragma unroll
                for (int j = 0; j < kClArcs; ++j) {
                    const bool disc = v[j] >= 0 && dv[j] == -1;
                    // the smallest source among this level's arcs into v
                    if (a.parent && v[j] >= 0 && (disc || dv[j] == d + 1))
                        atomicMin(reinterpret_cast<unsigned *>(a.parent + v[j]), (unsigned)ou[j]);
                    cta_append(nxt, &s_cnt[nb], kClQcap, v[j], disc, lane);
                }
            }
        }
        cl_barrier();  // level d complete: queues nb filled, queues cb no longer read
    }
    cl_barrier();  // no CTA leaves while a peer may still read its queue lengths
    if (a.ctr && lane == 0 && arcs) atomicAdd(a.ctr, arcs);
    if (threadIdx.x == 0 && rank == 0) {
        a.result[0] = d;
        a.result[1] = reason;
        if (reason == CL_TO_GRID) {
            a.cnt[d % 3] = total;
            a.cnt[(d + 1) % 3] = 0;
        } else if (reason == CL_OVERFLOW) {
            a.cnt[d % 3] = 0;  // rebuilt from the depths
            a.cnt[(d + 1) % 3] = 0;
        }
    }
}

// ------------------------------------------------- delta-stepping in one cluster
// The near/far loop of k_sssp_fused inside one thread-block cluster while the
// near lists are small.  Each CTA keeps, in its own shared memory, the near
// list entries it appended (two buffers, as the BFS above) and its part of
// the far pile (two piles, old and new epoch).  A near round relaxes an equal
// slice of the cluster's near list (read through distributed shared memory),
// four arcs per lane in flight; an improvement below the bucket threshold
// joins the CTA's next near list, one at or above it joins the CTA's far pile
// (deduplicated per round / epoch by the same stamps as the grid loop; on a
// bounded-degree graph the near lists skip the stamp, whose atomic would sit
// on every round's chain: a vertex improved twice in a round is then relaxed
// twice in the next, with its current distance both times).  When
// the near list empties, every CTA takes the smallest live distance of its
// own pile, the cluster minimum (read through distributed shared memory)
// fixes the next bucket, and each CTA splits its own pile into its near list
// and its new pile.
//
// Hand-over: the cluster stops before a near round of more than `hi`
// vertices and writes its near list and far pile to the global lists the grid
// loop starts from; the grid loop stops at a bucket boundary whose far pile
// holds at most `lo_far` entries and the cluster starts from that pile.  A
// near list or pile that outgrows its shared buffer (appends past the
// capacity are counted, not stored) stops the cluster too; the bucket's state
// is then rebuilt from the distances (k_sssp_rebuild) and the grid loop goes
// on.  Decisions use only counts that no CTA changes while they are read, so
// every CTA takes the same ones and passes the same cluster barriers.
constexpr int kCsQn = 12288;  // near entries per CTA and buffer
constexpr int kCsQf = 14336;  // far entries per CTA and pile
constexpr size_t kCsSmem = (2 * (size_t)kCsQn + 2 * (size_t)kCsQf) * 4;  // 208 KiB

struct ClusterSsspArgs {
    DevGraph g;
    int32_t *dist;
    int32_t delta;
    const int32_t *nq_in;    // first near list (global) ...
    const int32_t *ncnt_in;  // ... and its length (null: empty)
    const int32_t *fq_in;    // far pile at launch (global) ...
    const int32_t *fcnt_in;  // ... and its length; at most kCsQf * CL / 2 entries
    int32_t T0;              // threshold of the current bucket (clamped to G2_INF32)
    int32_t *stamp;          // near dedup: round r's appends carry round0 + r
    int32_t round0;
    int32_t *stamp2;         // far dedup: the pile of epoch e carries epoch0 + e
    int32_t epoch0;
    int32_t hi;              // stop before a near round with more vertices
    int32_t dedup_near;      // 0: near lists keep repeats (bounded-degree graphs)
    int32_t *nq_out;         // hand-over: near list ...
    int32_t *fq_out;         // ... and far pile for the grid loop
    int32_t *ncnt;           // the grid loop's near lengths [3], far lengths [2],
    int32_t *fcnt;           // far minima [2], set on hand-over
    int32_t *dmin;
    int32_t *result;         // out: [0] near rounds, [1] epochs advanced, [2] CL_*, [3] T
    int32_t *err;
    unsigned long long *ctr;
};

template <int CL>
__global__ void __launch_bounds__(kClCta, 1) k_sssp_cluster(ClusterSsspArgs a) {
    extern __shared__ int32_t s_mem[];
    int32_t *s_nq = s_mem;              // [2][kCsQn]
    int32_t *s_fq = s_mem + 2 * kCsQn;  // [2][kCsQf]
    __shared__ int32_t s_ncnt[2], s_fcnt[2];
    __shared__ int32_t s_off[CL + 1], s_foff[CL + 1];
    __shared__ int32_t s_nover, s_fover, s_min;
    const uint32_t rank = cl_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t *__restrict__ rowptr = a.g.rowptr;
    const int32_t *__restrict__ col = a.g.col;
    const int32_t *__restrict__ wt = a.g.w;
    // this CTA's slice of the far pile
    {
        const int32_t ftot = ld_relaxed_i32(a.fcnt_in);
        const int32_t flo = (int32_t)((int64_t)ftot * rank / CL);
        const int32_t fhi = (int32_t)((int64_t)ftot * (rank + 1) / CL);
        for (int32_t j = threadIdx.x; j < fhi - flo; j += kClCta) s_fq[j] = a.fq_in[flo + j];
        if (threadIdx.x == 0) {
            s_fcnt[0] = fhi - flo;
            s_fcnt[1] = 0;
            s_ncnt[0] = 0;
            s_ncnt[1] = 0;
        }
    }
    int32_t total = a.ncnt_in ? ld_relaxed_i32(a.ncnt_in) : 0;
    int32_t T = a.T0;
    int fp = 0, e = 0, r = 0, reason = CL_DONE;
    unsigned long long arcs = 0;
    cl_barrier();
    int d = 0;  // near buffer parity: level d reads buffer d & 1
    bool first = true;
    for (;;) {
        const int cb = d & 1, nb = cb ^ 1;
        if (!first) {
            if (warp == 0) {
                int32_t c = lane < CL ? cl_read(&s_ncnt[cb], lane) : 0;
                int32_t f = lane < CL ? cl_read(&s_fcnt[fp], lane) : 0;
                const bool nover = __any_sync(G2_FULL, c > kCsQn);
                const bool fover = __any_sync(G2_FULL, f > kCsQf);
#pragma unroll
                for (int o = 1; o < CL; o <<= 1) {
                    const int32_t t1 = __shfl_up_sync(G2_FULL, c, o);
                    const int32_t t2 = __shfl_up_sync(G2_FULL, f, o);
                    if (lane >= o) {
                        c += t1;
                        f += t2;
                    }
                }
                if (lane < CL) {
                    s_off[lane + 1] = c;
                    s_foff[lane + 1] = f;
                }
                if (lane == 0) {
                    s_off[0] = 0;
                    s_foff[0] = 0;
                    s_nover = nover;
                    s_fover = fover;  // meaningful only when no CTA appends this level
                    s_ncnt[nb] = 0;
                }
            }
            __syncthreads();
            total = s_off[CL];
            if (s_nover || ((total == 0 || total > a.hi) && s_fover)) {
                reason = CL_OVERFLOW;
                break;
            }
            if (total > a.hi) {
                // hand the bucket to the grid loop: this CTA's near list and pile
                const int32_t nmine = s_off[rank + 1] - s_off[rank];
                const int32_t fmine = s_foff[rank + 1] - s_foff[rank];
                for (int32_t j = threadIdx.x; j < nmine; j += kClCta)
                    a.nq_out[s_off[rank] + j] = s_nq[cb * kCsQn + j];
                for (int32_t j = threadIdx.x; j < fmine; j += kClCta)
                    a.fq_out[s_foff[rank] + j] = s_fq[fp * kCsQf + j];
                reason = CL_TO_GRID;
                break;
            }
        }
        if (total > 0) {
            // near round r: relax the arcs of this CTA's slice of the near list
            const int32_t rid = a.round0 + r, eid = a.epoch0 + e;
            const int32_t *cur = s_nq + cb * kCsQn;
            int32_t *nxt = s_nq + nb * kCsQn;
            int32_t *far = s_fq + fp * kCsQf;
            const int32_t lo = (int32_t)((int64_t)total * rank / CL);
            const int32_t hi = (int32_t)((int64_t)total * (rank + 1) / CL);
            for (int32_t base = lo + warp * 32; base < hi; base += kClCta) {
                const int32_t i = base + lane;
                int32_t u = 0, beg = 0, deg = 0, du = 0;
                if (i < hi) {
                    if (first) {
                        u = a.nq_in[i];
                    } else {
                        const int q = cl_owner<CL>(s_off, i);
                        u = cl_read(cur + (i - s_off[q]), (uint32_t)q);
                    }
                    beg = __ldg(rowptr + u);
                    deg = __ldg(rowptr + u + 1) - beg;
                    du = a.dist[u];
                }
                int32_t incl = deg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t t = __shfl_up_sync(G2_FULL, incl, o);
                    if (lane >= o) incl += t;
                }
                const int32_t tot = __shfl_sync(G2_FULL, incl, 31);
                const int32_t excl = incl - deg;
                arcs += (unsigned)tot;
                for (int32_t k0 = 0; k0 < tot; k0 += 32 * kClArcs) {
                    int32_t v[kClArcs], nv[kClArcs], old[kClArcs];
#pragma unroll
                    for (int j = 0; j < kClArcs; ++j) {
                        const int32_t k = k0 + 32 * j + lane;
                        int own = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const int32_t ex = __shfl_sync(G2_FULL, excl, own + step);
                            if (ex <= k) own += step;
                        }
                        const int32_t ob = __shfl_sync(G2_FULL, beg, own);
                        const int32_t oe = __shfl_sync(G2_FULL, excl, own);
                        const int32_t od = __shfl_sync(G2_FULL, du, own);
                        v[j] = -1;
                        nv[j] = 0;
                        if (k < tot) {
                            const int32_t arc = ob + (k - oe);
                            const int64_t nd = (int64_t)od + __ldg(wt + arc);
                            if (nd >= G2_INF32) {
                                set_error(a.err, G2_EOVERFLOW);
                            } else {
                                v[j] = __ldg(col + arc);
                                nv[j] = (int32_t)nd;
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kClArcs; ++j)
                        old[j] = v[j] >= 0 ? atomicMin(a.dist + v[j], nv[j]) : 0;
#pragma unroll
                    for (int j = 0; j < kClArcs; ++j) {
                        const bool better = v[j] >= 0 && nv[j] < old[j];
                        bool to_near = better && nv[j] < T;
                        bool to_far = better && nv[j] >= T;
                        if (to_near && a.dedup_near) to_near = atomicExch(a.stamp + v[j], rid) != rid;
                        if (to_far) to_far = atomicExch(a.stamp2 + v[j], eid) != eid;
                        cta_append(nxt, &s_ncnt[nb], kCsQn, v[j], to_near, lane);
                        cta_append(far, &s_fcnt[fp], kCsQf, v[j], to_far, lane);
                    }
                }
            }
            first = false;
            cl_barrier();  // round complete: lists nb and piles filled
            ++d;
            ++r;
            continue;
        }
        if (first) {  // launched at a bucket boundary: read the counts first
            first = false;
            continue;
        }
        // bucket boundary: the smallest live far distance over the cluster
        if (s_foff[CL] == 0) break;  // nothing left: done
        const int32_t Told = T;
        {
            if (threadIdx.x == 0) s_min = G2_INF32;
            __syncthreads();
            int32_t best = G2_INF32;
            const int32_t mine = s_fcnt[fp];
            for (int32_t j = threadIdx.x; j < mine; j += kClCta) {
                const int32_t dv = a.dist[s_fq[fp * kCsQf + j]];
                if (dv >= Told && dv < best) best = dv;
            }
            best = (int32_t)__reduce_min_sync(G2_FULL, (unsigned)best);
            if (lane == 0 && best != G2_INF32) atomicMin(&s_min, best);
        }
        cl_barrier();
        int32_t dm = lane < CL ? cl_read(&s_min, lane) : G2_INF32;
        dm = (int32_t)__reduce_min_sync(G2_FULL, (unsigned)dm);
        if (dm == G2_INF32) break;  // only stale entries left: done
        const int64_t Tnew = ((int64_t)dm / a.delta + 1) * (int64_t)a.delta;
        const int32_t Tn = (int32_t)(Tnew < G2_INF32 ? Tnew : G2_INF32);
        const int32_t neid = a.epoch0 + e + 1;
        if (threadIdx.x == 0) s_fcnt[fp ^ 1] = 0;
        __syncthreads();
        // split this CTA's pile: the next bucket to near list cb, the rest to
        // the new pile (stale entries, already settled, are dropped)
        {
            const int32_t mine = s_fcnt[fp];
            const int32_t *pile = s_fq + fp * kCsQf;
            int32_t *npile = s_fq + (fp ^ 1) * kCsQf;
            int32_t *nl = s_nq + cb * kCsQn;
            for (int32_t base = warp * 32; base < mine; base += kClCta) {
                const int32_t j = base + lane;
                int32_t v = 0, dv = G2_INF32;
                if (j < mine) {
                    v = pile[j];
                    dv = a.dist[v];
                }
                const bool to_near = j < mine && dv >= Told && dv < Tn;
                const bool to_far = j < mine && dv >= Tn;
                if (to_far) a.stamp2[v] = neid;
                cta_append(nl, &s_ncnt[cb], kCsQn, v, to_near, lane);
                cta_append(npile, &s_fcnt[fp ^ 1], kCsQf, v, to_far, lane);
            }
        }
        cl_barrier();  // split complete everywhere; the near counts of cb are final
        fp ^= 1;
        ++e;
        T = Tn;
    }
    cl_barrier();  // no CTA leaves while a peer may still read its counts
    if (a.ctr && lane == 0 && arcs) atomicAdd(a.ctr, arcs);
    if (threadIdx.x == 0 && rank == 0) {
        a.result[0] = r;
        a.result[1] = e;
        a.result[2] = reason;
        a.result[3] = T;
        if (reason == CL_TO_GRID) {
            a.ncnt[0] = total;
            a.ncnt[1] = 0;
            a.ncnt[2] = 0;
            a.fcnt[0] = s_foff[CL];
            a.fcnt[1] = 0;
            a.dmin[0] = G2_INF32;
            a.dmin[1] = G2_INF32;
        }
    }
}

// The state of the bucket below T rebuilt from the distances: every vertex in
// [T - delta, T) to near list 0 (settled ones among them relax nothing new),
// every finite distance >= T to far pile 0 with the epoch stamp `eid`.
__global__ void k_sssp_rebuild(const int32_t *dist, int32_t n, int32_t T, int32_t delta,
                               int32_t *nq, int32_t *ncnt, int32_t *fq, int32_t *fcnt,
                               int32_t *stamp2, int32_t eid, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int64_t Tb = (int64_t)T - delta;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + lane;
        const int32_t dv = v < n ? dist[v] : G2_INF32;
        const bool to_near = v < n && dv >= Tb && dv < T;
        const bool to_far = v < n && dv >= T && dv != G2_INF32;
        if (to_far) stamp2[v] = eid;
        warp_append(nq, ncnt, n, err, (int32_t)v, to_near);
        warp_append(fq, fcnt, n, err, (int32_t)v, to_far);
    }
}

static g2_status check_fused_lb(const g2_schedule &s) {
    if (s.direction != G2_PUSH)
        return fail(G2_EUNSUPPORTED, "fused loops run PUSH rounds");
    if (s.edge_blocking)
        return fail(G2_EUNSUPPORTED, "EdgeBlocking applies to EDGE_ONLY full sweeps only");
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
    a.d0 = 0;
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
    G2_TRY(put_i32(st, {{depth + src, zero}, {parent ? parent + src : nullptr, src}, {a.q[0], src},
                        {a.cnt, one}}));
    // WM rounds start in one cluster and move between it and the grid-wide
    // loop as the levels grow and shrink; the other strategies (and a device
    // without room for the cluster) run the grid-wide loop throughout.
    const int cl = s.load_balance == G2_LB_WM
                       ? cluster_size(0, k_bfs_cluster<16>, k_bfs_cluster<8>, 2 * (size_t)kClQcap * 4)
                       : 0;
    // measured on road grids 1024^2..4096^2 with 16-CTA clusters: hand a
    // level to the grid above 16384 vertices, take it back below 8192
    a.lo = cl ? env_i32("G2_CLUSTER_LO", 512 * cl) : 0;
    ClusterBfsArgs c;
    c.g = a.g;
    c.depth = depth;
    c.parent = parent;
    c.q[0] = a.q[0];
    c.q[1] = a.q[1];
    c.cnt = a.cnt;
    c.hi = env_i32("G2_CLUSTER_HI", 1024 * cl);
    c.result = ctrs + 32;
    c.ctr = a.ctr;
    int32_t level = 0;
    bool in_cluster = cl != 0;
    for (;;) {
        if (in_cluster) {
            c.d0 = level;
            if (cl == 16) G2_TRY(launch_cluster(k_bfs_cluster<16>, 16, 2 * (size_t)kClQcap * 4, c, st));
            else G2_TRY(launch_cluster(k_bfs_cluster<8>, 8, 2 * (size_t)kClQcap * 4, c, st));
            G2_TRY(read_counters(g, ctrs + 32, 2, st, d_err));
            const int32_t reached = g->h_ctr[0], why = g->h_ctr[1];
            if (reached <= level) return fail(G2_ECUDA, "cluster BFS made no progress");
            level = reached;
            if (why == CL_DONE) break;
            if (why == CL_OVERFLOW) {
                k_level_list<<<grid_for(g, n, kCta), kCta, 0, st>>>(depth, n, level, a.q[level & 1],
                                                                    a.cnt + level % 3, d_err);
                stats().launches += 1;
                G2_CK(cudaGetLastError());
            }
        } else {
            a.d0 = level;
            switch (s.load_balance) {
                case G2_LB_WM: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_WM>, a, st)); break;
                case G2_LB_CM: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_CM>, a, st)); break;
                case G2_LB_ETWC: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_ETWC>, a, st)); break;
                default: G2_TRY(launch_coop(g, k_bfs_fused<G2_LB_VERTEX_BASED>, a, st)); break;
            }
            G2_TRY(read_counters(g, ctrs + 24, 2, st, d_err));
            const int32_t reached = g->h_ctr[0], why = g->h_ctr[1];
            if (reached <= level) return fail(G2_ECUDA, "fused BFS made no progress");
            level = reached;
            if (!why) break;
        }
        in_cluster = !in_cluster;
    }
    stats().iterations = level;
    stats().push_rounds = level;
    stats().barriers = level;
    return G2_OK;
}

// The direction-optimising hybrid in one launch (k_bfs_fused_do): h.s1 is the
// PUSH schedule (a load balancing of the fused loops), h.s2 VERTEX_BASED
// PULL over a bitmap; PUSH while the frontier holds fewer than threshold * n
// vertices.
g2_status bfs_fused_do(g2_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                       const g2_hybrid &h, cudaStream_t st, int32_t *d_err) {
    // the PUSH half: a load balancing of the fused loops, or STRICT (its
    // prefix sum taken inside the launch)
    if (h.s1.load_balance == G2_LB_STRICT) {
        g2_schedule s1 = h.s1;
        s1.load_balance = G2_LB_WM;
        G2_TRY(check_fused_lb(s1));
    } else {
        G2_TRY(check_fused_lb(h.s1));
    }
    if (h.criteria != G2_INPUT_VERTEXSET_SIZE)
        return fail(G2_EUNSUPPORTED, "a fused hybrid switches on the input vertexset size");
    if (h.s2.direction != G2_PULL || h.s2.load_balance != G2_LB_VERTEX_BASED ||
        h.s2.pull_frontier != G2_BITMAP)
        return fail(G2_EUNSUPPORTED, "the fused hybrid's PULL schedule is VERTEX_BASED over a bitmap");
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    FusedDoBfsArgs a;
    a.g = t->view();
    a.depth = depth;
    a.parent = parent;
    G2_TRY(ws(g, B_Q0, (size_t)std::max(n, 1), &a.q[0]));
    G2_TRY(ws(g, B_Q1, (size_t)std::max(n, 1), &a.q[1]));
    const size_t words = ((size_t)n + 31) / 32 + 1;
    G2_TRY(ws(g, B_BM0, words, &a.bm[0]));
    G2_TRY(ws(g, B_BM1, words, &a.bm[1]));
    a.cnt = ctrs + 20;
    a.bcnt = ctrs + 46;  // [46..48]
    a.spq = nullptr;
    a.spcnt = nullptr;
    a.scan = nullptr;
    a.ctasum = nullptr;
    if (h.s1.load_balance == G2_LB_STRICT) {
        // one slice total per CTA: at most 2,048 threads, so 8 CTAs, per SM
        G2_TRY(ws(g, B_SCAN, (size_t)n + 1, &a.scan));
        G2_TRY(ws(g, B_SCANTMP, (size_t)t->sm_count * (2048 / kCta) + 1, &a.ctasum));
    }
    if (h.s1.load_balance == G2_LB_ETWC) {
        // every handed-off entry has at least kEtwcSpill arcs
        const size_t cap = (size_t)t->m / kEtwcSpill + 1;
        G2_TRY(ws(g, B_TWC_L, cap, &a.spq));
        a.spcnt = ctrs + 54;  // [54..55]
    }
    const double pb = (double)h.threshold * (double)n;
    a.push_below = (int32_t)std::min<double>(std::max<double>(pb, 0.0), 2147483647.0);
    a.result = ctrs + 24;
    a.bar = GridBarrier{reinterpret_cast<unsigned long long *>(ctrs + 28)};
    a.err = d_err;
    a.limit_ns = barrier_limit_ns();
    a.ctr = nullptr;
    if (count_arcs_enabled()) G2_TRY(ws(g, B_ARCS, 2, &a.ctr));
    if (parent) G2_CK(cudaMemsetAsync(parent, 0xFF, (size_t)n * 4, st));
    G2_CK(cudaMemsetAsync(depth, 0xFF, (size_t)n * 4, st));
    int32_t zero = 0, one = 1;
    G2_TRY(put_i32(st, {{depth + src, zero}, {parent ? parent + src : nullptr, src}, {a.q[0], src},
                        {a.cnt, one}, {a.cnt + 1, zero}, {a.cnt + 2, zero}}));
    G2_TRY(put_i32(st, {{a.bcnt, zero}, {a.bcnt + 1, zero}, {a.bcnt + 2, zero},
                        {a.spcnt, zero}, {a.spcnt ? a.spcnt + 1 : nullptr, zero}}));
    // the PULL levels sweep every vertex: four CTAs per SM (measured on
    // RMAT-21/22: 0.17-0.24 ms against 0.29-0.53 ms with one)
    const int want = env_i32("G2_FUSED_DO_CTAS_PER_SM", 4);
    switch (h.s1.load_balance) {
        case G2_LB_WM: G2_TRY(launch_coop(g, k_bfs_fused_do<G2_LB_WM>, a, st, want)); break;
        case G2_LB_CM: G2_TRY(launch_coop(g, k_bfs_fused_do<G2_LB_CM>, a, st, want)); break;
        case G2_LB_ETWC: G2_TRY(launch_coop(g, k_bfs_fused_do<G2_LB_ETWC>, a, st, want)); break;
        case G2_LB_STRICT: G2_TRY(launch_coop(g, k_bfs_fused_do<G2_LB_STRICT>, a, st, want)); break;
        default: G2_TRY(launch_coop(g, k_bfs_fused_do<G2_LB_VERTEX_BASED>, a, st, want)); break;
    }
    G2_TRY(read_counters(g, ctrs + 24, 2, st, d_err));
    stats().iterations = g->h_ctr[0];
    stats().pull_rounds = g->h_ctr[1];
    stats().push_rounds = g->h_ctr[0] - g->h_ctr[1];
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
    // ncnt[3] = {1, 0, 0}, fcnt[2] = 0 (counters are zero at entry), dmin[2] = inf
    G2_TRY(put_i32(st, {{ctrs + 20, 1}, {ctrs + 25, G2_INF32}, {ctrs + 26, G2_INF32}}));
    k_fill_dist<<<grid_for(g, n, kCta), kCta, 0, st>>>(dist, n);
    int32_t zero = 0;
    G2_TRY(put_i32(st, {{dist + src, zero}, {a.nq[0], src}}));
    // WM buckets start in one cluster; near rounds above `hi` vertices move to
    // the grid-wide loop, which hands back at a bucket boundary with at most
    // `lo_far` pile entries (never more than the next near list can start
    // with in the cluster, nor than the cluster's piles hold).
    const int cl = s.load_balance == G2_LB_WM
                       ? cluster_size(1, k_sssp_cluster<16>, k_sssp_cluster<8>, kCsSmem)
                       : 0;
    ClusterSsspArgs c;
    c.g = a.g;
    c.dist = dist;
    c.delta = delta;
    c.stamp = a.stamp;
    c.stamp2 = a.stamp2;
    c.hi = env_i32("G2_CLUSTER_HI", 1024 * cl);
    int32_t dmax = 0;
    if (cl) G2_TRY(max_out_degree(g, st, &dmax));
    c.dedup_near = !(t->symmetric && dmax <= kBoundedDegree);
    c.nq_out = a.nq[0];
    c.fq_out = a.fq[0];
    c.ncnt = a.ncnt;
    c.fcnt = a.fcnt;
    c.dmin = a.dmin;
    c.result = ctrs + 36;
    c.err = d_err;
    c.ctr = a.ctr;
    a.lo_far = cl ? std::min(std::min(env_i32("G2_CLUSTER_FAR_LO", 1024 * cl), c.hi),
                             (int32_t)(kCsQf / 2 * cl))
                  : 0;
    int32_t T = (int32_t)std::min<int64_t>(delta, G2_INF32);
    int32_t round0 = g->round + 1, epoch0 = g->round2 + 1;
    int32_t rounds = 0, buckets = 0;
    const int32_t *near_in = a.nq[0], *ncnt_in = a.ncnt, *far_in = a.fq[0], *fcnt_in = a.fcnt;
    bool in_cluster = cl != 0;
    for (;;) {
        if (in_cluster) {
            c.nq_in = near_in;
            c.ncnt_in = ncnt_in;
            c.fq_in = far_in;
            c.fcnt_in = fcnt_in;
            c.T0 = T;
            c.round0 = round0;
            c.epoch0 = epoch0;
            if (cl == 16) G2_TRY(launch_cluster(k_sssp_cluster<16>, 16, kCsSmem, c, st));
            else G2_TRY(launch_cluster(k_sssp_cluster<8>, 8, kCsSmem, c, st));
            G2_TRY(read_counters(g, ctrs + 36, 4, st, d_err));
            const int32_t r = g->h_ctr[0], e = g->h_ctr[1], why = g->h_ctr[2];
            rounds += r;
            buckets += e;
            round0 += r + 1;
            epoch0 += e;
            T = g->h_ctr[3];
            if (why == CL_DONE) break;
            if (r + e == 0) return fail(G2_ECUDA, "cluster SSSP made no progress");
            if (why == CL_OVERFLOW) {
                // near list and pile of the bucket below T from the distances
                G2_TRY(put_i32(st, {{ctrs + 20, 0}, {ctrs + 21, 0}, {ctrs + 22, 0}, {ctrs + 23, 0},
                                    {ctrs + 24, 0}, {ctrs + 25, G2_INF32}, {ctrs + 26, G2_INF32}}));
                ++epoch0;
                k_sssp_rebuild<<<grid_for(g, n, kCta), kCta, 0, st>>>(
                    dist, n, T, delta, a.nq[0], a.ncnt, a.fq[0], a.fcnt, a.stamp2, epoch0, d_err);
                stats().launches += 1;
                G2_CK(cudaGetLastError());
            }
        } else {
            a.T0 = T;
            a.round0 = round0;
            a.epoch0 = epoch0;
            switch (s.load_balance) {
                case G2_LB_WM: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_WM>, a, st)); break;
                case G2_LB_CM: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_CM>, a, st)); break;
                case G2_LB_ETWC: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_ETWC>, a, st)); break;
                default: G2_TRY(launch_coop(g, k_sssp_fused<G2_LB_VERTEX_BASED>, a, st)); break;
            }
            G2_TRY(read_counters(g, ctrs + 30, 6, st, d_err));
            const int32_t r = g->h_ctr[0], why = g->h_ctr[2], fp = g->h_ctr[4];
            rounds += r;
            buckets += g->h_ctr[1];
            round0 += r + 1;
            epoch0 += g->h_ctr[5];
            T = g->h_ctr[3];
            if (!why) break;
            if (r == 0) return fail(G2_ECUDA, "fused SSSP made no progress");
            near_in = nullptr;  // handed back at a bucket boundary: no near list
            ncnt_in = nullptr;
            far_in = a.fq[fp];
            fcnt_in = a.fcnt + fp;
        }
        in_cluster = !in_cluster;
    }
    stats().iterations = rounds;
    stats().push_rounds = rounds;
    stats().barriers = rounds + 2 * buckets;
    g->round = round0;
    g->round2 = epoch0 + 1;
    return G2_OK;
}

}  // namespace g2
