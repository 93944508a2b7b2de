// g2_lb.cuh — the load-balancing library (Sec. III and VI-C): how the arcs of
// the input vertexset are divided among threads in the PUSH direction, and
// how destinations are divided in the PULL direction.
//
// Every routine takes a virtual CTA index `bid` and CTA count `nb` so it can
// run from a per-round __global__ wrapper (bid = blockIdx.x) or inside the
// fused persistent kernel (Sec. VI-C, kernel fusion), where a few resident
// CTAs do the work of many.  All inner loops are warp-uniform so that the
// warp-aggregated enqueue (emit) sees all 32 lanes.
#pragma once
#include "g2_device.cuh"

namespace g2 {

template <class T>
__device__ __forceinline__ T shfl_xor_acc(T x, int d) {
    return __shfl_xor_sync(G2_FULL, x, d);
}

// --------------------------------------------------------------- VERTEX_BASED
// One thread per active vertex, serial walk of its arcs.
template <class Op>
__device__ void lb_vertex(const DevGraph &g, const FrontierIn &fin, int32_t fsize, const Op &op,
                          const OutCtx &out, int bid, int nb, unsigned long long *ctr) {
    const int lane = threadIdx.x & 31;
    const int gw = bid * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = nb * (blockDim.x >> 5);
    for (int64_t base = (int64_t)gw * 32; base < fsize; base += (int64_t)nw * 32) {
        int32_t i = (int32_t)base + lane;
        int32_t u = 0, beg = 0, len = 0;
        typename Op::S s{};
        if (i < fsize) {
            u = fin.vertex(i);
            s = op.load(u);
            if (!op.skip(s)) {
                beg = g.rowptr[u];
                len = g.rowptr[u + 1] - beg;
            }
        }
        count_arcs(ctr, len);
        int maxlen = (int)__reduce_max_sync(G2_FULL, (unsigned)len);
        for (int k = 0; k < maxlen; ++k) {
            int code = 0;
            int32_t v = 0;
            if (k < len) {
                v = g.col[beg + k];
                code = op.relax(u, s, v, beg + k);
            }
            emit(out, v, code);
        }
    }
}

// ------------------------------------------------------------------------ WM
// A warp takes 32 active vertices, prefix-sums their degrees with shuffles and
// walks the combined arc range 32 arcs at a time; each lane finds the owner of
// its arc by a 5-step binary search over the lanes' prefix sums.
template <class Op>
__device__ void lb_warp(const DevGraph &g, const FrontierIn &fin, int32_t fsize, const Op &op,
                        const OutCtx &out, int bid, int nb, unsigned long long *ctr) {
    const int lane = threadIdx.x & 31;
    const int gw = bid * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = nb * (blockDim.x >> 5);
    for (int64_t base = (int64_t)gw * 32; base < fsize; base += (int64_t)nw * 32) {
        int32_t i = (int32_t)base + lane;
        int32_t u = 0, beg = 0, len = 0;
        typename Op::S s{};
        if (i < fsize) {
            u = fin.vertex(i);
            s = op.load(u);
            if (!op.skip(s)) {
                beg = g.rowptr[u];
                len = g.rowptr[u + 1] - beg;
            }
        }
        count_arcs(ctr, len);
        int incl = warp_incl_scan(len);
        int total = __shfl_sync(G2_FULL, incl, 31);
        int excl = incl - len;
        for (int k0 = 0; k0 < total; k0 += 32) {
            int k = k0 + lane;
            int lo = 0, hi = 31;
#pragma unroll
            for (int st = 0; st < 5; ++st) {
                int mid = (lo + hi) >> 1;
                int im = __shfl_sync(G2_FULL, incl, mid);
                if (im > k) hi = mid;
                else lo = mid + 1;
            }
            int owner = lo;
            int32_t ou = __shfl_sync(G2_FULL, u, owner);
            typename Op::S os = shfl(s, owner);
            int32_t ob = __shfl_sync(G2_FULL, beg, owner);
            int oe = __shfl_sync(G2_FULL, excl, owner);
            int code = 0;
            int32_t v = 0;
            if (k < total) {
                int32_t e = ob + (k - oe);
                v = g.col[e];
                code = op.relax(ou, os, v, e);
            }
            emit(out, v, code);
        }
    }
}

// ------------------------------------------------------------------------ CM
// A CTA takes kCta active vertices, block-scans their degrees in shared memory
// and walks the combined arc range kCta arcs at a time.
template <class Op>
__device__ void lb_cta(const DevGraph &g, const FrontierIn &fin, int32_t fsize, const Op &op,
                       const OutCtx &out, int bid, int nb, unsigned long long *ctr) {
    __shared__ int s_incl[kCta];
    __shared__ int32_t s_u[kCta];
    __shared__ int32_t s_beg[kCta];
    __shared__ typename Op::S s_s[kCta];
    __shared__ int s_warp[kWarps];
    const int tid = threadIdx.x;
    for (int64_t base = (int64_t)bid * kCta; base < fsize; base += (int64_t)nb * kCta) {
        int32_t i = (int32_t)base + tid;
        int32_t u = 0, beg = 0, len = 0;
        typename Op::S s{};
        if (i < fsize) {
            u = fin.vertex(i);
            s = op.load(u);
            if (!op.skip(s)) {
                beg = g.rowptr[u];
                len = g.rowptr[u + 1] - beg;
            }
        }
        count_arcs(ctr, len);
        int total;
        int incl = block_incl_scan(len, s_warp, &total);
        s_incl[tid] = incl;
        s_u[tid] = u;
        s_beg[tid] = beg - (incl - len);  // arc index = s_beg[owner] + k
        s_s[tid] = s;
        __syncthreads();
        for (int k0 = 0; k0 < total; k0 += kCta) {
            int k = k0 + tid;
            int code = 0;
            int32_t v = 0;
            if (k < total) {
                int lo = 0, hi = kCta - 1;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (s_incl[mid] > k) hi = mid;
                    else lo = mid + 1;
                }
                int32_t e = s_beg[lo] + k;
                v = g.col[e];
                code = op.relax(s_u[lo], s_s[lo], v, e);
            }
            emit(out, v, code);
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------- STRICT
// Every thread gets the same number of arcs: arc k of the frontier-wide arc
// sequence belongs to the active vertex i with scan[i] <= k < scan[i+1]
// (scan = exclusive prefix sum of the active vertices' degrees, computed by a
// separate pass); found by binary search per arc.
template <class Op>
__device__ void lb_strict(const DevGraph &g, const FrontierIn &fin, int32_t fsize,
                          const int32_t *scan, const Op &op, const OutCtx &out, int bid, int nb,
                          unsigned long long *ctr) {
    const int32_t total = scan[fsize];
    constexpr int kPer = 4;  // arcs per thread per tile
    const int64_t tile = (int64_t)kCta * kPer;
    __shared__ int32_t s_lo, s_hi;
    for (int64_t t0 = (int64_t)bid * tile; t0 < total; t0 += (int64_t)nb * tile) {
        if (threadIdx.x == 0) {
            // owners of the first and last arc of the tile
            int64_t t1 = t0 + tile - 1 < total ? t0 + tile - 1 : total - 1;
            int lo = 0, hi = fsize - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (scan[mid] <= t0) lo = mid;
                else hi = mid - 1;
            }
            s_lo = lo;
            int lo2 = lo, hi2 = fsize - 1;
            while (lo2 < hi2) {
                int mid = (lo2 + hi2 + 1) >> 1;
                if (scan[mid] <= t1) lo2 = mid;
                else hi2 = mid - 1;
            }
            s_hi = lo2;
        }
        __syncthreads();
        const int32_t vlo = s_lo, vhi = s_hi;
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            int64_t k = t0 + (int64_t)j * kCta + threadIdx.x;
            int code = 0;
            int32_t v = 0;
            if (k < total) {
                int lo = vlo, hi = vhi;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (scan[mid] <= k) lo = mid;
                    else hi = mid - 1;
                }
                int32_t u = fin.vertex(lo);
                typename Op::S s = op.load(u);
                int32_t e = g.rowptr[u] + (int32_t)(k - scan[lo]);
                v = g.col[e];
                code = op.relax(u, s, v, e);
                ++cnt;
            }
            emit(out, v, code);
        }
        count_arcs(ctr, cnt);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------- ETWC
// Algorithm 3.  Inside each CTA every thread takes one active vertex and
// splits its arc range into a multiple of the CTA size, a multiple of the warp
// size and a remainder, pushed to three shared-memory queues; then the
// remainder entries are walked by single threads, the warp entries by whole
// warps and the CTA entries by the whole CTA (cyclic distribution).
template <class S>
struct EtwcEntry {
    int32_t beg, end, u;
    S s;
};

// Frontier-wide hand-off of ETWC's largest CTA-stage entries: a vertex whose
// CTA-granularity part reaches kEtwcSpill arcs would otherwise keep one CTA
// busy while the others idle (a hub on a power-law graph: RMAT-22's first
// round is one 163K-arc vertex); such entries go to a list that a second
// pass spreads over every CTA (k_push_etwc_spill).  q == null: no hand-off,
// every entry stays with its CTA, as in Algorithm 3.
constexpr int32_t kEtwcSpill = 4096;
template <class S>
struct EtwcSpill {
    EtwcEntry<S> *q;
    int32_t *cnt;
};

template <class Op>
__device__ void lb_etwc(const DevGraph &g, const FrontierIn &fin, int32_t fsize, const Op &op,
                        const OutCtx &out, int bid, int nb, unsigned long long *ctr,
                        EtwcSpill<typename Op::S> spill = {nullptr, nullptr}) {
    typedef typename Op::S S;
    __shared__ EtwcEntry<S> q0[kCta], q1[kCta], q2[kCta];
    __shared__ int n0, n1, n2;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int64_t base = (int64_t)bid * kCta; base < fsize; base += (int64_t)nb * kCta) {
        if (tid == 0) n0 = n1 = n2 = 0;
        __syncthreads();
        int32_t i = (int32_t)base + tid;
        int len0 = 0;
        if (i < fsize) {
            int32_t u = fin.vertex(i);
            S s = op.load(u);
            if (!op.skip(s)) {
                int32_t beg = g.rowptr[u], end = g.rowptr[u + 1];
                int32_t size = end - beg;
                len0 = size;
                int32_t c = (size / kCta) * kCta;  // CTA-granularity part
                if (c > 0) {
                    if (spill.q && c >= kEtwcSpill) {
                        spill.q[atomicAdd(spill.cnt, 1)] = EtwcEntry<S>{beg, beg + c, u, s};
                    } else {
                        int p = atomicAdd(&n2, 1);
                        q2[p] = EtwcEntry<S>{beg, beg + c, u, s};
                    }
                    beg += c;
                    size -= c;
                }
                int32_t wpart = (size / 32) * 32;  // warp-granularity part
                if (wpart > 0) {
                    int p = atomicAdd(&n1, 1);
                    q1[p] = EtwcEntry<S>{beg, beg + wpart, u, s};
                    beg += wpart;
                    size -= wpart;
                }
                if (size > 0) {  // remainder, < 32 arcs
                    int p = atomicAdd(&n0, 1);
                    q0[p] = EtwcEntry<S>{beg, end, u, s};
                }
            }
        }
        count_arcs(ctr, len0);
        __syncthreads();
        // stage 0: one thread per entry
        {
            int32_t beg = 0, len = 0, u = 0;
            S s{};
            if (tid < n0) {
                beg = q0[tid].beg;
                len = q0[tid].end - beg;
                u = q0[tid].u;
                s = q0[tid].s;
            }
            int maxlen = (int)__reduce_max_sync(G2_FULL, (unsigned)len);
            for (int k = 0; k < maxlen; ++k) {
                int code = 0;
                int32_t v = 0;
                if (k < len) {
                    v = g.col[beg + k];
                    code = op.relax(u, s, v, beg + k);
                }
                emit(out, v, code);
            }
        }
        // stage 1: one warp per entry, lanes cyclic
        for (int j = wid; j < n1; j += kWarps) {
            EtwcEntry<S> en = q1[j];
            for (int32_t e = en.beg + lane; e < en.end; e += 32) {
                int32_t v = g.col[e];
                emit(out, v, op.relax(en.u, en.s, v, e));
            }
        }
        // stage 2: the whole CTA per entry
        for (int j = 0; j < n2; ++j) {
            EtwcEntry<S> en = q2[j];
            for (int32_t e = en.beg + tid; e < en.end; e += kCta) {
                int32_t v = g.col[e];
                emit(out, v, op.relax(en.u, en.s, v, e));
            }
        }
        __syncthreads();
    }
}

// The handed-off entries, spread over the grid: entry j's arcs in chunks of
// kCta arcs, chunk c of every entry taken by CTA c mod gridDim.x.
template <class Op>
__device__ void lb_etwc_spill(const DevGraph &g, const EtwcEntry<typename Op::S> *q,
                              const int32_t *cnt, const Op &op, const OutCtx &out, int bid,
                              int nb) {
    const int32_t k = *cnt;
    const int lane = threadIdx.x & 31;
    for (int32_t j = 0; j < k; ++j) {
        const EtwcEntry<typename Op::S> en = q[j];
        // a warp takes 32 consecutive arcs a step, lanes past the entry's end
        // emit nothing, so every lane reaches the warp-wide append (entries
        // are whole multiples of kCta arcs, but the loop does not rely on it)
        for (int64_t base = en.beg + (int64_t)bid * kCta + (threadIdx.x & ~31); base < en.end;
             base += (int64_t)nb * kCta) {
            const int64_t e = base + lane;
            int32_t v = 0;
            int code = 0;
            if (e < en.end) {
                v = g.col[e];
                code = op.relax(en.u, en.s, v, (int32_t)e);
            }
            emit(out, v, code);
        }
    }
}

// ----------------------------------------------------------------------- TWC
// Frontier-wide degree buckets (Merrill et al.): a classification pass puts
// each active vertex into the small (< 32 arcs), medium (< kCta) or large
// queue; then small vertices are walked by one thread, medium by a warp and
// large by a whole CTA.
template <class Op>
__device__ void lb_twc_classify(const DevGraph &g, const FrontierIn &fin, int32_t fsize,
                                const Op &op, int32_t *qs, int32_t *qm, int32_t *ql,
                                int32_t *counts, int bid, int nb) {
    const int lane = threadIdx.x & 31;
    const int gw = bid * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = nb * (blockDim.x >> 5);
    for (int64_t base = (int64_t)gw * 32; base < fsize; base += (int64_t)nw * 32) {
        int32_t i = (int32_t)base + lane;
        int32_t u = 0, deg = 0;
        if (i < fsize) {
            u = fin.vertex(i);
            if (!op.skip(op.load(u))) deg = g.rowptr[u + 1] - g.rowptr[u];
        }
        warp_append(qs, counts + 0, fsize, nullptr, u, deg > 0 && deg < 32);
        warp_append(qm, counts + 1, fsize, nullptr, u, deg >= 32 && deg < kCta);
        warp_append(ql, counts + 2, fsize, nullptr, u, deg >= kCta);
    }
}

template <class Op>
__device__ void lb_twc_process(const DevGraph &g, const int32_t *qs, const int32_t *qm,
                               const int32_t *ql, const int32_t *counts, const Op &op,
                               const OutCtx &out, int bid, int nb, unsigned long long *ctr) {
    typedef typename Op::S S;
    const int tid = threadIdx.x, lane = tid & 31;
    const int gw = bid * kWarps + (tid >> 5);
    const int nw = nb * kWarps;
    const int32_t ns = counts[0], nm = counts[1], nl = counts[2];
    // small: thread per vertex
    for (int64_t base = (int64_t)gw * 32; base < ns; base += (int64_t)nw * 32) {
        int32_t i = (int32_t)base + lane;
        int32_t u = 0, beg = 0, len = 0;
        S s{};
        if (i < ns) {
            u = qs[i];
            s = op.load(u);
            beg = g.rowptr[u];
            len = g.rowptr[u + 1] - beg;
        }
        count_arcs(ctr, len);
        int maxlen = (int)__reduce_max_sync(G2_FULL, (unsigned)len);
        for (int k = 0; k < maxlen; ++k) {
            int code = 0;
            int32_t v = 0;
            if (k < len) {
                v = g.col[beg + k];
                code = op.relax(u, s, v, beg + k);
            }
            emit(out, v, code);
        }
    }
    // medium: warp per vertex
    for (int32_t j = gw; j < nm; j += nw) {
        int32_t u = qm[j];
        S s = op.load(u);
        int32_t beg = g.rowptr[u], end = g.rowptr[u + 1];
        if (ctr && lane == 0) atomicAdd(ctr, (unsigned long long)(end - beg));
        for (int32_t e0 = beg; e0 < end; e0 += 32) {
            int32_t e = e0 + lane;
            int code = 0;
            int32_t v = 0;
            if (e < end) {
                v = g.col[e];
                code = op.relax(u, s, v, e);
            }
            emit(out, v, code);
        }
    }
    // large: CTA per vertex
    for (int32_t j = bid; j < nl; j += nb) {
        int32_t u = ql[j];
        S s = op.load(u);
        int32_t beg = g.rowptr[u], end = g.rowptr[u + 1];
        if (ctr && tid == 0) atomicAdd(ctr, (unsigned long long)(end - beg));
        for (int32_t e0 = beg; e0 < end; e0 += kCta) {
            int32_t e = e0 + tid;
            int code = 0;
            int32_t v = 0;
            if (e < end) {
                v = g.col[e];
                code = op.relax(u, s, v, e);
            }
            emit(out, v, code);
        }
    }
}

// ----------------------------------------------------------------- EDGE_ONLY
// Arc-parallel over arcs [e0, e1) of a COO (src[], dst[]) array: the whole
// edge set, or one EdgeBlocking segment (Algorithm 2's cooperative for).
template <class Op>
__device__ void lb_edges(const int32_t *src, const int32_t *dst, int64_t e0, int64_t e1,
                         const Op &op, const OutCtx &out, int bid, int nb,
                         unsigned long long *ctr) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)bid * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)nb * (blockDim.x >> 5);
    int cnt = 0;
    for (int64_t base = e0 + gw * 32; base < e1; base += nw * 32) {
        int64_t e = base + lane;
        int code = 0;
        int32_t v = 0;
        if (e < e1) {
            int32_t u = src[e];
            v = dst[e];
            typename Op::S s = op.load(u);
            if (!op.skip(s)) code = op.relax(u, s, v, (int32_t)e);
            ++cnt;
        }
        emit(out, v, code);
    }
    count_arcs(ctr, cnt);
}

// ---------------------------------------------------------------- PULL side
// Destinations v in [0, n) (or the items of a candidate list) that pass the
// filter scan their in-neighbours u (CSC, ascending) that are in the input
// frontier.  Group size 1 (VERTEX_BASED), 32 (WM) or kCta (CM) threads per
// destination; the group combines its partial results and may stop early.
template <class P, int G>
__device__ void lb_pull(const DevGraph &g, const int32_t *cand, int32_t ncand, const Member &mem,
                        const P &op, const OutCtx &out, int bid, int nb, unsigned long long *ctr) {
    typedef typename P::Acc Acc;
    typedef typename P::Ctx Ctx;
    const int tid = threadIdx.x, lane = tid & 31;
    if (G == 1) {
        const int gw = bid * kWarps + (tid >> 5);
        const int nw = nb * kWarps;
        for (int64_t base = (int64_t)gw * 32; base < ncand; base += (int64_t)nw * 32) {
            int32_t i = (int32_t)base + lane;
            int code = 0;
            int32_t v = 0;
            int cnt = 0;
            if (i < ncand) {
                v = cand ? cand[i] : i;
                Ctx c = op.ctx(v);
                if (op.filter(c)) {
                    Acc acc = op.identity();
                    int32_t e1 = g.crowptr[v + 1];
                    for (int32_t e = g.crowptr[v]; e < e1; ++e) {
                        int32_t u = g.ccol[e];
                        ++cnt;
                        if (mem.has(u)) {
                            acc = op.combine(acc, op.edge(c, u, e));
                            if (op.stop(acc)) break;
                        }
                    }
                    code = op.finish(v, c, acc);
                }
            }
            count_arcs(ctr, cnt);
            if (out.mode == OUT_BITMAP && !cand) {
                // the warp's 32 destinations are one aligned bitmap word
                unsigned mask = __ballot_sync(G2_FULL, code & 1);
                if (lane == 0 && mask) atomicOr(&out.bitmap[base >> 5], mask);
            } else {
                emit(out, v, code);
            }
        }
    } else if (G == 32) {
        const int gw = bid * kWarps + (tid >> 5);
        const int nw = nb * kWarps;
        for (int32_t i = gw; i < ncand; i += nw) {
            int32_t v = cand ? cand[i] : i;
            Ctx c = op.ctx(v);
            int code = 0;
            int cnt = 0;
            if (op.filter(c)) {
                Acc acc = op.identity();
                int32_t e1 = g.crowptr[v + 1];
                for (int32_t e0 = g.crowptr[v]; e0 < e1; e0 += 32) {
                    int32_t e = e0 + lane;
                    Acc a = op.identity();
                    if (e < e1) {
                        int32_t u = g.ccol[e];
                        ++cnt;
                        if (mem.has(u)) a = op.edge(c, u, e);
                    }
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) a = op.combine(a, shfl_xor_acc(a, d));
                    acc = op.combine(acc, a);
                    if (op.stop(acc)) break;
                }
                if (lane == 0) code = op.finish(v, c, acc);
            }
            count_arcs(ctr, cnt);
            // one destination per warp: only lane 0 may emit
            emit(out, v, code);
        }
    } else {
        __shared__ Acc s_red[kWarps];
        __shared__ int s_stop;
        for (int32_t i = bid; i < ncand; i += nb) {
            int32_t v = cand ? cand[i] : i;
            Ctx c = op.ctx(v);
            int code = 0;
            int cnt = 0;
            if (op.filter(c)) {
                Acc acc = op.identity();
                int32_t e1 = g.crowptr[v + 1];
                for (int32_t e0 = g.crowptr[v]; e0 < e1; e0 += kCta) {
                    int32_t e = e0 + tid;
                    Acc a = op.identity();
                    if (e < e1) {
                        int32_t u = g.ccol[e];
                        ++cnt;
                        if (mem.has(u)) a = op.edge(c, u, e);
                    }
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) a = op.combine(a, shfl_xor_acc(a, d));
                    if (lane == 0) s_red[tid >> 5] = a;
                    __syncthreads();
                    if (tid == 0) {
                        Acc t = s_red[0];
                        for (int k = 1; k < kWarps; ++k) t = op.combine(t, s_red[k]);
                        acc = op.combine(acc, t);
                        s_stop = op.stop(acc);
                    }
                    __syncthreads();
                    if (s_stop) break;
                }
                if (tid == 0) code = op.finish(v, c, acc);
            }
            count_arcs(ctr, cnt);
            emit(out, v, code);
            __syncthreads();
        }
    }
}

}  // namespace g2
