// g2_pr.cu — PageRank, the topology-driven algorithm of Sec. VII: every round
// sweeps all arcs.  Round t computes
//   x_t[v] = (1-d)/n + d * ( sum_{u->v} x_{t-1}[u]/outdeg(u) + D_{t-1}/n ),
// D = total rank of the vertices without out-arcs (spread uniformly).
//
// Schedules:
//  PULL + EDGE_ONLY (the default): arc-balanced segmented sums over the CSC.
//    Rows and arcs are merged into one sequence of n + m items (merge-path
//    partitioning) cut into equal tiles, so every CTA gets the same share of
//    row ends and arcs whatever the degree distribution; no atomics except
//    for the few rows cut by a tile boundary.  The next round's per-source
//    shares and the dangling mass are produced in the same pass.
//  PULL + VERTEX_BASED / WM / CM: one thread / warp / CTA per destination.
//  PUSH + any load balancing over the all-vertices frontier, including
//    EDGE_ONLY with EdgeBlocking (Algorithms 1-2): arc-parallel atomic adds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "g2_host.h"
#include "g2_lb.cuh"

namespace g2 {

constexpr int kPrIPT = 8;                 // merge items per thread per tile
constexpr int kPrTile = kCta * kPrIPT;    // merge items per tile

struct PrArgs {
    int32_t n;
    int32_t m;
    const int32_t *crowptr;
    const int32_t *ccol;
    const int32_t *rowptr;   // CSR offsets for out-degrees (null: symmetric, use CSC)
    const int32_t *tile_r;   // merge-path row coordinate of every tile boundary
    int32_t ntiles;
    const float *contrib;    // x_{t-1}[u] / outdeg(u)
    float *contrib_next;
    float *x;                // written when write_x
    int write_x;
    float *acc;              // partial sums of rows cut by a tile boundary (kept zero)
    const double *dprev;     // D_{t-1}
    double *dnext;           // D_t accumulator (zeroed before the launch)
    float base;              // (1-d)/n
    float damp;
    double inv_n;
};

// Merge-path search: how many row ends precede merged item `diag` when row
// ends a[] (one past each row's last arc) are merged with arc indices.
__device__ __forceinline__ int32_t merge_rows_global(const int32_t *a, int32_t na, int64_t nb,
                                                     int64_t diag) {
    int64_t lo = diag - nb > 0 ? diag - nb : 0;
    int64_t hi = diag < na ? diag : na;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] <= diag - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    return (int32_t)lo;
}

__global__ void k_pr_tiles(const int32_t *crowptr, int32_t n, int32_t m, int32_t ntiles,
                           int32_t *tile_r) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= ntiles;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t diag = b * kPrTile;
        int64_t total = (int64_t)n + m;
        if (diag > total) diag = total;
        tile_r[b] = merge_rows_global(crowptr + 1, n, m, diag);
    }
}

// rows cut by a tile boundary, each listed once (at its first cut)
__global__ void k_pr_split_rows(const int32_t *crowptr, int32_t n, int32_t ntiles,
                                const int32_t *tile_r, int32_t *list, int32_t *cnt) {
    int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < ntiles;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = base + lane;
        bool split = false;
        int32_t r = 0;
        if (b >= 1 && b < ntiles) {
            r = tile_r[b];
            int64_t e = b * kPrTile - r;
            split = r < n && crowptr[r] < e;
            if (split && b >= 2 && tile_r[b - 1] == r) {
                int64_t ep = (b - 1) * (int64_t)kPrTile - r;
                if (crowptr[r] < ep) split = false;  // already cut at an earlier boundary
            }
        }
        warp_append(list, cnt, ntiles + 1, nullptr, r, split);
    }
}

__device__ __forceinline__ void pr_finalize(const PrArgs &a, int32_t r, float y, int32_t in_beg,
                                            int32_t in_end, float dterm, double &dsum) {
    float xr = a.base + a.damp * (y + dterm);
    int32_t od = a.rowptr ? a.rowptr[r + 1] - a.rowptr[r] : in_end - in_beg;
    if (od > 0) {
        a.contrib_next[r] = xr / (float)od;
    } else {
        a.contrib_next[r] = 0.f;
        dsum += xr;
    }
    if (a.write_x) a.x[r] = xr;
}

__device__ __forceinline__ void block_add_double(double v, double *target) {
    __shared__ double s_red[kWarps];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(G2_FULL, v, d);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < kWarps; ++k) t += s_red[k];
        if (t != 0.0) atomicAdd(target, t);
    }
}

// Tile coordinates on the merge path: rows r0..r1 (r1 partial), arcs e0..e1.
struct PrTile {
    int32_t r0, r1, e0, e1;
};

__device__ __forceinline__ PrTile pr_tile(const PrArgs &a, int32_t tile) {
    const int64_t total = (int64_t)a.n + a.m;
    const int64_t d0 = (int64_t)tile * kPrTile;
    const int64_t d1 = d0 + kPrTile < total ? d0 + kPrTile : total;
    PrTile c;
    c.r0 = a.tile_r[tile];
    c.r1 = a.tile_r[tile + 1];
    c.e0 = (int32_t)(d0 - c.r0);
    c.e1 = (int32_t)(d1 - c.r1);
    return c;
}

// Stage layout of one tile in shared memory: the arc slice [e0 & ~3, ...)
// rounded to whole 16-byte chunks, then the row-end slice crowptr[(r0+1) & ~3
// ...] likewise.  Both come in by TMA bulk copies counted on one mbarrier.
struct PrStage {
    int32_t ea, ne_al, ra, nr_al;
};

__device__ __forceinline__ PrStage pr_stage(const PrTile &c) {
    PrStage s;
    s.ea = c.e0 & ~3;
    s.ne_al = ((c.e1 - s.ea) + 3) & ~3;
    s.ra = (c.r0 + 1) & ~3;
    s.nr_al = ((c.r1 + 2 - s.ra) + 3) & ~3;
    return s;
}

constexpr int kPrBuf = kPrTile + 32;  // ints per stage (slices + rounding)

__device__ __forceinline__ void pr_issue(const PrArgs &a, const PrTile &c, int32_t *buf,
                                         uint64_t *bar) {
    PrStage s = pr_stage(c);
    mbar_arrive_expect_tx(bar, (uint32_t)(s.ne_al + s.nr_al) * 4u);
    if (s.ne_al > 0) tma_load_1d(buf, a.ccol + s.ea, (uint32_t)s.ne_al * 4u, bar);
    tma_load_1d(buf + s.ne_al, a.crowptr + s.ra, (uint32_t)s.nr_al * 4u, bar);
}

__global__ void __launch_bounds__(kCta) k_pr_merge(PrArgs a, uint64_t limit_ns, int32_t *err) {
    __shared__ __align__(16) int32_t buf[2][kPrBuf];
    __shared__ float s_acc[kPrTile + 1];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x, lane = tid & 31;
    const float dterm = (float)(*a.dprev * a.inv_n);
    double dsum = 0.0;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    int32_t tile = blockIdx.x;
    if (tid == 0 && tile < a.ntiles) pr_issue(a, pr_tile(a, tile), buf[0], &bar[0]);
    uint32_t phase0 = 0, phase1 = 0;
    for (int s = 0; tile < a.ntiles; tile += gridDim.x, s ^= 1) {
        const PrTile c = pr_tile(a, tile);
        const int32_t next = tile + gridDim.x;
        // prefetch the next tile into the other stage (freed by the barrier
        // that ended the previous tile)
        if (tid == 0 && next < a.ntiles) pr_issue(a, pr_tile(a, next), buf[s ^ 1], &bar[s ^ 1]);
        const uint32_t ph = s ? phase1 : phase0;
        bool ok = mbar_wait_bounded(&bar[s], ph, limit_ns);
        if (s) phase1 ^= 1u;
        else phase0 ^= 1u;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                set_error(err, G2_ETIMEOUT);
                // let the prefetch already issued land before the CTA exits
                if (next < a.ntiles) mbar_wait_bounded(&bar[s ^ 1], s ? phase0 : phase1, limit_ns);
            }
            break;
        }
        const PrStage sg = pr_stage(c);
        int32_t *scol = buf[s] + (c.e0 - sg.ea);                   // arc j of the tile
        const int32_t *send = buf[s] + sg.ne_al + (c.r0 + 1 - sg.ra);  // end of row r0+i
        const int32_t nr = c.r1 - c.r0, ne = c.e1 - c.e0;
        const bool last_row_real = c.r1 < a.n;
        for (int32_t i = tid; i <= nr; i += kCta) s_acc[i] = 0.f;
        // this thread's slice [dl, dl2) of the merged sequence
        const int32_t items = nr + ne;
        int32_t dl = tid * kPrIPT;
        if (dl > items) dl = items;
        const int32_t dl2 = dl + kPrIPT < items ? dl + kPrIPT : items;
        int32_t ri, ej, ej2;
        {
            int32_t lo = dl - ne > 0 ? dl - ne : 0, hi = dl < nr ? dl : nr;
            while (lo < hi) {
                int32_t mid = (lo + hi) >> 1;
                if (send[mid] <= c.e0 + (dl - mid - 1)) lo = mid + 1;
                else hi = mid;
            }
            ri = lo;
            ej = dl - lo;
            lo = dl2 - ne > 0 ? dl2 - ne : 0;
            hi = dl2 < nr ? dl2 : nr;
            if (lo < ri) lo = ri;
            while (lo < hi) {
                int32_t mid = (lo + hi) >> 1;
                if (send[mid] <= c.e0 + (dl2 - mid - 1)) lo = mid + 1;
                else hi = mid;
            }
            ej2 = dl2 - lo;
        }
        // gather the shares of this thread's arcs (independent loads), write
        // them over the arc ids, which no other thread reads
        {
            const int32_t ne_t = ej2 - ej;
            float v[kPrIPT];
#pragma unroll
            for (int k = 0; k < kPrIPT; ++k)
                v[k] = k < ne_t ? __ldg(a.contrib + scol[ej + k]) : 0.f;
#pragma unroll
            for (int k = 0; k < kPrIPT; ++k)
                if (k < ne_t) scol[ej + k] = __float_as_int(v[k]);
        }
        __syncthreads();  // s_acc zeroed everywhere before the adds
        int32_t row_end = (ri < nr || last_row_real) ? send[ri] : G2_INF32;
        float run = 0.f;
        for (int32_t k = dl; k < dl2; ++k) {
            if (c.e0 + ej < row_end) {
                run += __int_as_float(scol[ej]);
                ++ej;
            } else {
                if (run != 0.f) atomicAdd(&s_acc[ri], run);
                run = 0.f;
                ++ri;
                row_end = (ri < nr || last_row_real) ? send[ri] : G2_INF32;
            }
        }
        // carry of the unfinished row: combine equal rows across the warp
        // (row ids do not decrease with the lane), one atomic per row
        int32_t key = ri;
        float v = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            float ov = __shfl_up_sync(G2_FULL, v, d);
            int32_t ok2 = __shfl_up_sync(G2_FULL, key, d);
            if (lane >= d && ok2 == key) v += ov;
        }
        int32_t nk = __shfl_down_sync(G2_FULL, key, 1);
        if ((lane == 31 || nk != key) && v != 0.f) atomicAdd(&s_acc[key], v);
        __syncthreads();
        // finish the rows that ended in this tile
        for (int32_t i = tid; i < nr; i += kCta) {
            int32_t r = c.r0 + i;
            int32_t beg = i == 0 ? a.crowptr[c.r0] : send[i - 1];
            if (i == 0 && beg < c.e0) {
                atomicAdd(&a.acc[r], s_acc[0]);  // started in an earlier tile
                continue;
            }
            pr_finalize(a, r, s_acc[i], beg, send[i], dterm, dsum);
        }
        if (tid == 0 && last_row_real) {
            int32_t beg1 = nr > 0 ? send[nr - 1] : a.crowptr[c.r1];
            if (c.e1 > beg1) atomicAdd(&a.acc[c.r1], s_acc[nr]);  // continues in a later tile
        }
        __syncthreads();
    }
    block_add_double(dsum, a.dnext);
}

__global__ void __launch_bounds__(kCta) k_pr_fixup(PrArgs a, const int32_t *rows,
                                                   const int32_t *nrows) {
    const float dterm = (float)(*a.dprev * a.inv_n);
    double dsum = 0.0;
    const int32_t cnt = *nrows;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        int32_t r = rows[i];
        float y = a.acc[r];
        a.acc[r] = 0.f;
        pr_finalize(a, r, y, a.crowptr[r], a.crowptr[r + 1], dterm, dsum);
    }
    block_add_double(dsum, a.dnext);
}

// x0 = 1/n: contrib0[u] = (1/n)/outdeg(u); D0 = (#vertices without out-arcs)/n
__global__ void __launch_bounds__(kCta) k_pr_init(const int32_t *rowptr, int32_t n, float *contrib,
                                                  double *d0, float *x, double inv_n) {
    double dsum = 0.0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int32_t od = rowptr[u + 1] - rowptr[u];
        contrib[u] = od > 0 ? (float)(inv_n / od) : 0.f;
        if (od == 0) dsum += inv_n;
        if (x) x[u] = (float)inv_n;
    }
    block_add_double(dsum, d0);
}

// generic schedules: x from the accumulated sums, next shares, next D
__global__ void __launch_bounds__(kCta) k_pr_vertex(const int32_t *rowptr, int32_t n,
                                                    const float *acc, float *contrib_next,
                                                    float *x, const double *dprev, double *dnext,
                                                    float base, float damp, double inv_n) {
    const float dterm = (float)(*dprev * inv_n);
    double dsum = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        float xr = base + damp * (acc[v] + dterm);
        int32_t od = rowptr[v + 1] - rowptr[v];
        if (od > 0) contrib_next[v] = xr / (float)od;
        else {
            contrib_next[v] = 0.f;
            dsum += xr;
        }
        x[v] = xr;
    }
    block_add_double(dsum, dnext);
}

static int pr_blocks(const g2_graph *g) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pr_merge, kCta, 0) != cudaSuccess ||
            b < 1)
            b = 1;
        per_sm = b;
    }
    return g->topo->sm_count * per_sm;
}

g2_status pagerank_run(g2_graph *g, float damping, int32_t iters, float *rank, const g2_hybrid &h,
                       bool tuned_default, cudaStream_t st, int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    if (n == 0) return G2_OK;
    const double inv_n = 1.0 / (double)n;
    float *cbuf[2], *acc;
    G2_TRY(ws(g, B_F0, (size_t)n, &cbuf[0]));
    G2_TRY(ws(g, B_F1, (size_t)n, &cbuf[1]));
    G2_TRY(ws(g, B_F2, (size_t)n + 1, &acc));
    double *dd;
    G2_TRY(ws(g, B_D1, 4, &dd));
    G2_CK(cudaMemsetAsync(dd, 0, 4 * sizeof(double), st));
    k_pr_init<<<grid_for(g, n, kCta), kCta, 0, st>>>(t->rowptr, n, cbuf[0], dd, rank, inv_n);
    stats().launches += 1;
    if (iters <= 0) return G2_OK;
    const g2_schedule &s = h.s1;  // one schedule for every round (the frontier is always all vertices)
    const float base = (float)((1.0 - damping) * inv_n);
    const bool merge = tuned_default || (s.direction == G2_PULL && s.load_balance == G2_LB_EDGE_ONLY);
    if (!merge) {
        G2_TRY(check_schedule(g, s, K_PR, true));
        if (s.kernel_fusion) return fail(G2_EUNSUPPORTED, "PageRank has no fused variant");
    }
    if (merge) {
        const int64_t total = (int64_t)n + t->m;
        const int32_t ntiles = (int32_t)((total + kPrTile - 1) / kPrTile);
        int32_t *tile_r, *split, *ctrs = d_err - 62;
        G2_TRY(ws(g, B_SCAN, (size_t)ntiles + 2, &tile_r));
        G2_TRY(ws(g, B_TWC_M, (size_t)ntiles + 2, &split));
        G2_CK(cudaMemsetAsync(acc, 0, (size_t)(n + 1) * 4, st));
        G2_CK(cudaMemsetAsync(ctrs + 10, 0, 4, st));
        k_pr_tiles<<<grid_for(g, ntiles + 1, kCta), kCta, 0, st>>>(t->crowptr, n, t->m, ntiles,
                                                                   tile_r);
        k_pr_split_rows<<<grid_for(g, ntiles, kCta), kCta, 0, st>>>(t->crowptr, n, ntiles, tile_r,
                                                                    split, ctrs + 10);
        stats().launches += 2;
        const int grid = std::min<int64_t>(ntiles, pr_blocks(g));
        PrArgs a;
        a.n = n;
        a.m = t->m;
        a.crowptr = t->crowptr;
        a.ccol = t->ccol;
        a.rowptr = t->symmetric ? nullptr : t->rowptr;
        a.tile_r = tile_r;
        a.ntiles = ntiles;
        a.acc = acc;
        a.base = base;
        a.damp = damping;
        a.inv_n = inv_n;
        a.x = rank;
        for (int32_t it = 0; it < iters; ++it) {
            a.contrib = cbuf[it & 1];
            a.contrib_next = cbuf[(it + 1) & 1];
            a.write_x = it == iters - 1;
            a.dprev = dd + (it & 1);
            a.dnext = dd + ((it + 1) & 1);
            G2_CK(cudaMemsetAsync(dd + ((it + 1) & 1), 0, sizeof(double), st));
            KTime kt;
            ktime_begin(kt, "pr_merge", st);
            k_pr_merge<<<grid, kCta, 0, st>>>(a, 2000000000ULL, d_err);
            ktime_end(kt, st);
            k_pr_fixup<<<(ntiles + kCta) / kCta, kCta, 0, st>>>(a, split, ctrs + 10);
            stats().launches += 2;
            stats().iterations++;
            stats().pull_rounds++;
        }
        G2_CK(cudaGetLastError());
        return G2_OK;
    }
    VSet all{-1, nullptr, 0, nullptr, nullptr, nullptr, n};
    OutArgs none;
    memset(&none, 0, sizeof(none));
    none.rep = OUT_NONE;
    for (int32_t it = 0; it < iters; ++it) {
        OpArgs a;
        memset(&a, 0, sizeof(a));
        a.kind = K_PR;
        a.f0 = cbuf[it & 1];
        a.f1 = acc;
        a.err = d_err;
        G2_CK(cudaMemsetAsync(acc, 0, (size_t)n * 4, st));
        G2_CK(cudaMemsetAsync(dd + ((it + 1) & 1), 0, sizeof(double), st));
        G2_TRY(apply_round(g, s, a, all, none, st));
        k_pr_vertex<<<grid_for(g, n, kCta), kCta, 0, st>>>(t->rowptr, n, acc, cbuf[(it + 1) & 1],
                                                           rank, dd + (it & 1), dd + ((it + 1) & 1),
                                                           base, damping, inv_n);
        stats().launches += 1;
        stats().iterations++;
        s.direction == G2_PUSH ? stats().push_rounds++ : stats().pull_rounds++;
    }
    G2_CK(cudaGetLastError());
    return G2_OK;
}

}  // namespace g2

using namespace g2;

extern "C" g2_status g2_pagerank(g2_graph *g, float damping, int32_t iters, float *rank,
                                 const g2_hybrid *sched, void *stream) {
    if (!g || !rank) return fail(G2_EINVAL, "null graph or rank");
    if (iters < 0 || !(damping >= 0.f && damping <= 1.f))
        return fail(G2_EINVAL, "iters must be >= 0 and damping in [0, 1]");
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : default_hybrid();
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    G2_TRY(pagerank_run(g, damping, iters, rank, h, sched == nullptr, st, d_err));
    return end_call(g, st, d_err);
}
