// g2_pr.cu — PageRank, the topology-driven algorithm of Sec. VII: every round
// sweeps all arcs.  Round t computes
//   x_t[v] = (1-d)/n + d * ( sum_{u->v} x_{t-1}[u]/outdeg(u) + D_{t-1}/n ),
// D = total rank of the vertices without out-arcs (spread uniformly).
//
// Schedules:
//  PULL + EDGE_ONLY (the default): arc-balanced sums over the CSC.  The tuned
//    kernel is a segmented sweep (g2_pr_seg.cuh): every warp takes 128
//    consecutive arcs, gathers their shares and adds them per row with a
//    warp segmented scan over precomputed row-head flags; a vertex pass then
//    forms x_t, the next shares and the next dangling mass.  The shares of the
//    H highest-degree vertices are held in shared memory for the whole launch
//    (a one-time layout step renumbers the CSC's column ids so that those
//    vertices come first); the other gathers go through L1/L2.  A merge-path
//    tile kernel (rows and arcs merged into one sequence of n + m items cut
//    into equal tiles, arc slices and row ends brought in by TMA bulk copies,
//    double-buffered) is kept as the alternative (G2_PR_KERNEL=merge).
//  PULL + VERTEX_BASED / WM / CM: one thread / warp / CTA per destination.
//  PUSH + any load balancing over the all-vertices frontier, including
//    EDGE_ONLY with EdgeBlocking (Algorithms 1-2): arc-parallel atomic adds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "g2_host.h"
#include "g2_lb.cuh"
#include "g2_pr_blk.cuh"
#include "g2_pr_seg.cuh"

namespace g2 {

struct PrArgs {
    int32_t n;
    int32_t m;
    int32_t tile;            // merged items per tile
    const int32_t *crowptr;
    const int32_t *ccol;     // column ids as share slots (renumbered with a hot layout)
    const int32_t *rowptr;   // CSR offsets for out-degrees (null: symmetric, use CSC)
    const int32_t *slot_of;  // share slot of every vertex (hot > 0)
    int32_t hot_min_deg;     // every cached vertex has at least this out-degree
    const int32_t *tile_r;   // merge-path row coordinate of every tile boundary
    int32_t ntiles;
    int32_t hot;             // shares [0, hot) are cached in shared memory
    const float *contrib;    // share slot -> x_{t-1}[u] / outdeg(u)
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

__global__ void k_pr_tiles(const int32_t *crowptr, int32_t n, int32_t m, int32_t tile,
                           int32_t ntiles, int32_t *tile_r) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= ntiles;
         b += (int64_t)gridDim.x * blockDim.x) {
        int64_t diag = b * tile;
        int64_t total = (int64_t)n + m;
        if (diag > total) diag = total;
        tile_r[b] = merge_rows_global(crowptr + 1, n, m, diag);
    }
}

// rows cut by a tile boundary, each listed once (at its first cut)
__global__ void k_pr_split_rows(const int32_t *crowptr, int32_t n, int32_t tile, int32_t ntiles,
                                const int32_t *tile_r, int32_t *list, int32_t *cnt) {
    int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < ntiles;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = base + lane;
        bool split = false;
        int32_t r = 0;
        if (b >= 1 && b < ntiles) {
            r = tile_r[b];
            int64_t e = b * tile - r;
            split = r < n && crowptr[r] < e;
            if (split && b >= 2 && tile_r[b - 1] == r) {
                int64_t ep = (b - 1) * (int64_t)tile - r;
                if (crowptr[r] < ep) split = false;  // already cut at an earlier boundary
            }
        }
        warp_append(list, cnt, ntiles + 1, nullptr, r, split);
    }
}

// Share layout.  With H cached (hot) vertices, share slot H + v holds vertex
// v's share x[v]/outdeg(v) for every v, and slots 0..H-1 repeat the shares of
// the cached vertices, which the sweep keeps in shared memory; a CSC column id
// is renumbered to the cached slot or H + u (slot_of[u]).  Shares are written
// in vertex order; a vertex whose out-degree reaches min_deg (every cached
// vertex does) reads slot_of[v] and, if below H, writes that slot too.
// Without a hot layout H = 0 and slot v is vertex v.
struct ShareMap {
    int32_t hot;
    int32_t min_deg;
    const int32_t *slot_of;
};

__device__ __forceinline__ void store_cached_share(float *contrib, const ShareMap &sm, int32_t v,
                                                   int32_t od, float share) {
    if (sm.hot == 0 || od < sm.min_deg) return;
    const int32_t slot = __ldg(sm.slot_of + v);
    if (slot < sm.hot) contrib[slot] = share;
}

__device__ __forceinline__ void pr_finalize(const PrArgs &a, int32_t r, float y, int32_t in_beg,
                                            int32_t in_end, float dterm, double &dsum) {
    float xr = a.base + a.damp * (y + dterm);
    int32_t od = a.rowptr ? a.rowptr[r + 1] - a.rowptr[r] : in_end - in_beg;
    float share = 0.f;
    if (od > 0) share = xr / (float)od;
    else dsum += xr;
    a.contrib_next[a.hot + r] = share;
    store_cached_share(a.contrib_next, ShareMap{a.hot, a.hot_min_deg, a.slot_of}, r, od, share);
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
    const int64_t d0 = (int64_t)tile * a.tile;
    const int64_t d1 = d0 + a.tile < total ? d0 + a.tile : total;
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
// Rounding reads at most 3 + 4 elements past the slices; every device graph
// array carries kPad spare elements for that.
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

__device__ __forceinline__ void pr_issue(const PrArgs &a, const PrTile &c, int32_t *buf,
                                         uint64_t *bar) {
    PrStage s = pr_stage(c);
    mbar_arrive_expect_tx(bar, (uint32_t)(s.ne_al + s.nr_al) * 4u);
    if (s.ne_al > 0) tma_load_1d(buf, a.ccol + s.ea, (uint32_t)s.ne_al * 4u, bar);
    tma_load_1d(buf + s.ne_al, a.crowptr + s.ra, (uint32_t)s.nr_al * 4u, bar);
}

// shared-memory bytes of one launch configuration
__host__ __device__ constexpr size_t pr_smem_bytes(int ipt, int hot) {
    return (size_t)hot * 4                                  // hot shares
           + 2 * ((size_t)kCta * ipt + 32) * 4              // two stages
           + ((size_t)kCta * ipt + 4) * 4                   // row sums
           + ((size_t)kCta * ipt + kCta * ipt / 32) * 4     // padded gathered shares
           + 16;                                            // mbarriers
}

template <int IPT, bool HOT>
__global__ void __launch_bounds__(kCta) k_pr_merge(PrArgs a, uint64_t limit_ns, int32_t *err) {
    constexpr int TILE = kCta * IPT;
    constexpr int BUF = TILE + 32;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_hot = reinterpret_cast<float *>(smem);
    int32_t *buf0 = reinterpret_cast<int32_t *>(smem + (size_t)a.hot * 4);
    int32_t *buf1 = buf0 + BUF;
    float *s_acc = reinterpret_cast<float *>(buf1 + BUF);
    float *s_val = s_acc + TILE + 4;
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_val + TILE + TILE / 32);
    const int tid = threadIdx.x, lane = tid & 31;
    const float dterm = (float)(*a.dprev * a.inv_n);
    double dsum = 0.0;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (HOT)
        for (int32_t i = tid; i < a.hot; i += kCta) s_hot[i] = __ldg(a.contrib + i);
    __syncthreads();
    int32_t tile = blockIdx.x;
    if (tid == 0 && tile < a.ntiles) pr_issue(a, pr_tile(a, tile), buf0, &bar[0]);
    uint32_t phase0 = 0, phase1 = 0;
    for (int s = 0; tile < a.ntiles; tile += gridDim.x, s ^= 1) {
        int32_t *bufs = s ? buf1 : buf0;
        const PrTile c = pr_tile(a, tile);
        const int32_t next = tile + gridDim.x;
        // prefetch the next tile into the other stage (freed by the barrier
        // that ended the previous tile)
        if (tid == 0 && next < a.ntiles) pr_issue(a, pr_tile(a, next), s ? buf0 : buf1, &bar[s ^ 1]);
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
        const int32_t *scol = bufs + (c.e0 - sg.ea);                 // arc j of the tile
        const int32_t *send = bufs + sg.ne_al + (c.r0 + 1 - sg.ra);  // end of row r0+i
        const int32_t nr = c.r1 - c.r0, ne = c.e1 - c.e0;
        const bool last_row_real = c.r1 < a.n;
        for (int32_t i = tid; i <= nr; i += kCta) s_acc[i] = 0.f;
        // gather the shares of the tile's arcs with a strided assignment
        // (consecutive threads, consecutive arcs: coalesced, no bank conflicts),
        // IPT independent loads per thread, into a padded array (one spare
        // word per 32) so the contiguous per-thread reads below hit distinct
        // banks as well
        {
            float v[IPT];
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                int32_t j = tid + k * kCta;
                float x = 0.f;
                if (j < ne) {
                    int32_t u = scol[j];
                    x = (HOT && u < a.hot) ? s_hot[u] : __ldg(a.contrib + u);
                }
                v[k] = x;
            }
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                int32_t j = tid + k * kCta;
                if (j < ne) s_val[j + (j >> 5)] = v[k];
            }
        }
        // this thread's slice [dl, dl2) of the merged sequence
        const int32_t items = nr + ne;
        int32_t dl = tid * IPT;
        if (dl > items) dl = items;
        const int32_t dl2 = dl + IPT < items ? dl + IPT : items;
        int32_t ri, ej;
        {
            int32_t lo = dl - ne > 0 ? dl - ne : 0, hi = dl < nr ? dl : nr;
            while (lo < hi) {
                int32_t mid = (lo + hi) >> 1;
                if (send[mid] <= c.e0 + (dl - mid - 1)) lo = mid + 1;
                else hi = mid;
            }
            ri = lo;
            ej = dl - lo;
        }
        __syncthreads();  // s_acc zeroed and s_val filled before the adds
        int32_t row_end = (ri < nr || last_row_real) ? send[ri] : G2_INF32;
        float run = 0.f;
        for (int32_t k = dl; k < dl2; ++k) {
            if (c.e0 + ej < row_end) {
                run += s_val[ej + (ej >> 5)];
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


// Out-degrees of the four vertices v0..v0+3 of a quad.
struct PrQuad {
    int32_t od[4];
};

// Shares of a quad into slots H + v0 .. H + v0 + 3 (one 16-byte store for a
// full quad: H and v0 are multiples of 4), and the cached slots.
__device__ __forceinline__ void store_quad_shares(float *contrib, const ShareMap &sm, int32_t n,
                                                  int64_t v0, const PrQuad &q, const float sh[4]) {
    if (v0 + 4 <= n)
        *reinterpret_cast<float4 *>(contrib + sm.hot + v0) = make_float4(sh[0], sh[1], sh[2], sh[3]);
    else
        for (int k = 0; k < 4; ++k)
            if (v0 + k < n) contrib[sm.hot + v0 + k] = sh[k];
    for (int k = 0; k < 4; ++k)
        if (v0 + k < n) store_cached_share(contrib, sm, (int32_t)(v0 + k), q.od[k], sh[k]);
}

// Offsets rowptr[v0 .. v0+4] of a quad of four consecutive vertices, one
// quad per thread: a 16-byte load, the fifth offset from the next lane (the
// last lane of a warp and the last full quad load it).  Every lane of the
// warp must call it.
__device__ __forceinline__ bool pr_quad_offsets(const int32_t *rowptr, int32_t n, int64_t v0,
                                                int32_t r[5]) {
    const bool full = v0 + 4 <= n;
    for (int k = 0; k < 5; ++k) r[k] = 0;
    if (full) {
        const int4 r4 = *reinterpret_cast<const int4 *>(rowptr + v0);
        r[0] = r4.x; r[1] = r4.y; r[2] = r4.z; r[3] = r4.w;
    } else if (v0 < n) {
        for (int k = 0; k < 4; ++k)
            if (v0 + k <= n) r[k] = rowptr[v0 + k];
    }
    const int32_t r_next = __shfl_down_sync(G2_FULL, r[0], 1);
    if (full) r[4] = ((threadIdx.x & 31) == 31 || v0 + 4 == n) ? rowptr[v0 + 4] : r_next;
    return full;
}

// x0 = 1/n: shares (1/n)/outdeg(u) (fp32); D0 = (#vertices without out-arcs)/n
// into the D slots.  One quad of four consecutive vertices per thread.
__global__ void __launch_bounds__(kCta) k_pr_init(const int32_t *rowptr, int32_t n, ShareMap sm,
                                                  float *contrib, double *dslots, float *x,
                                                  double inv_n) {
    const int64_t v0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    int32_t r[5];
    const bool full = pr_quad_offsets(rowptr, n, v0, r);
    const float x0 = (float)inv_n;
    float dangling = 0.f;
    if (v0 < n) {
        PrQuad q;
        float sh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            q.od[k] = v0 + k < n ? r[k + 1] - r[k] : 0;
            sh[k] = q.od[k] > 0 ? x0 / (float)q.od[k] : 0.f;
            if (v0 + k < n && q.od[k] == 0) dangling += 1.f;
        }
        store_quad_shares(contrib, sm, n, v0, q, sh);
        if (x) {
            if (full && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0))
                *reinterpret_cast<float4 *>(x + v0) = make_float4(x0, x0, x0, x0);
            else
                for (int k = 0; k < 4 && v0 + k < n; ++k) x[v0 + k] = x0;
        }
    }
    // at most 128 per warp: exact in fp32; scaled by 1/n in fp64
    for (int o = 16; o > 0; o >>= 1) dangling += __shfl_xor_sync(G2_FULL, dangling, o);
    if ((threadIdx.x & 31) == 0 && dangling != 0.f) {
        const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        atomicAdd(dslots + (gw % kDSlots) * kDStride, (double)dangling * inv_n);
    }
}

// Folds the D slots into *fin (one warp).
__global__ void k_pr_fold(double *dslots, double *fin) { fold_dslots(dslots, fin); }

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

__global__ void k_remap_cols(const int32_t *ccol, const int32_t *perm, int32_t m, int32_t *out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = perm[ccol[e]];
}

__global__ void k_seg_heads(const int32_t *crowptr, int32_t n, uint32_t *head, int32_t *nz) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        int32_t b = crowptr[r], e = crowptr[r + 1];
        nz[r] = e > b;
        if (e > b) atomicOr(&head[b >> 5], 1u << (b & 31));
    }
}

__global__ void k_seg_nzrow(const int32_t *nz, const int32_t *pos, int32_t n, int32_t *nzrow) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        if (nz[r]) nzrow[pos[r]] = (int32_t)r;
}

__global__ void k_seg_chunk_heads(const uint32_t *head, int64_t nchunks, int32_t *cnt) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x)
        cnt[c] = __popc(head[4 * c]) + __popc(head[4 * c + 1]) + __popc(head[4 * c + 2]) +
                 __popc(head[4 * c + 3]);
}

// vertex pass after a segmented sweep: x, next shares, next D; y back to zero.
// Four consecutive vertices per thread with 16-byte loads, every vertex in
// its own thread group, so the pass has the memory parallelism to stream; a
// thread issues its loads before it reads D (one word, folded by the sweep
// that ran in between), and the pass has no block barrier.
template <bool WRITE_X, int MIN_BLOCKS>
__global__ void __launch_bounds__(kCta, MIN_BLOCKS) k_pr_seg_vertex(const int32_t *rowptr, int32_t n,
                                                           ShareMap sm, float *y,
                                                           float *contrib_next, float *x,
                                                           const double *dprev, double *dslots,
                                                           float base, float damp, double inv_n) {
    const int lane = threadIdx.x & 31;
    const int64_t v0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const bool full = v0 + 4 <= n;
    int32_t r[5] = {0, 0, 0, 0, 0};
    float yv[4] = {0.f, 0.f, 0.f, 0.f};
    if (full) {
        const int4 r4 = *reinterpret_cast<const int4 *>(rowptr + v0);
        const float4 y4 = *reinterpret_cast<const float4 *>(y + v0);
        r[0] = r4.x; r[1] = r4.y; r[2] = r4.z; r[3] = r4.w;
        yv[0] = y4.x; yv[1] = y4.y; yv[2] = y4.z; yv[3] = y4.w;
    } else if (v0 < n) {
        for (int k = 0; k < 4; ++k) {
            if (v0 + k <= n) r[k] = rowptr[v0 + k];
            if (v0 + k < n) yv[k] = y[v0 + k];
        }
    }
    // rowptr[v0 + 4] is the next lane's first offset; the last lane of a warp
    // and the last full quad load it
    const int32_t r_next = __shfl_down_sync(G2_FULL, r[0], 1);
    if (full) r[4] = (lane == 31 || v0 + 4 == n) ? rowptr[v0 + 4] : r_next;
    const float dterm = (float)(*dprev * inv_n);
    float dsum = 0.f;
    if (v0 < n) {
        PrQuad q;
        float xs[4], sh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            q.od[k] = v0 + k < n ? r[k + 1] - r[k] : 0;
            xs[k] = base + damp * (yv[k] + dterm);
            sh[k] = 0.f;
            if (v0 + k >= n) continue;
            if (q.od[k] > 0) sh[k] = xs[k] / (float)q.od[k];
            else dsum += xs[k];
        }
        store_quad_shares(contrib_next, sm, n, v0, q, sh);
        if (full) {
            *reinterpret_cast<float4 *>(y + v0) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            for (int k = 0; k < 4; ++k)
                if (v0 + k < n) y[v0 + k] = 0.f;
        }
        if (WRITE_X) {
            // x is the caller's array: vector stores only when 16-byte aligned
            if (full && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0))
                *reinterpret_cast<float4 *>(x + v0) = make_float4(xs[0], xs[1], xs[2], xs[3]);
            else
                for (int k = 0; k < 4 && v0 + k < n; ++k) x[v0 + k] = xs[k];
        }
    }
    // D partial of the warp (a sum of at most 128 ranks, in fp32) into one of
    // the fp64 slots, no block barrier; the next sweep folds the slots
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(G2_FULL, dsum, o);
    if (lane == 0 && dsum != 0.f) {
        const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        atomicAdd(dslots + (gw % kDSlots) * kDStride, (double)dsum);
    }
}

// ---------------------------------------------------------------- host side
struct PrCfg {
    int blk;        // blocks of this many sources: the source-blocked sweep (0: off)
    int merge;      // 1: merge-path tile kernel, 0: segmented arc sweep
    int ipt;        // merge kernel: 8 or 16 items per thread
    int hot;        // cached shares (0 = none)
    int per_sm;     // merge kernel: resident CTAs per SM (0 = as many as fit)
    int cta;        // segmented sweep: 512 or 1024 threads per CTA
    int vtx_full;   // vertex pass: 8 resident CTAs per SM (32 registers) or 6
};

// Defaults (measured on GB300 with RMAT-22): the source-blocked sweep with
// blocks of 49,152 sources (192 KB of shares per CTA, one CTA per SM) where
// its layout applies (at most 1,024 blocks); else the segmented sweep with
// 1024-thread CTAs and the shares of the 16,384 highest-degree vertices
// cached in shared memory (64 KB per CTA, two CTAs per SM).  The environment
// overrides them for tuning sweeps: G2_PR_KERNEL = blk | seg | merge.
static PrCfg pr_config(const g2_graph *g) {
    PrCfg c{kBlkDefaultS, 0, 8, 16384, 0, 1024, 1};
    if (const char *e = getenv("G2_PR_BLK_S")) c.blk = atoi(e);
    if (const char *e = getenv("G2_PR_KERNEL")) {
        c.merge = strcmp(e, "merge") == 0;
        if (strcmp(e, "blk") != 0) c.blk = 0;
    }
    if (c.blk > 0 && !pr_blk_applies(g->topo, c.blk)) c.blk = 0;
    if (const char *e = getenv("G2_PR_IPT")) c.ipt = atoi(e) == 16 ? 16 : 8;
    if (const char *e = getenv("G2_PR_HOT")) c.hot = std::max(0, atoi(e));
    if (const char *e = getenv("G2_PR_CTAS_PER_SM")) c.per_sm = std::max(0, atoi(e));
    if (const char *e = getenv("G2_PR_SEG_CTA")) c.cta = atoi(e) == 512 ? 512 : 1024;
    if (const char *e = getenv("G2_PR_VTX_BLOCKS")) c.vtx_full = atoi(e) != 6;
    c.hot = std::min<int64_t>(c.hot, g->topo->n);
    c.hot &= ~3;  // keeps the stage buffers 16-byte aligned
    return c;
}

// ------------------------------------------------ hot-vertex selection
// The shared-memory share cache holds the slots 0..hot-1: the `hot` vertices
// of highest out-degree get them (ties to the lower ids), the others follow in
// id order.  The selection runs on the device: a 256-bin histogram of the
// degrees (exact below 16, then 8 bins per power of two) finds the bin that
// holds the hot-th largest degree, a second histogram of up to 4,096 bins
// inside that bin narrows it to one degree (one bin of 2^shift degrees above
// 2^15), and two scans give each vertex its slot.  Which vertices share a
// slot range does not change any sum: the sweep adds each row's arcs in CSC
// order whatever the slot numbers are.
constexpr int kHotBins1 = kDegBuckets;
constexpr int kHotBins2 = 4096;

// first degree of coarse bin b and its width (a power of two)
static inline void hot_bin_range(int b, int64_t *lo, int64_t *width) {
    if (b < 16) {
        *lo = b;
        *width = 1;
        return;
    }
    const int e = 4 + (b - 16) / 8, k = (b - 16) % 8;
    *width = (int64_t)1 << (e - 3);
    *lo = ((int64_t)1 << e) + k * *width;
}

__global__ void __launch_bounds__(kCta) k_hot_hist1(const int32_t *rowptr, int32_t n, int32_t *hist) {
    __shared__ int32_t s[kHotBins1];
    for (int i = threadIdx.x; i < kHotBins1; i += blockDim.x) s[i] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&s[deg_bucket(__ldg(rowptr + v + 1) - __ldg(rowptr + v))], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHotBins1; i += blockDim.x)
        if (s[i]) atomicAdd(hist + i, s[i]);
}

// histogram of (d - lo) >> shift over the degrees d in [lo, lo + width)
__global__ void __launch_bounds__(kCta) k_hot_hist2(const int32_t *rowptr, int32_t n, int64_t lo,
                                                    int64_t width, int shift, int32_t *hist) {
    __shared__ int32_t s[kHotBins2];
    for (int i = threadIdx.x; i < kHotBins2; i += blockDim.x) s[i] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = __ldg(rowptr + v + 1) - __ldg(rowptr + v);
        if (d >= lo && d < lo + width) atomicAdd(&s[(int)((d - lo) >> shift)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHotBins2; i += blockDim.x)
        if (s[i]) atomicAdd(hist + i, s[i]);
}

// tie[v] = 1 iff tlo <= deg(v) < thi
__global__ void k_hot_ties(const int32_t *rowptr, int32_t n, int64_t tlo, int64_t thi,
                           int32_t *tie) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rowptr[v + 1] - rowptr[v];
        tie[v] = d >= tlo && d < thi;
    }
}

// hot[v] = deg(v) >= thi, or a tie among the first `need` ties by id
__global__ void k_hot_flags(const int32_t *rowptr, int32_t n, int64_t tlo, int64_t thi,
                            const int32_t *tie_rank, int32_t need, int32_t *hot) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rowptr[v + 1] - rowptr[v];
        hot[v] = d >= thi || (d >= tlo && tie_rank[v] < need);
    }
}

// slot of v: its rank among the hot vertices, or hot + v
__global__ void k_hot_perm(const int32_t *hotf, int32_t n, int32_t hot, int32_t *perm) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = perm[v];  // hot vertices before v
        perm[v] = hotf[v] ? r : hot + (int32_t)v;
    }
}

// The `hot` highest-degree vertices (0 < hot <= n): the share slot of every
// vertex, perm (n entries plus one spare for the scan total), and the least
// degree among the hot vertices.
static g2_status select_hot(g2_graph *g, int32_t hot, int32_t *perm, int32_t *min_deg,
                            cudaStream_t st) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *hist, *a, *b;
    G2_TRY(ws(g, B_TWC_M, kHotBins1 + kHotBins2, &hist));
    G2_TRY(ws(g, B_I0, (size_t)n + 1, &a));
    G2_TRY(ws(g, B_I1, (size_t)n + 1, &b));
    G2_CK(cudaMemsetAsync(hist, 0, (kHotBins1 + kHotBins2) * sizeof(int32_t), st));
    const int grid = grid_for(g, n, kCta);
    k_hot_hist1<<<grid, kCta, 0, st>>>(t->rowptr, n, hist);
    std::vector<int32_t> h1(kHotBins1);
    G2_CK(cudaMemcpyAsync(h1.data(), hist, kHotBins1 * 4, cudaMemcpyDeviceToHost, st));
    G2_CK(cudaStreamSynchronize(st));
    // coarse bin holding the hot-th largest degree; c_above = vertices above it
    int bsel = 0;
    int64_t c_above = 0;
    for (int k = kHotBins1 - 1; k >= 0; --k) {
        if (c_above + h1[k] >= hot) {
            bsel = k;
            break;
        }
        c_above += h1[k];
    }
    int64_t lo, width;
    hot_bin_range(bsel, &lo, &width);
    int shift = 0;
    while ((width >> shift) > kHotBins2) ++shift;
    const int nb2 = (int)(width >> shift);
    k_hot_hist2<<<grid, kCta, 0, st>>>(t->rowptr, n, lo, width, shift, hist + kHotBins1);
    std::vector<int32_t> h2(nb2);
    G2_CK(cudaMemcpyAsync(h2.data(), hist + kHotBins1, (size_t)nb2 * 4, cudaMemcpyDeviceToHost, st));
    G2_CK(cudaStreamSynchronize(st));
    int jsel = 0;
    for (int k = nb2 - 1; k >= 0; --k) {
        if (c_above + h2[k] >= hot) {
            jsel = k;
            break;
        }
        c_above += h2[k];
    }
    // degrees >= thi are hot; of those in [tlo, thi), the first `need` by id
    const int64_t tlo = lo + ((int64_t)jsel << shift), thi = lo + ((int64_t)(jsel + 1) << shift);
    const int32_t need = (int32_t)(hot - c_above);
    k_hot_ties<<<grid, kCta, 0, st>>>(t->rowptr, n, tlo, thi, a);
    G2_TRY(exclusive_scan_i32(g, a, b, n, st));
    k_hot_flags<<<grid, kCta, 0, st>>>(t->rowptr, n, tlo, thi, b, need, a);
    G2_TRY(exclusive_scan_i32(g, a, perm, n, st));
    k_hot_perm<<<grid, kCta, 0, st>>>(a, n, hot, perm);
    *min_deg = (int32_t)tlo;
    stats().launches += 6;
    G2_CK(cudaGetLastError());
    return G2_OK;
}

static g2_status ensure_pr_hot_layout(g2_graph *g, int hot, cudaStream_t st, ShareMap *sm,
                                      const int32_t **ccol) {
    Topology *t = g->topo;
    std::lock_guard<std::recursive_mutex> lk(t->pr_mu);
    if (t->pr_hot != hot || !t->pr_slot_of) {
        const int32_t n = t->n, m = t->m;
        dfree(t->pr_slot_of, st);
        dfree(t->pr_ccol, st);
        t->pr_slot_of = t->pr_ccol = nullptr;
        t->pr_hot = -1;
        G2_CK(dmalloc(&t->pr_slot_of, ((size_t)std::max(n, 1) + 1) * 4, st));
        G2_CK(dmalloc(&t->pr_ccol, ((size_t)std::max(m, 1) + kPad) * 4, st));
        G2_TRY(select_hot(g, hot, t->pr_slot_of, &t->pr_hot_min_deg, st));
        // only the padding past the last arc needs zeroing; the arcs are all written
        G2_CK(cudaMemsetAsync(t->pr_ccol + m, 0, ((size_t)std::max(m, 1) - m + kPad) * 4, st));
        if (m > 0)
            k_remap_cols<<<grid_for(g, m, kCta), kCta, 0, st>>>(t->ccol, t->pr_slot_of, m,
                                                                t->pr_ccol);
        G2_CK(cudaGetLastError());
        G2_CK(cudaStreamSynchronize(st));
        t->pr_hot = hot;
    }
    *sm = ShareMap{hot, t->pr_hot_min_deg, t->pr_slot_of};
    *ccol = t->pr_ccol;
    return G2_OK;
}

static g2_status ensure_seg_layout(g2_graph *g, cudaStream_t st) {
    Topology *t = g->topo;
    std::lock_guard<std::recursive_mutex> lk(t->pr_mu);
    if (t->seg_head) return G2_OK;
    const int32_t n = t->n, m = t->m;
    const size_t words = ((size_t)m + 31) / 32 + 8;
    const int64_t nchunks = ((int64_t)m + kSegArcs - 1) / kSegArcs;
    int32_t *nz, *pos, *ccount;
    G2_TRY(ws(g, B_I0, (size_t)n + 1, &nz));
    G2_TRY(ws(g, B_I1, (size_t)n + 1, &pos));
    G2_TRY(ws(g, B_TWC_S, (size_t)nchunks + 1, &ccount));
    G2_CK(dmalloc(&t->seg_head, words * 4, st));
    G2_CK(cudaMemsetAsync(t->seg_head, 0, words * 4, st));
    k_seg_heads<<<grid_for(g, n, kCta), kCta, 0, st>>>(t->crowptr, n, t->seg_head, nz);
    G2_TRY(exclusive_scan_i32(g, nz, pos, n, st));
    G2_CK(cudaMemcpyAsync(g->h_ctr + 60, pos + n, 4, cudaMemcpyDeviceToHost, st));
    G2_CK(cudaStreamSynchronize(st));
    const int32_t nnz = g->h_ctr[60];
    G2_CK(dmalloc(&t->seg_nzrow, ((size_t)nnz + 1) * 4, st));
    k_seg_nzrow<<<grid_for(g, n, kCta), kCta, 0, st>>>(nz, pos, n, t->seg_nzrow);
    G2_CK(dmalloc(&t->seg_chunk_rank, ((size_t)nchunks + 1) * 4, st));
    if (nchunks > 0) {
        k_seg_chunk_heads<<<grid_for(g, nchunks, kCta), kCta, 0, st>>>(t->seg_head, nchunks, ccount);
        G2_TRY(exclusive_scan_i32(g, ccount, t->seg_chunk_rank, (int32_t)nchunks, st));
    }
    G2_CK(cudaGetLastError());
    G2_CK(cudaStreamSynchronize(st));
    t->seg_nnzrow = nnz;
    return G2_OK;
}

template <int CTA, bool HOT>
static g2_status launch_pr_seg(g2_graph *g, const int32_t *pcol, int32_t hot, const float *contrib,
                               float *y, double *dslots, double *dfin, cudaStream_t st) {
    Topology *t = g->topo;
    // launched even without arcs: its first warp folds the dangling mass
    const int64_t nchunks = ((int64_t)t->m + kSegArcs - 1) / kSegArcs;
    const size_t smem = HOT ? (size_t)hot * 4 : 0;
    auto kern = k_pr_seg<CTA, HOT>;
    if (smem > 48 * 1024)
        G2_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    G2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, CTA, smem));
    if (b < 1) return fail(G2_EUNSUPPORTED, "PageRank sweep kernel does not fit on an SM");
    int64_t want = (nchunks * 32 + CTA - 1) / CTA;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)b * t->sm_count));
    // slots [hot, warm) are loaded with L1 evict-last priority (off by
    // default: warm = hot; G2_PR_WARM sets it for sweeps)
    int32_t warm = hot;
    if (const char *e = getenv("G2_PR_WARM")) warm = std::max<int32_t>(hot, atoi(e));
    KTime kt;
    ktime_begin(kt, "pr_round", st);
    kern<<<grid, CTA, smem, st>>>(pcol, t->seg_head, t->seg_chunk_rank, t->seg_nzrow, t->m, nchunks,
                                  contrib, hot, warm, y, dslots, dfin);
    ktime_end(kt, st);
    return G2_OK;
}

template <int IPT, bool HOT>
static g2_status launch_pr_merge(g2_graph *g, const PrArgs &a, int per_sm, cudaStream_t st,
                                 int32_t *d_err) {
    const size_t smem = pr_smem_bytes(IPT, a.hot);
    auto kern = k_pr_merge<IPT, HOT>;
    G2_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int b = 0;
    G2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kCta, smem));
    if (b < 1) return fail(G2_EUNSUPPORTED, "PageRank tile kernel does not fit on an SM");
    if (per_sm > 0 && per_sm < b) b = per_sm;
    int grid = (int)std::min<int64_t>(a.ntiles, (int64_t)b * g->topo->sm_count);
    KTime kt;
    ktime_begin(kt, "pr_round", st);
    kern<<<grid, kCta, smem, st>>>(a, 2000000000ULL, d_err);
    ktime_end(kt, st);
    return G2_OK;
}

g2_status pagerank_run(g2_graph *g, float damping, int32_t iters, float *rank, const g2_hybrid &h,
                       bool tuned_default, cudaStream_t st, int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    if (n == 0) return G2_OK;
    const double inv_n = 1.0 / (double)n;
    float *cbuf[2], *acc;
    G2_TRY(ws(g, B_F2, (size_t)n + 1, &acc));
    // D: dd[0], dd[1] for the merge and generic paths, dd[2], dd[3] for the
    // segmented sweep's rounds; dd[8..8+R) the slots the x0 and vertex
    // passes accumulate into (zero to start; every fold zeroes them again)
    constexpr size_t R = (size_t)kDSlots * kDStride;
    double *dd;
    G2_TRY(ws(g, B_D1, 8 + R, &dd));
    G2_CK(cudaMemsetAsync(dd, 0, (8 + R) * sizeof(double), st));
    const g2_schedule &s = h.s1;  // one schedule for every round (the frontier is always all vertices)
    const float base = (float)((1.0 - damping) * inv_n);
    const bool merge = tuned_default || (s.direction == G2_PULL && s.load_balance == G2_LB_EDGE_ONLY);
    if (!merge) {
        G2_TRY(check_schedule(g, s, K_PR, true));
        if (s.kernel_fusion) return fail(G2_EUNSUPPORTED, "PageRank has no fused variant");
    }
    PrCfg cfg = pr_config(g);
    if (merge && cfg.blk > 0) return pagerank_blk_run(g, damping, iters, rank, cfg.blk, st);
    ShareMap sm{0, 0, nullptr};
    const int32_t *ccol = t->ccol;
    if (merge && cfg.hot > 0) G2_TRY(ensure_pr_hot_layout(g, cfg.hot, st, &sm, &ccol));
    // shares: slots 0..H-1 for the cached vertices, H + v for vertex v
    G2_TRY(ws(g, B_F0, (size_t)n + sm.hot, &cbuf[0]));
    G2_TRY(ws(g, B_F1, (size_t)n + sm.hot, &cbuf[1]));
    // vertex passes end with one fp64 atomic per CTA on a single address, and
    // same-address atomics serialise: few CTAs, each striding over many vertices
    const int vgrid = (int)std::min<int64_t>((n + kCta - 1) / kCta, (int64_t)t->sm_count * 2);
    // the x0 pass, one quad per thread; D0 goes into the slots, which the
    // first sweep folds into dd[2] (segmented sweep) or k_pr_fold into dd[0]
    const bool seg = merge && !cfg.merge;
    const int igrid = (int)((((int64_t)n + 3) / 4 + kCta - 1) / kCta);
    k_pr_init<<<std::max(igrid, 1), kCta, 0, st>>>(t->rowptr, n, sm, cbuf[0], dd + 8, rank, inv_n);
    stats().launches += 1;
    if (!seg) {
        k_pr_fold<<<1, 32, 0, st>>>(dd + 8, dd);
        stats().launches += 1;
    }
    if (iters <= 0) return G2_OK;
    if (merge && !cfg.merge) {
        G2_TRY(ensure_seg_layout(g, st));
        const int32_t hot = sm.hot;
        G2_CK(cudaMemsetAsync(acc, 0, (size_t)(n + 1) * 4, st));
        const int vblocks = (int)((((int64_t)n + 3) / 4 + kCta - 1) / kCta);
        for (int32_t it = 0; it < iters; ++it) {
            const float *c0 = cbuf[it & 1];
            float *c1 = cbuf[(it + 1) & 1];
            // D_{t-1}: the sweep folds the slots of the previous pass (the x0
            // pass for round 0) into dd[2 + (t & 1)] for this round's vertex pass
            double *dprev = dd + 2 + (it & 1);
            double *fold = dd + 8;
            if (cfg.cta == 512) {
                if (hot) G2_TRY((launch_pr_seg<512, true>(g, ccol, hot, c0, acc, fold, dprev, st)));
                else G2_TRY((launch_pr_seg<512, false>(g, ccol, hot, c0, acc, fold, dprev, st)));
            } else {
                if (hot) G2_TRY((launch_pr_seg<1024, true>(g, ccol, hot, c0, acc, fold, dprev, st)));
                else G2_TRY((launch_pr_seg<1024, false>(g, ccol, hot, c0, acc, fold, dprev, st)));
            }
            KTime kv;
            ktime_begin(kv, "pr_vertex", st);
            // x itself is written by the last round only
            auto vk = it == iters - 1 ? (cfg.vtx_full ? k_pr_seg_vertex<true, 8>
                                                      : k_pr_seg_vertex<true, 6>)
                                      : (cfg.vtx_full ? k_pr_seg_vertex<false, 8>
                                                      : k_pr_seg_vertex<false, 6>);
            vk<<<vblocks, kCta, 0, st>>>(t->rowptr, n, sm, acc, c1, rank, dprev, dd + 8, base,
                                         damping, inv_n);
            ktime_end(kv, st);
            stats().launches += 2;
            stats().iterations++;
            stats().pull_rounds++;
        }
        G2_CK(cudaGetLastError());
        return G2_OK;
    }
    if (merge) {
        const int32_t tile = kCta * cfg.ipt;
        const int64_t total = (int64_t)n + t->m;
        const int32_t ntiles = (int32_t)((total + tile - 1) / tile);
        int32_t *tile_r, *split, *ctrs = d_err - 62;
        G2_TRY(ws(g, B_SCAN, (size_t)ntiles + 2, &tile_r));
        G2_TRY(ws(g, B_TWC_M, (size_t)ntiles + 2, &split));
        G2_CK(cudaMemsetAsync(acc, 0, (size_t)(n + 1) * 4, st));
        G2_CK(cudaMemsetAsync(ctrs + 10, 0, 4, st));
        k_pr_tiles<<<grid_for(g, ntiles + 1, kCta), kCta, 0, st>>>(t->crowptr, n, t->m, tile, ntiles,
                                                                   tile_r);
        k_pr_split_rows<<<grid_for(g, ntiles, kCta), kCta, 0, st>>>(t->crowptr, n, tile, ntiles,
                                                                    tile_r, split, ctrs + 10);
        stats().launches += 2;
        PrArgs a;
        a.n = n;
        a.m = t->m;
        a.tile = tile;
        a.crowptr = t->crowptr;
        a.ccol = ccol;
        a.rowptr = t->symmetric ? nullptr : t->rowptr;
        a.slot_of = sm.slot_of;
        a.hot_min_deg = sm.min_deg;
        a.tile_r = tile_r;
        a.ntiles = ntiles;
        a.hot = sm.hot;
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
            if (cfg.ipt == 16) {
                if (a.hot) G2_TRY((launch_pr_merge<16, true>(g, a, cfg.per_sm, st, d_err)));
                else G2_TRY((launch_pr_merge<16, false>(g, a, cfg.per_sm, st, d_err)));
            } else {
                if (a.hot) G2_TRY((launch_pr_merge<8, true>(g, a, cfg.per_sm, st, d_err)));
                else G2_TRY((launch_pr_merge<8, false>(g, a, cfg.per_sm, st, d_err)));
            }
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
        k_pr_vertex<<<vgrid, kCta, 0, st>>>(t->rowptr, n, acc, cbuf[(it + 1) & 1],
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

namespace g2 {

// The layouts of the tuned sweep for handle g (its workspace, stream st).
g2_status pr_build_layouts(g2_graph *g, cudaStream_t st) {
    g->st = st;
    const PrCfg cfg = pr_config(g);
    if (cfg.blk > 0) return ensure_blk_layout(g, cfg.blk, st);
    if (cfg.hot > 0) {
        ShareMap sm{0, 0, nullptr};
        const int32_t *ccol = nullptr;
        G2_TRY(ensure_pr_hot_layout(g, cfg.hot, st, &sm, &ccol));
    }
    if (!cfg.merge) G2_TRY(ensure_seg_layout(g, st));
    return G2_OK;
}

}  // namespace g2

extern "C" g2_status g2_pagerank(g2_graph *g, float damping, int32_t iters, float *rank,
                                 const g2_hybrid *sched, void *stream) {
    if (!g || !rank) return fail(G2_EINVAL, "null graph or rank");
    if (iters < 0 || !(damping >= 0.f && damping <= 1.f))
        return fail(G2_EINVAL, "iters must be >= 0 and damping in [0, 1]");
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : default_hybrid();
    G2_TRY(pr_prepare_wait(g->topo));  // layouts a G2_PREPARE_PAGERANK load started
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    G2_TRY(pagerank_run(g, damping, iters, rank, h, sched == nullptr, st, d_err));
    return end_call(g, st, d_err);
}
