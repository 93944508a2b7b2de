// g2_bc.cu — betweenness centrality (Sec. VII; Brandes, "A faster algorithm
// for betweenness centrality", 2001) summed over a list of sources.
//
// Per source: a level-synchronous BFS whose levels are appended to one list,
// path counts sigma for each new level (pull over in-neighbours one level up),
// then dependencies delta level by level from the deepest (pull over
// out-neighbours one level down), bc[v] += delta[v] for v != source.
//
// Path counts grow like binomials on grids (C(2k, k) after 2k levels) and two
// vertices of one level can differ by more than the fp64 range, so sigma is an
// extended-range number: a 64-bit integer mantissa and an int32 exponent per
// vertex.  The dependency sum delta_v = sum_w sigma_v / sigma_w (1 + delta_w)
// is formed as m_v * sum_w c_w 2^(e_v - e_w) with c_w = (1 + delta_w) / m_w
// kept per vertex (one fp64 division per vertex, when its sigma is known),
// so an arc costs a power-of-two scaling and an add (fp64 is slow on this
// GPU).
//
// Schedules: each level's discovery is one edgeset.apply round (PUSH or PULL
// per the hybrid schedule); with kernel fusion the whole source runs in one
// persistent cooperative kernel with one grid barrier per level and pass.
// The sigma and delta pulls give a warp to every vertex and a whole CTA to
// the vertices with at least kBigDeg arcs, or a thread to every vertex on a
// symmetric bounded-degree graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "g2_cluster.cuh"
#include "g2_host.h"
#include "g2_lb.cuh"

namespace g2 {

constexpr int32_t kBigDeg = 4096;    // a CTA per vertex from this many arcs
constexpr int32_t kThreadDeg = 32;   // a thread per vertex below this many arcs

// Extended-range path count: an integer mantissa m, 0 or in [2^62, 2^63),
// and an exponent e; the value is m * 2^(e - 63).  Sums take integer shifts
// and adds only (no fp64 on the per-arc path; fp64 is slow on this GPU), with
// 63 mantissa bits.
struct BigF {
    unsigned long long m;
    int e;
};

// m * 2^-63 in [0.5, 1) as fp64 (once per vertex)
__device__ __forceinline__ double bf_mant(unsigned long long m) {
    return (double)m * 0x1p-63;
}

// x * 2^k for k <= 1023, by a multiply with the power of two built from its
// exponent bits; 0 below 2^-1022 (a term that small is below the rounding of
// every sum it joins).
__device__ __forceinline__ double scale2(double x, int k) {
    if (k < -1022) return 0.0;
    return x * __hiloint2double((k + 1023) << 20, 0);
}

// a + b: the smaller mantissa shifted to the larger one's exponent (the
// bits shifted out are dropped: below 2^-62 of the sum), the sum brought back
// under 2^63.
__device__ __forceinline__ BigF bf_add(BigF a, BigF b) {
    if (a.m == 0) return b;
    if (b.m == 0) return a;
    if (a.e < b.e) {
        BigF t = a;
        a = b;
        b = t;
    }
    const int d = a.e - b.e;
    unsigned long long sum = d > 63 ? a.m : a.m + (b.m >> d);
    int e = a.e;
    if (sum >> 63) {
        sum >>= 1;
        ++e;
    }
    return BigF{sum, e};
}

__device__ __forceinline__ BigF bf_shfl_xor(BigF a, int d) {
    return BigF{__shfl_xor_sync(G2_FULL, a.m, d), __shfl_xor_sync(G2_FULL, a.e, d)};
}

struct BcState {
    DevGraph g;
    int32_t *depth;
    unsigned long long *sm;  // sigma mantissas (BigF)
    int32_t *se; // sigma exponents
    // (1 + delta_v) / m_v: 1 / m_v once sigma_v is known, then (1 + delta_v) /
    // m_v once delta_v is, so that delta_u = m_u * sum over successors w of
    // coef_w * 2^(e_u - e_w): per arc a scaling and an add, no division
    double *coef;
    double *bc;
    int32_t *lvl;  // all levels, in order
    int32_t src;
    // level-pass granularity: one thread per vertex on a symmetric
    // bounded-degree graph (every list short), else one warp per vertex and,
    // when some vertex may have kBigDeg or more arcs (`big`), one CTA for those
    int32_t per_thread;
    int32_t big;
};

// sigma of vertex w at level d+1: sum over in-neighbours u at level d
__device__ __forceinline__ BigF bc_sigma_part(const BcState &s, int32_t w, int32_t d, int32_t b,
                                              int32_t e, int32_t step, int32_t off) {
    BigF acc{0, 0};
    for (int32_t k = b + off; k < e; k += step) {
        int32_t u = s.g.ccol[k];
        if (s.depth[u] == d) acc = bf_add(acc, BigF{s.sm[u], s.se[u]});
    }
    return acc;
}

// delta of vertex v at level d, over its out-neighbours w at level d+1:
// the sum of coef_w * 2^(e_v - e_w) (bc_finish_delta multiplies by m_v)
__device__ __forceinline__ double bc_delta_part(const BcState &s, int32_t v, int32_t d, int32_t b,
                                                int32_t e, int32_t step, int32_t off) {
    const int ev = s.se[v];
    double acc = 0.0;
    for (int32_t k = b + off; k < e; k += step) {
        int32_t w = s.g.col[k];
        if (s.depth[w] == d + 1) acc += scale2(s.coef[w], ev - s.se[w]);
    }
    return acc;
}

// delta_v from the sum of its successors' terms: added to bc (but for the
// source) and kept as the coefficient the level above uses
__device__ __forceinline__ void bc_finish_delta(const BcState &s, int32_t v, double sum) {
    const double dl = bf_mant(s.sm[v]) * sum;
    if (v != s.src) s.bc[v] += dl;
    s.coef[v] *= 1.0 + dl;
}

// sigma_v found: stored, and 1 / m_v as the first coefficient
__device__ __forceinline__ void bc_finish_sigma(const BcState &s, int32_t v, BigF a) {
    s.sm[v] = a.m;
    s.se[v] = a.e;
    s.coef[v] = 1.0 / bf_mant(a.m);
}

// The same sums for one thread over a whole (short) list, four arcs' loads in
// flight at a time and the terms added in arc order, so the result is the
// one bc_sigma_part / bc_delta_part give with step 1.
__device__ __forceinline__ BigF bc_sigma_thread(const BcState &s, int32_t w, int32_t d) {
    const int32_t b = s.g.crowptr[w], e = s.g.crowptr[w + 1];
    BigF acc{0, 0};
    for (int32_t k = b; k < e; k += 4) {
        int32_t u[4], du[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = k + j < e ? s.g.ccol[k + j] : -1;
#pragma unroll
        for (int j = 0; j < 4; ++j) du[j] = u[j] >= 0 ? s.depth[u[j]] : -2;
        BigF t[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            t[j] = du[j] == d ? BigF{s.sm[u[j]], s.se[u[j]]} : BigF{0, 0};
#pragma unroll
        for (int j = 0; j < 4; ++j) acc = bf_add(acc, t[j]);
    }
    return acc;
}

__device__ __forceinline__ double bc_delta_thread(const BcState &s, int32_t v, int32_t d) {
    const int32_t b = s.g.rowptr[v], e = s.g.rowptr[v + 1];
    const int ev = s.se[v];
    double acc = 0.0;
    for (int32_t k = b; k < e; k += 4) {
        int32_t w[4], dw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = k + j < e ? s.g.col[k + j] : -1;
#pragma unroll
        for (int j = 0; j < 4; ++j) dw[j] = w[j] >= 0 ? s.depth[w[j]] : -2;
        double cw[4];
        int ew[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool on = dw[j] == d + 1;
            cw[j] = on ? s.coef[w[j]] : 0.0;
            ew[j] = on ? s.se[w[j]] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (dw[j] == d + 1) acc += scale2(cw[j], ev - ew[j]);
    }
    return acc;
}

// Level pass over list[0, cnt): small vertices one per warp, big ones one per
// CTA.  `bid`/`nb` as in the load-balancing library (plain or fused).
template <bool SIGMA>
__device__ void bc_level_pass(const BcState &s, const int32_t *list, int32_t cnt, int32_t d,
                              int bid, int nb) {
    if (s.per_thread) {  // uniform over the grid
        const int64_t nt = (int64_t)nb * blockDim.x;
        for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < cnt; i += nt) {
            const int32_t v = list[i];
            if (SIGMA) bc_finish_sigma(s, v, bc_sigma_thread(s, v, d));
            else bc_finish_delta(s, v, bc_delta_thread(s, v, d));
        }
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gw = bid * kWarps + wid, nw = nb * kWarps;
    // threads: vertices with fewer than kThreadDeg arcs (on a power-law
    // graph most of a level, whose few arcs would leave a warp nearly idle)
    {
        const int64_t nt = (int64_t)nb * blockDim.x;
        for (int64_t i = (int64_t)bid * blockDim.x + threadIdx.x; i < cnt; i += nt) {
            const int32_t v = list[i];
            const int32_t deg = SIGMA ? s.g.crowptr[v + 1] - s.g.crowptr[v]
                                      : s.g.rowptr[v + 1] - s.g.rowptr[v];
            if (deg >= kThreadDeg) continue;
            if (SIGMA) bc_finish_sigma(s, v, bc_sigma_thread(s, v, d));
            else bc_finish_delta(s, v, bc_delta_thread(s, v, d));
        }
    }
    // warps: vertices with kThreadDeg .. kBigDeg - 1 arcs
    for (int32_t i = gw; i < cnt; i += nw) {
        int32_t v = list[i];
        int32_t b = SIGMA ? s.g.crowptr[v] : s.g.rowptr[v];
        int32_t e = SIGMA ? s.g.crowptr[v + 1] : s.g.rowptr[v + 1];
        if (e - b < kThreadDeg || e - b >= kBigDeg) continue;
        if (SIGMA) {
            BigF a = bc_sigma_part(s, v, d, b, e, 32, lane);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a = bf_add(a, bf_shfl_xor(a, o));
            if (lane == 0) bc_finish_sigma(s, v, a);
        } else {
            double a = bc_delta_part(s, v, d, b, e, 32, lane);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(G2_FULL, a, o);
            if (lane == 0) bc_finish_delta(s, v, a);
        }
    }
    // CTAs: vertices with at least kBigDeg arcs
    __shared__ double s_m[kWarps];
    __shared__ unsigned long long s_mu[kWarps];
    __shared__ int s_e[kWarps];
    if (!s.big) return;  // uniform: no vertex has that many arcs
    for (int32_t i = bid; i < cnt; i += nb) {
        int32_t v = list[i];
        int32_t b = SIGMA ? s.g.crowptr[v] : s.g.rowptr[v];
        int32_t e = SIGMA ? s.g.crowptr[v + 1] : s.g.rowptr[v + 1];
        if (e - b < kBigDeg) continue;
        if (SIGMA) {
            BigF a = bc_sigma_part(s, v, d, b, e, kCta, threadIdx.x);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a = bf_add(a, bf_shfl_xor(a, o));
            if (lane == 0) {
                s_mu[wid] = a.m;
                s_e[wid] = a.e;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                BigF t{0, 0};
                for (int k = 0; k < kWarps; ++k) t = bf_add(t, BigF{s_mu[k], s_e[k]});
                bc_finish_sigma(s, v, t);
            }
        } else {
            double a = bc_delta_part(s, v, d, b, e, kCta, threadIdx.x);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(G2_FULL, a, o);
            if (lane == 0) s_m[wid] = a;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int k = 0; k < kWarps; ++k) t += s_m[k];
                bc_finish_delta(s, v, t);
            }
        }
        __syncthreads();
    }
}

template <bool SIGMA>
__global__ void __launch_bounds__(kCta) k_bc_level(BcState s, const int32_t *list, int32_t cnt,
                                                   int32_t d) {
    bc_level_pass<SIGMA>(s, list, cnt, d, blockIdx.x, gridDim.x);
}

__global__ void k_bc_init(BcState s, int32_t n, int32_t *cnt3) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        bool is_src = v == s.src;
        s.depth[v] = is_src ? 0 : -1;
        s.sm[v] = is_src ? (1ull << 62) : 0ull;  // sigma(src) = 1 = 2^62 * 2^(1 - 63)
        s.se[v] = is_src ? 1 : 0;
        s.coef[v] = is_src ? 2.0 : 0.0;  // 1 / m_src
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.lvl[0] = s.src;
        if (cnt3) {
            cnt3[0] = cnt3[1] = cnt3[2] = 0;
        }
    }
}

// ------------------------------------------------------------ fused source
struct BcFusedArgs {
    BcState s;
    int32_t *off;    // level offsets into lvl (off[d] = start of level d)
    int32_t *cnt3;   // rotating append counters (zero at launch)
    GridBarrier bar;
    int32_t *err;
    uint64_t limit_ns;
    int32_t fwd;     // 1: forward phases from level d0, whose list is lvl[b0, e0)
    int32_t d0, b0, e0;
    int32_t lo;      // > 0: after a phase, stop before a level of fewer vertices
    int32_t bwd;     // 1: backward pass after the forward pass (levels D-2 .. 0)
    int32_t Lhi, Llo;  // without the forward pass: backward over levels Lhi down to Llo
    int32_t *result; // out: [0] 1 if stopped for the cluster loop, [1] levels found (or
                     // the next level), [2] its start in lvl, [3] its size
};

template <int LB>
__global__ void __launch_bounds__(kCta) k_bc_fused(BcFusedArgs a) {
    const BcState &s = a.s;
    int32_t Lhi = a.Lhi;
    const int32_t Llo = a.Llo;
    if (a.fwd) {
        OpBFS op{s.depth, nullptr};
        OutCtx out;
        memset(&out, 0, sizeof(out));
        out.mode = OUT_SPARSE;
        out.dedup = DD_NONE;
        out.err = a.err;
        int32_t b = a.b0, e = a.e0, d = a.d0;
        // one barrier per level: the discovery of level d+1 from level d and
        // the sigma of level d (pulled from level d-1) share a phase.  The
        // discovery reads no sigma, and the sigma pass only looks for depth
        // d-1, which no vertex discovered in the same phase (-1 -> d+1) has.
        for (;; ++d) {
            FrontierIn fin{s.lvl + b, e - b, nullptr};
            out.q = s.lvl + e;
            out.cnt = a.cnt3 + d % 3;
            out.cap = s.g.n - e;
            if (blockIdx.x == 0 && threadIdx.x == 0) a.cnt3[(d + 1) % 3] = 0;
            if (LB == G2_LB_WM) lb_warp(s.g, fin, e - b, op, out, blockIdx.x, gridDim.x, nullptr);
            else if (LB == G2_LB_CM) lb_cta(s.g, fin, e - b, op, out, blockIdx.x, gridDim.x, nullptr);
            else if (LB == G2_LB_ETWC) lb_etwc(s.g, fin, e - b, op, out, blockIdx.x, gridDim.x, nullptr);
            else lb_vertex(s.g, fin, e - b, op, out, blockIdx.x, gridDim.x, nullptr);
            if (d > 0) bc_level_pass<true>(s, s.lvl + b, e - b, d - 1, blockIdx.x, gridDim.x);
            if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
            const int32_t nn = ld_relaxed_i32(a.cnt3 + d % 3);
            if (nn == 0) break;
            if (blockIdx.x == 0 && threadIdx.x == 0) a.off[d + 2] = e + nn;
            b = e;
            e += nn;
            if (nn < a.lo) {  // the same length in every CTA
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    a.result[0] = 1;
                    a.result[1] = d + 1;
                    a.result[2] = b;
                    a.result[3] = nn;
                }
                return;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.result[0] = 0;
            a.result[1] = d + 1;
        }
        if (!a.bwd) return;
        Lhi = d - 1;  // levels 0..d: from the deepest but one
    }
    for (int32_t L = Lhi; L >= Llo; --L) {
        const int32_t lb0 = ld_relaxed_i32(a.off + L), lb1 = ld_relaxed_i32(a.off + L + 1);
        bc_level_pass<false>(s, s.lvl + lb0, lb1 - lb0, L, blockIdx.x, gridDim.x);
        if (!grid_sync(a.bar, a.err, a.limit_ns)) return;
    }
}

// --------------------------------------------------- fused source in one cluster
// On a symmetric bounded-degree graph (the thread-per-vertex passes) the
// small levels of a fused WM source run inside one thread-block cluster, as
// the fused BFS does: the CTAs keep the vertices they discover in shared
// memory, a level ends at the cluster barrier, and every CTA takes an equal
// slice of the concatenated level, read through distributed shared memory.
// In the phase of level d a CTA copies its part of level d to the global
// level list (for the backward pass), discovers level d+1 from its slice
// (the slice's arcs spread over the warp's lanes, four deep) and computes the
// slice's sigma from level d-1.  A level of more than `hi` vertices goes to
// the grid-wide kernel (k_bc_fused), which hands the forward pass back below
// `lo`; the backward pass runs level ranges on one or the other by level
// size.  A level that outgrows a CTA's buffer (appends past the capacity are
// counted, not stored) ends the launch; its vertices all carry their depth,
// so the host rebuilds the level's list from the depths.
constexpr int kBcQcap = 28672;  // level entries per CTA and buffer (2 buffers: 224 KiB)
constexpr size_t kBcSmem = 2 * (size_t)kBcQcap * 4;

struct ClusterBcArgs {
    BcState s;
    int32_t *off;     // level offsets into s.lvl (off[d] = start of level d)
    int32_t fwd;      // 1: forward phases from level d0 (list lvl[start0, start0 + n0))
    int32_t d0, start0, n0;
    int32_t hi;       // stop before a level with more vertices
    int32_t Lhi, Llo; // without the forward pass: backward over levels Lhi down to Llo
    int32_t *result;  // out: [0] CL_DONE / CL_TO_GRID / CL_OVERFLOW, [1] levels found (or
                      // the level handed over), [2] its start in lvl, [3] its size
};

template <int CL>
__global__ void __launch_bounds__(kClCta, 1) k_bc_cluster(ClusterBcArgs a) {
    const BcState &s = a.s;
    extern __shared__ int32_t s_q[];  // [2][kBcQcap]
    __shared__ int32_t s_cnt[2];
    __shared__ int32_t s_off[CL + 1];
    __shared__ int32_t s_over;
    const uint32_t rank = cl_rank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t *__restrict__ rowptr = s.g.rowptr;
    const int32_t *__restrict__ col = s.g.col;
    if (!a.fwd) {
        for (int32_t L = a.Lhi; L >= a.Llo; --L) {
            const int32_t b0 = a.off[L], cnt = a.off[L + 1] - b0;
            const int32_t lo = (int32_t)((int64_t)cnt * rank / CL);
            const int32_t hi = (int32_t)((int64_t)cnt * (rank + 1) / CL);
            for (int32_t i = lo + threadIdx.x; i < hi; i += kClCta) {
                const int32_t v = s.lvl[b0 + i];
                bc_finish_delta(s, v, bc_delta_thread(s, v, L));
            }
            cl_barrier();  // level L's dependencies visible to level L-1
        }
        return;
    }
    if (threadIdx.x == 0) {
        s_cnt[0] = 0;
        s_cnt[1] = 0;
    }
    int32_t start = a.start0, total = a.n0;  // level d: lvl[start, start + total)
    int reason = CL_DONE;
    cl_barrier();
    int d = a.d0;
    for (;; ++d) {
        const int cb = d & 1, nb = cb ^ 1;
        const bool first = d == a.d0;
        if (!first) {
            if (warp == 0) {
                int32_t c = lane < CL ? cl_read(&s_cnt[cb], lane) : 0;
                const bool ov = __any_sync(G2_FULL, c > kBcQcap);
#pragma unroll
                for (int o = 1; o < CL; o <<= 1) {
                    const int32_t t = __shfl_up_sync(G2_FULL, c, o);
                    if (lane >= o) c += t;
                }
                if (lane < CL) s_off[lane + 1] = c;
                if (lane == 0) {
                    s_off[0] = 0;
                    s_over = ov;
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
            // level d to the global list
            const int32_t mine = s_off[rank + 1] - s_off[rank];
            int32_t *dst = s.lvl + start + s_off[rank];
            for (int32_t j = threadIdx.x; j < mine; j += kClCta) dst[j] = s_q[cb * kBcQcap + j];
            if (total > a.hi) {
                reason = CL_TO_GRID;
                break;
            }
        }
        if (rank == 0 && threadIdx.x == 0) a.off[d] = start;
        const int32_t *cur = s_q + cb * kBcQcap;
        int32_t *nxt = s_q + nb * kBcQcap;
        const int32_t lo = (int32_t)((int64_t)total * rank / CL);
        const int32_t hi = (int32_t)((int64_t)total * (rank + 1) / CL);
        for (int32_t base = lo + warp * 32; base < hi; base += kClCta) {
            const int32_t i = base + lane;
            int32_t u = 0, beg = 0, deg = 0;
            if (i < hi) {
                if (first) {
                    u = s.lvl[start + i];
                } else {
                    const int r = cl_owner<CL>(s_off, i);
                    u = cl_read(cur + (i - s_off[r]), (uint32_t)r);
                }
                beg = __ldg(rowptr + u);
                deg = __ldg(rowptr + u + 1) - beg;
                if (d > 0) bc_finish_sigma(s, u, bc_sigma_thread(s, u, d - 1));
            }
            int32_t incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t t = __shfl_up_sync(G2_FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const int32_t tot = __shfl_sync(G2_FULL, incl, 31);
            const int32_t excl = incl - deg;
            for (int32_t k0 = 0; k0 < tot; k0 += 32 * 4) {
                int32_t v[4], dv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t k = k0 + 32 * j + lane;
                    int own = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int32_t ex = __shfl_sync(G2_FULL, excl, own + step);
                        if (ex <= k) own += step;
                    }
                    const int32_t ob = __shfl_sync(G2_FULL, beg, own);
                    const int32_t oe = __shfl_sync(G2_FULL, excl, own);
                    v[j] = k < tot ? __ldg(col + ob + (k - oe)) : -1;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) dv[j] = v[j] >= 0 ? atomicCAS(s.depth + v[j], -1, d + 1) : 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    cta_append(nxt, &s_cnt[nb], kBcQcap, v[j], v[j] >= 0 && dv[j] == -1, lane);
            }
        }
        start += total;
        cl_barrier();  // level d+1 found, sigma of level d and the list of level d written
    }
    cl_barrier();  // no CTA leaves while a peer may still read its counts
    if (rank == 0 && threadIdx.x == 0) {
        a.result[0] = reason;
        a.result[1] = d;
        a.result[2] = start;
        a.result[3] = total;
        a.off[d] = start;
        if (reason == CL_TO_GRID) a.off[d + 1] = start + total;
    }
}

// ------------------------------------------------------------------- host
static g2_status bc_one_plain(g2_graph *g, const BcState &s, const g2_hybrid &h,
                              std::vector<int32_t> &off, cudaStream_t st, int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    uint32_t *bm;
    uint8_t *bo;
    G2_TRY(ws(g, B_BM0, (size_t)(n + 31) / 32 + 1, &bm));
    G2_TRY(ws(g, B_BOOL0, (size_t)std::max(n, 1), &bo));
    k_bc_init<<<grid_for(g, n, kCta), kCta, 0, st>>>(s, n, nullptr);
    stats().launches += 1;
    off.assign(1, 0);
    off.push_back(1);
    for (int d = 0;; ++d) {
        int32_t b = off[d], e = off[d + 1];
        int32_t size = e - b;
        const g2_schedule &sc = pick_schedule(h, size, n);
        G2_TRY(check_schedule(g, sc, K_BFS, false));
        if (sc.load_balance == G2_LB_EDGE_ONLY)
            return fail(G2_EUNSUPPORTED, "BC's BFS is frontier-driven; EDGE_ONLY is for full sweeps");
        VSet in{OUT_SPARSE, s.lvl + b, size, nullptr, nullptr, nullptr, size};
        if (sc.direction == G2_PULL) {
            int want = sc.pull_frontier == G2_BITMAP ? OUT_BITMAP : OUT_BOOLMAP;
            VSet tt{want, nullptr, 0, nullptr, bm, bo, size};
            G2_TRY(vset_convert(g, in, want, tt, st));
            in = tt;
        }
        OpArgs a;
        memset(&a, 0, sizeof(a));
        a.kind = K_BFS;
        a.i0 = s.depth;
        a.err = d_err;
        a.threshold = G2_INF32;
        OutArgs o;
        memset(&o, 0, sizeof(o));
        o.rep = OUT_SPARSE;  // the level lists are needed for the backward pass
        o.q = s.lvl + e;
        o.qcap = n - e;
        o.cnt = ctrs + 3;
        o.dedup = DD_NONE;
        G2_CK(cudaMemsetAsync(o.cnt, 0, 4, st));
        G2_TRY(apply_round(g, sc, a, in, o, st));
        sc.direction == G2_PUSH ? stats().push_rounds++ : stats().pull_rounds++;
        G2_TRY(read_counters(g, ctrs, 4, st, d_err));
        int32_t nn = g->h_ctr[3];
        if (nn == 0) break;
        k_bc_level<true><<<grid_for(g, (int64_t)nn * 32, kCta), kCta, 0, st>>>(s, s.lvl + e, nn, d);
        stats().launches += 1;
        stats().iterations++;
        off.push_back(e + nn);
    }
    const int D = (int)off.size() - 1;  // number of levels
    for (int L = D - 2; L >= 0; --L) {
        int32_t cnt = off[L + 1] - off[L];
        k_bc_level<false><<<grid_for(g, (int64_t)cnt * 32, kCta), kCta, 0, st>>>(s, s.lvl + off[L],
                                                                                cnt, L);
        stats().launches += 1;
    }
    G2_CK(cudaGetLastError());
    return G2_OK;
}

template <class A>
static g2_status launch_bc_grid(g2_graph *g, const g2_schedule &sc, A &a, cudaStream_t st) {
    auto launch = [&](auto kern) -> g2_status {
        int per_sm = 0;
        G2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCta, 0));
        if (per_sm < 1) return fail(G2_EUNSUPPORTED, "fused BC kernel does not fit on an SM");
        void *params[] = {&a};
        G2_CK(cudaLaunchCooperativeKernel((const void *)kern, dim3(g->topo->sm_count), dim3(kCta),
                                          params, 0, st));
        stats().launches += 1;
        return G2_OK;
    };
    switch (sc.load_balance) {
        case G2_LB_WM: return launch(k_bc_fused<G2_LB_WM>);
        case G2_LB_CM: return launch(k_bc_fused<G2_LB_CM>);
        case G2_LB_ETWC: return launch(k_bc_fused<G2_LB_ETWC>);
        default: return launch(k_bc_fused<G2_LB_VERTEX_BASED>);
    }
}

static g2_status check_fused_bc(const g2_schedule &sc) {
    switch (sc.load_balance) {
        case G2_LB_VERTEX_BASED: case G2_LB_WM: case G2_LB_CM: case G2_LB_ETWC: break;
        default:
            return fail(G2_EUNSUPPORTED, "fused BC supports VERTEX_BASED, WM, CM and ETWC");
    }
    if (sc.direction != G2_PUSH) return fail(G2_EUNSUPPORTED, "fused BC runs PUSH discovery");
    return G2_OK;
}

// One source in one grid-wide cooperative launch (forward and backward).
static g2_status bc_one_fused(g2_graph *g, const BcState &s, const g2_schedule &sc, cudaStream_t st,
                              int32_t *d_err) {
    G2_TRY(check_fused_bc(sc));
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    BcFusedArgs a;
    memset(&a, 0, sizeof(a));
    a.s = s;
    G2_TRY(ws(g, B_I1, (size_t)n + 2, &a.off));
    a.cnt3 = ctrs + 20;
    a.bar = GridBarrier{reinterpret_cast<unsigned long long *>(ctrs + 28)};
    a.err = d_err;
    a.limit_ns = barrier_limit_ns();
    a.fwd = 1;
    a.d0 = 0;
    a.b0 = 0;
    a.e0 = 1;
    a.lo = 0;
    a.bwd = 1;
    a.Llo = 0;
    a.result = ctrs + 24;
    k_bc_init<<<grid_for(g, n, kCta), kCta, 0, st>>>(s, n, ctrs + 20);
    stats().launches += 1;
    G2_TRY(put_i32(st, {{a.off, 0}, {a.off + 1, 1}}));
    G2_CK(cudaMemsetAsync(ctrs + 28, 0, 8, st));  // barrier words
    G2_TRY(launch_bc_grid(g, sc, a, st));
    G2_TRY(read_counters(g, ctrs + 24, 2, st, d_err));
    stats().iterations += g->h_ctr[1];
    stats().barriers += 2 * g->h_ctr[1];
    return G2_OK;
}

// One fused WM source whose small levels run in one cluster of `cl` CTAs and
// large ones in the grid-wide kernel: the forward pass moves between the two
// at level boundaries (to the grid above `hi` vertices, back below `lo`), the
// backward pass runs each maximal range of small or large levels on one or
// the other.
static g2_status bc_one_cluster(g2_graph *g, const BcState &s, const g2_schedule &sc, int cl,
                                cudaStream_t st, int32_t *d_err) {
    G2_TRY(check_fused_bc(sc));
    Topology *t = g->topo;
    const int32_t n = t->n;
    int32_t *ctrs = d_err - 62;
    int32_t *off;
    G2_TRY(ws(g, B_I1, (size_t)n + 2, &off));
    ClusterBcArgs c;
    memset(&c, 0, sizeof(c));
    c.s = s;
    c.off = off;
    c.hi = env_i32("G2_CLUSTER_BC_HI", 256 * cl);
    c.result = ctrs + 32;
    BcFusedArgs a;
    memset(&a, 0, sizeof(a));
    a.s = s;
    a.off = off;
    a.cnt3 = ctrs + 20;
    a.bar = GridBarrier{reinterpret_cast<unsigned long long *>(ctrs + 28)};
    a.err = d_err;
    a.limit_ns = barrier_limit_ns();
    a.lo = std::max(1, env_i32("G2_CLUSTER_BC_LO", 128 * cl));
    a.result = ctrs + 24;
    const size_t smem = kBcSmem;
    auto cluster = [&]() -> g2_status {
        return cl == 16 ? launch_cluster(k_bc_cluster<16>, 16, smem, c, st)
                        : launch_cluster(k_bc_cluster<8>, 8, smem, c, st);
    };
    k_bc_init<<<grid_for(g, n, kCta), kCta, 0, st>>>(s, n, nullptr);
    stats().launches += 1;
    G2_CK(cudaGetLastError());
    G2_CK(cudaMemsetAsync(ctrs + 28, 0, 8, st));  // barrier words
    // forward
    int32_t level = 0, start = 0, count = 1, D = 0;
    bool in_cluster = true;
    for (;;) {
        if (in_cluster) {
            c.fwd = 1;
            c.d0 = level;
            c.start0 = start;
            c.n0 = count;
            G2_TRY(cluster());
            G2_TRY(read_counters(g, ctrs + 32, 4, st, d_err));
            const int32_t why = g->h_ctr[0], d = g->h_ctr[1];
            if (d <= level) return fail(G2_ECUDA, "cluster BC made no progress");
            level = d;
            start = g->h_ctr[2];
            count = g->h_ctr[3];
            if (why == CL_DONE) {
                D = d;
                break;
            }
            if (why == CL_OVERFLOW) {  // the level's list from the depths
                G2_CK(cudaMemsetAsync(ctrs + 36, 0, 4, st));
                k_level_list<<<grid_for(g, n, kCta), kCta, 0, st>>>(s.depth, n, level, s.lvl + start,
                                                                    ctrs + 36, d_err);
                stats().launches += 1;
                G2_TRY(read_counters(g, ctrs + 36, 1, st, d_err));
                count = g->h_ctr[0];
            }
        } else {
            G2_TRY(put_i32(st, {{off + level, start}, {off + level + 1, start + count}}));
            G2_CK(cudaMemsetAsync(a.cnt3, 0, 12, st));
            a.fwd = 1;
            a.bwd = 0;
            a.d0 = level;
            a.b0 = start;
            a.e0 = start + count;
            G2_TRY(launch_bc_grid(g, sc, a, st));
            G2_TRY(read_counters(g, ctrs + 24, 4, st, d_err));
            const int32_t back = g->h_ctr[0], d = g->h_ctr[1];
            if (d <= level) return fail(G2_ECUDA, "fused BC made no progress");
            if (!back) {
                D = d;
                break;
            }
            level = d;
            start = g->h_ctr[2];
            count = g->h_ctr[3];
        }
        in_cluster = !in_cluster;
    }
    stats().iterations += D;
    stats().barriers += 2 * D;
    // backward over levels D-2 .. 0, by ranges of small / large levels
    if (D < 2) return G2_OK;
    std::vector<int32_t> offs((size_t)D + 1);
    G2_CK(cudaMemcpyAsync(offs.data(), off, ((size_t)D + 1) * 4, cudaMemcpyDeviceToHost, st));
    G2_TRY(sync_and_check(g, st, d_err));
    for (int32_t L = D - 2; L >= 0;) {
        const bool small = offs[L + 1] - offs[L] <= c.hi;
        int32_t Llo = L;
        while (Llo > 0 && (offs[Llo] - offs[Llo - 1] <= c.hi) == small) --Llo;
        if (small) {
            c.fwd = 0;
            c.Lhi = L;
            c.Llo = Llo;
            G2_TRY(cluster());
        } else {
            a.fwd = 0;
            a.Lhi = L;
            a.Llo = Llo;
            G2_TRY(launch_bc_grid(g, sc, a, st));
        }
        L = Llo - 1;
    }
    return G2_OK;
}

g2_status bc_run(g2_graph *g, const int32_t *srcs, int32_t k, double *bc, const g2_hybrid &h,
                 cudaStream_t st, int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    BcState s;
    s.g = t->view();
    s.bc = bc;
    int32_t dmax = 0;
    G2_TRY(max_out_degree(g, st, &dmax));
    s.per_thread = t->symmetric && dmax <= kBoundedDegree;
    s.big = !(t->symmetric && dmax < kBigDeg);
    G2_TRY(ws(g, B_I0, (size_t)std::max(n, 1), &s.depth));
    G2_TRY(ws(g, B_LVL, (size_t)std::max(n, 1), &s.lvl));
    G2_TRY(ws(g, B_D0, (size_t)std::max(n, 1), &s.sm));
    G2_TRY(ws(g, B_D1, (size_t)std::max(n, 1), &s.coef));
    G2_TRY(ws(g, B_F2, (size_t)std::max(n, 1), &s.se));
    G2_CK(cudaMemsetAsync(bc, 0, (size_t)n * 8, st));
    std::vector<int32_t> off;
    // fused WM sources on a symmetric bounded-degree graph use the cluster
    const int cl = h.s1.kernel_fusion && h.s1.load_balance == G2_LB_WM && s.per_thread
                       ? cluster_size(2, k_bc_cluster<16>, k_bc_cluster<8>, kBcSmem)
                       : 0;
    for (int32_t i = 0; i < k; ++i) {
        s.src = srcs[i];
        if (cl) G2_TRY(bc_one_cluster(g, s, h.s1, cl, st, d_err));
        else if (h.s1.kernel_fusion) G2_TRY(bc_one_fused(g, s, h.s1, st, d_err));
        else G2_TRY(bc_one_plain(g, s, h, off, st, d_err));
        G2_TRY(sync_and_check(g, st, d_err));
    }
    return G2_OK;
}

}  // namespace g2

using namespace g2;

// Tuned schedule when the caller passes none: the direction-optimising
// hybrid of BFS (STRICT PUSH below 2% of n, VERTEX_BASED PULL over a bitmap);
// on a bounded-degree graph each source runs fused (WM PUSH).
static g2_hybrid tuned_bc_hybrid(g2_graph *g, cudaStream_t st) {
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
    h.s2.pull_frontier = G2_BITMAP;
    h.s2.dedup = G2_DEDUP_DISABLED;
    return h;
}

extern "C" g2_status g2_bc(g2_graph *g, const int32_t *srcs, int32_t k, double *bc,
                           const g2_hybrid *sched, void *stream) {
    if (!g || !bc || (k > 0 && !srcs) || k < 0) return fail(G2_EINVAL, "bad BC arguments");
    for (int32_t i = 0; i < k; ++i)
        if (srcs[i] < 0 || srcs[i] >= g->topo->n) return fail(G2_EINVAL, "source vertex out of range");
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : tuned_bc_hybrid(g, st);
    if (h.s1.kernel_fusion && h.criteria != G2_CRITERIA_NONE && !h.s2.kernel_fusion)
        return fail(G2_EUNSUPPORTED, "kernel fusion must be set on both hybrid schedules");
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    G2_TRY(bc_run(g, srcs, k, bc, h, st, d_err));
    return end_call(g, st, d_err);
}
