// g2_algos.cu — BFS, connected components, delta-stepping SSSP and
// betweenness centrality (Sec. VII) as host loops over edgeset.apply rounds
// (the default, unfused schedules: the host reads the frontier size every
// round, Fig. 5 left / right).  The fused variants live in g2_fused.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "g2_host.h"
#include "g2_lb.cuh"

namespace g2 {

g2_status bfs_fused(g2_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                    const g2_schedule &s, cudaStream_t st, int32_t *d_err);
g2_status bfs_fused_do(g2_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                       const g2_hybrid &h, cudaStream_t st, int32_t *d_err);
g2_status sssp_fused(g2_graph *g, int32_t src, int32_t delta, int32_t *dist,
                     const g2_schedule &s, cudaStream_t st, int32_t *d_err);

// ------------------------------------------------------------------ kernels
__global__ void k_bfs_init(int32_t *depth, int32_t *parent, int32_t n, int32_t src, int32_t *q,
                           int32_t *cnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        depth[v] = v == src ? 0 : -1;
        if (parent) parent[v] = v == src ? src : -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        q[0] = src;
        *cnt = 1;
    }
}

__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t val) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        a[v] = val;
}

__global__ void k_iota(int32_t *a, int32_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        a[v] = (int32_t)v;
}

// Pointer jumping: every label is replaced by the root of its chain.  Roots
// do not change during this kernel (hooking ran before it), so the chase ends.
__global__ void k_compress(int32_t *label, int32_t n) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t l = label[v];
        int32_t p = label[l];
        while (p != l) {
            l = p;
            p = label[l];
        }
        label[v] = l;
    }
}

// Lock-free union of the trees of u and v: the higher root is hung under the
// lower one by compare-and-swap, so the minimum id of every tree stays its
// root.  Labels only decrease, so the loop ends (Sutton et al., "Optimizing
// parallel graph connectivity computation via subgraph sampling", 2018).
__device__ __forceinline__ void cc_link(int32_t *label, int32_t u, int32_t v) {
    int32_t p1 = label[u], p2 = label[v];
    while (p1 != p2) {
        int32_t hi = p1 > p2 ? p1 : p2, lo = p1 + p2 - hi;
        int32_t ph = label[hi];
        if (ph == lo) break;
        if (ph == hi && atomicCAS(&label[hi], hi, lo) == hi) break;
        p1 = label[label[hi]];
        p2 = label[lo];
    }
}

// link every vertex with its r-th neighbour
__global__ void k_cc_sample(const int32_t *rowptr, const int32_t *col, int32_t n, int32_t r,
                            int32_t *label, unsigned long long *ctr) {
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + threadIdx.x;
        bool linked = false;
        if (v < n) {
            int32_t b = rowptr[v];
            if (rowptr[v + 1] - b > r) {
                cc_link(label, (int32_t)v, col[b + r]);
                linked = true;
            }
        }
        count_arcs(ctr, linked);
    }
}

// labels of a fixed pseudo-random sample of vertices
__global__ void k_cc_probe(const int32_t *label, int32_t n, int32_t k, int32_t *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) {
        uint32_t h = (uint32_t)i * 2654435761u + 0x9E3779B9u;
        h ^= h >> 16;
        h *= 0x85EBCA6Bu;
        h ^= h >> 13;
        out[i] = label[h % (uint32_t)n];
    }
}

// link the remaining arcs (from position `skip` on) of every vertex outside
// the component `giant`; a warp walks one vertex so long lists are shared
__global__ void k_cc_finish(const int32_t *rowptr, const int32_t *col, int32_t n, int32_t skip,
                            int32_t giant, int32_t *label, unsigned long long *ctr) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < n; base += nw * 32) {
        int64_t v = base + lane;
        bool act = v < n && label[v] != giant && rowptr[v + 1] - rowptr[v] > skip;
        unsigned m = __ballot_sync(G2_FULL, act);
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1;
            int32_t u = (int32_t)(base + src);
            int32_t b = rowptr[u] + skip, e = rowptr[u + 1];
            for (int32_t k = b + lane; k < e; k += 32) cc_link(label, u, col[k]);
            if (ctr && lane == 0) atomicAdd(ctr, (unsigned long long)(e - b));
        }
    }
}

// list of vertices whose label differs from the round-start snapshot
__global__ void k_changed(const int32_t *label, const int32_t *lab0, int32_t n, int32_t *q,
                          int32_t *cnt) {
    int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = base + lane;
        bool p = v < n && label[v] != lab0[v];
        warp_append(q, cnt, n, nullptr, (int32_t)v, p);
    }
    (void)lane;
}

// smallest dist among far-pile entries that are not stale (dist >= T)
__global__ void k_far_min(const int32_t *far, int32_t nfar, const int32_t *dist, int32_t T,
                          int32_t *out_min) {
    int32_t best = G2_INF32;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nfar;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = dist[far[i]];
        if (d >= T && d < best) best = d;
    }
    best = (int32_t)__reduce_min_sync(G2_FULL, (unsigned)best);
    if ((threadIdx.x & 31) == 0 && best != G2_INF32) atomicMin(out_min, best);
}

// split the far pile at the new threshold: stale entries (dist < Told) are
// dropped, dist < Tnew go to the near list, the rest to the next far pile
__global__ void k_far_split(const int32_t *far, int32_t nfar, const int32_t *dist, int32_t Told,
                            int32_t Tnew, int32_t *nearq, int32_t *nearcnt, int32_t *far2,
                            int32_t *far2cnt, int32_t cap, int32_t *stamp2, int32_t round2,
                            int32_t *err) {
    int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nfar;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + lane;
        int32_t v = 0, d = G2_INF32;
        bool ok = i < nfar;
        if (ok) {
            v = far[i];
            d = dist[v];
        }
        bool to_near = ok && d >= Told && d < Tnew;
        bool to_far = ok && d >= Tnew;
        if (to_far) stamp2[v] = round2;
        warp_append(nearq, nearcnt, cap, err, v, to_near);
        warp_append(far2, far2cnt, cap, err, v, to_far);
    }
    (void)lane;
}


// --------------------------------------------------------------- helpers
struct Ping {
    int32_t *q[2];
    uint32_t *bm[2];
    uint8_t *bo[2];
    int32_t qcap;
};

static g2_status get_ping(g2_graph *g, Ping &p, bool bitmaps, bool boolmaps) {
    const int32_t n = std::max(g->topo->n, 1);
    G2_TRY(ws(g, B_Q0, (size_t)n, &p.q[0]));
    G2_TRY(ws(g, B_Q1, (size_t)n, &p.q[1]));
    p.qcap = n;
    p.bm[0] = p.bm[1] = nullptr;
    p.bo[0] = p.bo[1] = nullptr;
    size_t words = (size_t)(n + 31) / 32 + 1;
    if (bitmaps) {
        G2_TRY(ws(g, B_BM0, words, &p.bm[0]));
        G2_TRY(ws(g, B_BM1, words, &p.bm[1]));
    }
    if (boolmaps) {
        G2_TRY(ws(g, B_BOOL0, (size_t)n, &p.bo[0]));
        G2_TRY(ws(g, B_BOOL1, (size_t)n, &p.bo[1]));
    }
    return G2_OK;
}

static bool hybrid_uses(const g2_hybrid &h, int what) {
    auto uses = [&](const g2_schedule &s) {
        if (what == 0) return s.direction == G2_PULL || s.frontier_creation != G2_FUSED;
        return false;
    };
    return uses(h.s1) || (h.criteria == G2_INPUT_VERTEXSET_SIZE && uses(h.s2));
}

static int dedup_of(const g2_schedule &s) {
    if (s.dedup == G2_DEDUP_DISABLED) return DD_NONE;
    if (s.dedup_type == G2_DEDUP_BITMAP) return DD_BITMAP;
    if (s.dedup_type == G2_DEDUP_BOOLMAP) return DD_BOOLMAP;
    return DD_STAMP;
}

// One frontier round of a vertex-set loop: brings `cur` (parity p) to the
// representation the schedule wants, runs the round into parity 1-p with the
// schedule's frontier creation, and returns the new vertexset with its size.
static g2_status frontier_round(g2_graph *g, const g2_schedule &s, const OpArgs &a, VSet cur,
                                int p, const Ping &pp, int32_t *ctrs, int32_t *d_err, VSet &next,
                                cudaStream_t st) {
    VSet in = cur;
    if (cur.rep != -1) {
        if (s.direction == G2_PUSH && cur.rep != OUT_SPARSE) {
            VSet t{OUT_SPARSE, pp.q[p], pp.qcap, ctrs + p, nullptr, nullptr, cur.size};
            G2_TRY(vset_convert(g, cur, OUT_SPARSE, t, st));
            in = t;
        } else if (s.direction == G2_PULL) {
            int want = s.pull_frontier == G2_BITMAP ? OUT_BITMAP : OUT_BOOLMAP;
            if (cur.rep != want) {
                VSet t{want, nullptr, 0, nullptr, pp.bm[p], pp.bo[p], cur.size};
                G2_TRY(vset_convert(g, cur, want, t, st));
                in = t;
            }
        }
    }
    const int32_t n = g->topo->n;
    OutArgs o;
    memset(&o, 0, sizeof(o));
    int q = 1 - p;
    if (s.frontier_creation == G2_FUSED) {
        o.rep = OUT_SPARSE;
        o.q = pp.q[q];
        o.qcap = pp.qcap;
        o.cnt = ctrs + q;
        o.dedup = dedup_of(s);
        G2_CK(cudaMemsetAsync(o.cnt, 0, 4, st));
        next = VSet{OUT_SPARSE, o.q, o.qcap, o.cnt, nullptr, nullptr, 0};
    } else if (s.frontier_creation == G2_UNFUSED_BITMAP) {
        o.rep = OUT_BITMAP;
        o.bitmap = pp.bm[q];
        G2_CK(cudaMemsetAsync(o.bitmap, 0, ((size_t)(n + 31) / 32 + 1) * 4, st));
        next = VSet{OUT_BITMAP, nullptr, 0, nullptr, o.bitmap, nullptr, 0};
    } else {
        o.rep = OUT_BOOLMAP;
        o.boolmap = pp.bo[q];
        G2_CK(cudaMemsetAsync(o.boolmap, 0, (size_t)std::max(n, 1), st));
        next = VSet{OUT_BOOLMAP, nullptr, 0, nullptr, nullptr, o.boolmap, 0};
    }
    G2_TRY(apply_round(g, s, a, in, o, st));
    if (s.direction == G2_PUSH) stats().push_rounds++;
    else stats().pull_rounds++;
    if (next.rep != OUT_SPARSE) G2_TRY(vset_count(g, next, ctrs + 2, st));
    G2_TRY(read_counters(g, ctrs, 4, st, d_err));
    next.size = next.rep == OUT_SPARSE ? g->h_ctr[q] : g->h_ctr[2];
    return G2_OK;
}

static g2_status check_src(const g2_graph *g, int32_t src) {
    if (src < 0 || src >= g->topo->n) return fail(G2_EINVAL, "source vertex out of range");
    return G2_OK;
}

// ===================================================================== BFS
g2_status bfs_plain(g2_graph *g, int32_t src, int32_t *depth, int32_t *parent, const g2_hybrid &h,
                    cudaStream_t st, int32_t *d_err) {
    const int32_t n = g->topo->n;
    Ping pp;
    G2_TRY(get_ping(g, pp, true, true));
    int32_t *ctrs = d_err - 62;
    k_bfs_init<<<grid_for(g, n, kCta), kCta, 0, st>>>(depth, parent, n, src, pp.q[0], ctrs + 0);
    stats().launches += 1;
    VSet cur{OUT_SPARSE, pp.q[0], pp.qcap, ctrs + 0, nullptr, nullptr, 1};
    OpArgs a;
    memset(&a, 0, sizeof(a));
    a.kind = K_BFS;
    a.i0 = depth;
    a.i1 = parent;
    a.err = d_err;
    a.threshold = G2_INF32;
    int p = 0;
    while (cur.size > 0) {
        const g2_schedule &s = pick_schedule(h, cur.size, n);
        G2_TRY(check_schedule(g, s, K_BFS, false));
        if (s.load_balance == G2_LB_EDGE_ONLY)
            return fail(G2_EUNSUPPORTED, "BFS is frontier-driven; EDGE_ONLY is for full sweeps");
        VSet next;
        G2_TRY(frontier_round(g, s, a, cur, p, pp, ctrs, d_err, next, st));
        cur = next;
        p = 1 - p;
        stats().iterations++;
        if (stats().iterations > n + 1) return fail(G2_EOVERFLOW, "BFS did not terminate");
    }
    return G2_OK;
}

// ====================================================================== CC
g2_status cc_run(g2_graph *g, int32_t *label, const g2_hybrid &h, cudaStream_t st,
                 int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    Ping pp;
    G2_TRY(get_ping(g, pp, true, true));
    int32_t *ctrs = d_err - 62;
    int32_t *lab0;
    G2_TRY(ws(g, B_I0, (size_t)std::max(n, 1), &lab0));
    k_iota<<<grid_for(g, n, kCta), kCta, 0, st>>>(label, n);
    stats().launches += 1;
    VSet cur{-1, nullptr, 0, nullptr, nullptr, nullptr, n};
    int p = 0;
    while (cur.size > 0) {
        const g2_schedule &s = pick_schedule(h, cur.size, n);
        G2_TRY(check_schedule(g, s, s.direction == G2_PULL ? K_LABEL : K_HOOK, true));
        G2_CK(cudaMemcpyAsync(lab0, label, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
        OpArgs a;
        memset(&a, 0, sizeof(a));
        a.i0 = label;
        a.err = d_err;
        a.threshold = G2_INF32;
        OutArgs none;
        memset(&none, 0, sizeof(none));
        none.rep = OUT_NONE;
        VSet in = cur;
        if (s.direction == G2_PUSH) {
            a.kind = K_HOOK;
            // an EDGE_ONLY sweep covers every arc, a superset of the active ones
            if (s.load_balance == G2_LB_EDGE_ONLY) in = VSet{-1, nullptr, 0, nullptr, nullptr, nullptr, n};
            stats().push_rounds++;
        } else {
            a.kind = K_LABEL;
            if (cur.rep != -1) {
                int want = s.pull_frontier == G2_BITMAP ? OUT_BITMAP : OUT_BOOLMAP;
                VSet tt{want, nullptr, 0, nullptr, pp.bm[p], pp.bo[p], cur.size};
                G2_TRY(vset_convert(g, cur, want, tt, st));
                in = tt;
            }
            stats().pull_rounds++;
        }
        G2_TRY(apply_round(g, s, a, in, none, st));
        k_compress<<<grid_for(g, n, kCta), kCta, 0, st>>>(label, n);
        int q = 1 - p;
        G2_CK(cudaMemsetAsync(ctrs + q, 0, 4, st));
        k_changed<<<grid_for(g, n, kCta), kCta, 0, st>>>(label, lab0, n, pp.q[q], ctrs + q);
        stats().launches += 2;
        G2_TRY(read_counters(g, ctrs, 4, st, d_err));
        cur = VSet{OUT_SPARSE, pp.q[q], pp.qcap, ctrs + q, nullptr, nullptr, g->h_ctr[q]};
        p = q;
        stats().iterations++;
        if (stats().iterations > n + 2) return fail(G2_EOVERFLOW, "CC did not converge");
    }
    return G2_OK;
}

// Tuned CC: neighbour sampling with lock-free linking (two sampling rounds,
// compress, giant component from a sample of labels, link the rest of the
// arcs of the vertices outside it, compress).  Output: min-id labels.
g2_status cc_sampled(g2_graph *g, int32_t *label, cudaStream_t st, int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    if (n == 0) return G2_OK;
    constexpr int kSample = 2, kProbe = 1024;
    const int grid = grid_for(g, n, kCta);
    // arcs linked (stats mode): one per vertex and sampling round, then the
    // remaining arcs of the vertices outside the giant component
    unsigned long long *ctr = nullptr;
    if (count_arcs_enabled()) G2_TRY(ws(g, B_ARCS, 2, &ctr));
    k_iota<<<grid, kCta, 0, st>>>(label, n);
    for (int r = 0; r < kSample; ++r) {
        k_cc_sample<<<grid, kCta, 0, st>>>(t->rowptr, t->col, n, r, label, ctr);
        k_compress<<<grid, kCta, 0, st>>>(label, n);
    }
    int32_t *probe;
    G2_TRY(ws(g, B_I1, kProbe, &probe));
    k_cc_probe<<<(kProbe + kCta - 1) / kCta, kCta, 0, st>>>(label, n, kProbe, probe);
    std::vector<int32_t> h(kProbe);
    G2_CK(cudaMemcpyAsync(h.data(), probe, kProbe * 4, cudaMemcpyDeviceToHost, st));
    G2_TRY(sync_and_check(g, st, d_err));
    std::sort(h.begin(), h.end());
    int32_t giant = h[0];
    int best = 0;
    for (int i = 0; i < kProbe;) {
        int j = i;
        while (j < kProbe && h[j] == h[i]) ++j;
        if (j - i > best) {
            best = j - i;
            giant = h[i];
        }
        i = j;
    }
    k_cc_finish<<<grid_for(g, n, kCta), kCta, 0, st>>>(t->rowptr, t->col, n, kSample, giant, label,
                                                        ctr);
    k_compress<<<grid, kCta, 0, st>>>(label, n);
    stats().launches += 2 * kSample + 5;
    stats().iterations = kSample + 1;
    G2_CK(cudaGetLastError());
    return G2_OK;
}

// ==================================================================== SSSP
g2_status sssp_plain(g2_graph *g, int32_t src, int32_t delta, int32_t *dist, const g2_hybrid &h,
                     cudaStream_t st, int32_t *d_err) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    Ping pp;
    G2_TRY(get_ping(g, pp, false, false));
    int32_t *ctrs = d_err - 62;
    int32_t *far[2], *stamp2;
    G2_TRY(ws(g, B_Q2, (size_t)std::max(n, 1), &far[0]));
    G2_TRY(ws(g, B_Q3, (size_t)std::max(n, 1), &far[1]));
    G2_TRY(ws(g, B_STAMP2, (size_t)std::max(n, 1), &stamp2));
    if (g->round2 == 0 || g->round2 > 0x7ffffff0) {
        G2_CK(cudaMemsetAsync(stamp2, 0, (size_t)std::max(n, 1) * 4, st));
        g->round2 = 0;
    }
    // near lists: capacity n with deduplication; without it one round can
    // enqueue a vertex once per improving arc, so up to m entries
    const g2_schedule &s0 = h.s1;
    int32_t *nq[2] = {pp.q[0], pp.q[1]};
    int32_t ncap = pp.qcap;
    if (s0.dedup == G2_DEDUP_DISABLED ||
        (h.criteria == G2_INPUT_VERTEXSET_SIZE && h.s2.dedup == G2_DEDUP_DISABLED)) {
        int32_t *big;
        size_t half = (size_t)t->m + (size_t)n + 1;
        G2_TRY(ws(g, B_BIG, 2 * half, &big));
        nq[0] = big;
        nq[1] = big + half;
        ncap = (int32_t)std::min<size_t>(half, 2147483647u);
    }
    k_fill_i32<<<grid_for(g, n, kCta), kCta, 0, st>>>(dist, n, G2_INF32);
    int32_t zero = 0, one = 1;
    G2_TRY(put_i32(st, {{dist + src, zero}, {nq[0], src}, {ctrs + 0, one}}));
    stats().launches += 1;
    int64_t T = delta;  // bucket 0 = [0, delta)
    int fp = 0;
    int32_t round2 = ++g->round2;
    G2_CK(cudaMemsetAsync(ctrs + 4, 0, 8, st));
    int32_t near_size = 1, p = 0;
    for (;;) {
        while (near_size > 0) {
            const g2_schedule &s = pick_schedule(h, near_size, n);
            G2_TRY(check_schedule(g, s, K_RELAX, false));
            if (s.direction != G2_PUSH || s.load_balance == G2_LB_EDGE_ONLY)
                return fail(G2_EUNSUPPORTED, "delta-stepping relaxes in the PUSH direction");
            if (s.frontier_creation != G2_FUSED)
                return fail(G2_EUNSUPPORTED, "the near/far queue needs FUSED frontier creation");
            OpArgs a;
            memset(&a, 0, sizeof(a));
            a.kind = K_RELAX;
            a.i0 = dist;
            a.err = d_err;
            a.threshold = (int32_t)std::min<int64_t>(T, G2_INF32);
            OutArgs o;
            memset(&o, 0, sizeof(o));
            o.rep = OUT_SPARSE;
            o.dedup = dedup_of(s);
            int q = 1 - p;
            if (o.dedup == DD_NONE && nq[0] == pp.q[0])
                return fail(G2_EINVAL, "dedup DISABLED must be set on the first schedule too");
            o.q = nq[q];
            o.qcap = ncap;
            o.cnt = ctrs + q;
            G2_CK(cudaMemsetAsync(o.cnt, 0, 4, st));
            o.q2 = far[fp];
            o.q2cap = std::max(n, 1);
            o.cnt2 = ctrs + 4 + fp;
            o.stamp2 = stamp2;
            o.round2 = round2;
            VSet in{OUT_SPARSE, nq[p], ncap, ctrs + p, nullptr, nullptr, near_size};
            G2_TRY(apply_round(g, s, a, in, o, st));
            stats().push_rounds++;
            G2_TRY(read_counters(g, ctrs, 8, st, d_err));
            near_size = g->h_ctr[q];
            p = q;
            stats().iterations++;
        }
        int32_t nfar = g->h_ctr[4 + fp];
        if (nfar == 0) break;
        int32_t Told = (int32_t)std::min<int64_t>(T, G2_INF32);
        int32_t inf = G2_INF32;
        G2_TRY(put_i32(st, {{ctrs + 6, inf}}));
        k_far_min<<<grid_for(g, nfar, kCta), kCta, 0, st>>>(far[fp], nfar, dist, Told, ctrs + 6);
        G2_TRY(read_counters(g, ctrs, 8, st, d_err));
        int32_t dmin = g->h_ctr[6];
        if (dmin == G2_INF32) break;
        int64_t Tnew = ((int64_t)dmin / delta + 1) * (int64_t)delta;
        int32_t Tn = (int32_t)std::min<int64_t>(Tnew, G2_INF32);
        int nf = 1 - fp;
        int32_t round2n = ++g->round2;
        G2_CK(cudaMemsetAsync(ctrs + p, 0, 4, st));
        G2_CK(cudaMemsetAsync(ctrs + 4 + nf, 0, 4, st));
        k_far_split<<<grid_for(g, nfar, kCta), kCta, 0, st>>>(far[fp], nfar, dist, Told, Tn, nq[p],
                                                             ctrs + p, far[nf], ctrs + 4 + nf,
                                                             std::max(n, 1), stamp2, round2n, d_err);
        stats().launches += 2;
        G2_TRY(read_counters(g, ctrs, 8, st, d_err));
        near_size = g->h_ctr[p];
        fp = nf;
        round2 = round2n;
        T = Tnew;
        stats().barriers++;  // buckets advanced
    }
    return G2_OK;
}

}  // namespace g2

using namespace g2;

// The fused WM PUSH loop that bounded-degree graphs run by default.
static g2_hybrid fused_wm_hybrid() {
    g2_hybrid h = default_hybrid();
    h.s1.load_balance = G2_LB_WM;
    h.s1.kernel_fusion = 1;
    h.s2 = h.s1;
    return h;
}

static bool bounded_degree(g2_graph *g, cudaStream_t st) {
    int32_t d = 0;
    return max_out_degree(g, st, &d) == G2_OK && d <= kBoundedDegree;
}

// Tuned schedule for BFS when the caller passes none (measured on GB300 with
// RMAT-21 and RMAT-22): the direction-optimising hybrid fused into one
// launch, STRICT PUSH on a sparse queue while the frontier holds < 2% of the
// vertices, else VERTEX_BASED PULL over a bitmap.  Against the same hybrid
// as per-level launches it is faster from every source measured (RMAT-22,
// the hub and 8 random sources: 5.7 ms against 6.9 ms in all; from the hub
// 0.26 against 0.35 ms): no frontier size goes back to the host per level.
// STRICT divides a level's arcs evenly over the persistent grid where ETWC's
// stages leave it unbalanced behind hub arcs (fused ETWC: 20.8 ms over the
// same sources).  On a bounded-degree graph: fused WM PUSH (measured on a
// 1024^2 road grid: 7.2 ms against 35 ms for the hybrid).
static g2_hybrid tuned_bfs_hybrid(g2_graph *g, cudaStream_t st) {
    if (bounded_degree(g, st)) return fused_wm_hybrid();
    g2_hybrid h = default_hybrid();
    h.criteria = G2_INPUT_VERTEXSET_SIZE;
    h.threshold = 0.02f;
    h.s1.load_balance = G2_LB_STRICT;
    h.s1.kernel_fusion = 1;
    h.s2.load_balance = G2_LB_VERTEX_BASED;
    h.s2.direction = G2_PULL;
    h.s2.pull_frontier = G2_BITMAP;
    h.s2.frontier_creation = G2_UNFUSED_BITMAP;
    h.s2.dedup = G2_DEDUP_DISABLED;
    h.s2.kernel_fusion = 1;
    return h;
}

// Tuned schedule for delta-stepping when the caller passes none: STRICT PUSH;
// fused WM PUSH on a bounded-degree graph.
static g2_hybrid tuned_sssp_hybrid(g2_graph *g, cudaStream_t st) {
    if (bounded_degree(g, st)) return fused_wm_hybrid();
    g2_hybrid h = default_hybrid();
    h.s1.load_balance = G2_LB_STRICT;
    return h;
}

// ====================================================================== C ABI
extern "C" {

g2_status g2_bfs(g2_graph *g, int32_t src, int32_t *depth, int32_t *parent, const g2_hybrid *sched,
                 void *stream) {
    if (!g || !depth) return fail(G2_EINVAL, "null graph or depth");
    G2_TRY(check_src(g, src));
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : tuned_bfs_hybrid(g, st);
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    if (h.s1.kernel_fusion) {
        if (h.criteria != G2_CRITERIA_NONE && !h.s2.kernel_fusion)
            return fail(G2_EUNSUPPORTED, "kernel fusion must be set on both hybrid schedules");
        if (h.criteria != G2_CRITERIA_NONE && h.s2.direction == G2_PULL)
            G2_TRY(bfs_fused_do(g, src, depth, parent, h, st, d_err));
        else
            G2_TRY(bfs_fused(g, src, depth, parent, h.s1, st, d_err));
    } else {
        G2_TRY(bfs_plain(g, src, depth, parent, h, st, d_err));
    }
    return end_call(g, st, d_err);
}

g2_status g2_cc(g2_graph *g, int32_t *label, const g2_hybrid *sched, void *stream) {
    if (!g || !label) return fail(G2_EINVAL, "null graph or label");
    if (!g->topo->symmetric) return fail(G2_EINVAL, "connected components need a symmetric graph");
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : default_hybrid();
    if (h.s1.kernel_fusion) return fail(G2_EUNSUPPORTED, "CC has no fused variant");
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    if (sched) G2_TRY(cc_run(g, label, h, st, d_err));
    else G2_TRY(cc_sampled(g, label, st, d_err));
    return end_call(g, st, d_err);
}

g2_status g2_sssp_delta(g2_graph *g, int32_t src, int32_t delta, int32_t *dist,
                        const g2_hybrid *sched, void *stream) {
    if (!g || !dist) return fail(G2_EINVAL, "null graph or dist");
    G2_TRY(check_src(g, src));
    if (!g->topo->w) return fail(G2_EINVAL, "SSSP needs arc weights");
    cudaStream_t st = as_stream(stream);
    g2_hybrid h = sched ? *sched : tuned_sssp_hybrid(g, st);
    if (delta <= 0) delta = h.s1.delta > 0 ? h.s1.delta : 1;
    if (h.s1.kernel_fusion && h.criteria != G2_CRITERIA_NONE && !h.s2.kernel_fusion)
        return fail(G2_EUNSUPPORTED, "kernel fusion must be set on both hybrid schedules");
    int32_t *d_err;
    G2_TRY(begin_call(g, st, &d_err));
    if (h.s1.kernel_fusion) {
        G2_TRY(sssp_fused(g, src, delta, dist, h.s1, st, d_err));
    } else {
        G2_TRY(sssp_plain(g, src, delta, dist, h, st, d_err));
    }
    return end_call(g, st, d_err);
}

}  // extern "C"
