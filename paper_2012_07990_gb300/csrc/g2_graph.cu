// g2_graph.cu — runtime of libg2: graph load (Sec. VI-C host side) with
// device validation (inside the upload kernel where the device can read the
// caller's arrays), transpose, the stream-ordered device memory pool, the
// workspace that lets every round reuse its frontier buffers (Sec. VI-A),
// vertexset conversions, the device-wide scan, EdgeBlocking preprocessing
// (Algorithm 1) and the public frontier API.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "g2_host.h"

namespace g2 {

// ================================================================ errors/stats
static thread_local std::string t_err;
static thread_local g2_stats t_stats;
static thread_local bool t_count_arcs = false;

void set_error_msg(const std::string &msg) { t_err = msg; }
g2_status fail(g2_status st, const std::string &msg) {
    t_err = msg;
    return st;
}
g2_status cuda_fail(cudaError_t e, const char *what) {
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return G2_ENOMEM;
    return G2_ECUDA;
}
g2_stats &stats() { return t_stats; }
bool count_arcs_enabled() { return t_count_arcs; }

// --- kernel timing (events recorded around named launches)
struct KTotal {
    std::string name;
    double ms;
    int64_t launches;
};
static thread_local bool t_ktime = false;
static thread_local std::vector<cudaEvent_t> t_ev_pool;
static thread_local std::vector<KTime> t_ev_pending;
static thread_local std::vector<KTotal> t_ktotals;

static cudaEvent_t ev_get() {
    if (!t_ev_pool.empty()) {
        cudaEvent_t e = t_ev_pool.back();
        t_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void ktime_begin(KTime &k, const char *name, cudaStream_t st) {
    k.name = nullptr;
    if (!t_ktime) return;
    k.name = name;
    k.e0 = ev_get();
    k.e1 = ev_get();
    cudaEventRecord(k.e0, st);
}

void ktime_end(KTime &k, cudaStream_t st) {
    if (!k.name) return;
    cudaEventRecord(k.e1, st);
    t_ev_pending.push_back(k);
}

static void ktime_resolve() {
    for (KTime &k : t_ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, k.e0, k.e1) == cudaSuccess) {
            KTotal *tot = nullptr;
            for (KTotal &x : t_ktotals)
                if (x.name == k.name) tot = &x;
            if (!tot) {
                t_ktotals.push_back(KTotal{k.name, 0.0, 0});
                tot = &t_ktotals.back();
            }
            tot->ms += ms;
            tot->launches += 1;
        }
        t_ev_pool.push_back(k.e0);
        t_ev_pool.push_back(k.e1);
    }
    t_ev_pending.clear();
}

// ================================================================== kernels
__global__ void k_validate_rows(const int32_t *rowptr, int32_t n, int32_t m, uint32_t *rowstart,
                                int32_t *bad) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n) return;
    int32_t r = rowptr[v];
    if (v == 0 && r != 0) atomicExch(bad, 1);
    if (v == n && r != m) atomicExch(bad, 2);
    if (v < n) {
        int32_t r1 = rowptr[v + 1];
        if (r1 < r || r < 0 || r1 > m) atomicExch(bad, 3);
        else if (r1 > r) atomicOr(&rowstart[r >> 5], 1u << (r & 31));
    }
}

// Copy of the caller's column ids (and weights) into the graph's arrays with
// their checks done on the way (ids in [0, n), each list strictly ascending,
// weights >= 0; the code of the failed check to *bad): the arcs are read once.
// With dst null the kernel checks only (arcs already on the device).
// `src`/`wsrc` are device-readable addresses: device memory, pinned host
// memory, or pageable host memory on a device that reads it through the host
// page tables (a coherent CPU-GPU link); the caller checks 16-byte alignment.
// Four arcs per thread with 16-byte accesses; a warp covers 128 consecutive
// arcs per group, and the id after a thread's last arc comes from the next
// lane.  A thread loads U groups before it checks and stores them, so a small
// grid still keeps enough reads in flight to fill the host link.
template <int U>
__global__ void __launch_bounds__(256) k_load_cols(const int32_t *__restrict__ src,
                                                   const int32_t *__restrict__ wsrc,
                                                   int32_t *__restrict__ dst,
                                                   int32_t *__restrict__ wdst, int32_t n,
                                                   int32_t m, const uint32_t *rowstart,
                                                   int32_t *bad) {
    const int lane = threadIdx.x & 31;
    const int64_t nq = ((int64_t)m + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * U;
    // warp-uniform trip count (base is a multiple of 32): the shuffle below
    // always has every lane present
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * U; base < nq;
         base += stride) {
        int32_t c[U][4], wv[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t q = base + 32 * u + lane, e0 = q * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) c[u][k] = wv[u][k] = 0;
            if (q < nq) {
                if (e0 + 4 <= m) {
                    const int4 v = *reinterpret_cast<const int4 *>(src + e0);
                    c[u][0] = v.x; c[u][1] = v.y; c[u][2] = v.z; c[u][3] = v.w;
                    if (wsrc) {
                        const int4 x = *reinterpret_cast<const int4 *>(wsrc + e0);
                        wv[u][0] = x.x; wv[u][1] = x.y; wv[u][2] = x.z; wv[u][3] = x.w;
                    }
                } else {
                    for (int k = 0; k < 4; ++k)
                        if (e0 + k < m) {
                            c[u][k] = src[e0 + k];
                            if (wsrc) wv[u][k] = wsrc[e0 + k];
                        }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t q = base + 32 * u + lane, e0 = q * 4;
            const bool inq = q < nq, full = e0 + 4 <= m;
            int32_t nxt = __shfl_down_sync(G2_FULL, c[u][0], 1);
            if (lane == 31 && inq && e0 + 4 < m) nxt = src[e0 + 4];
            if (!inq) continue;
            int code = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t e = e0 + k;
                if (e >= m) break;
                if (c[u][k] < 0 || c[u][k] >= n) code = 4;
                const int64_t f = e + 1;
                if (f < m) {
                    const bool start = (rowstart[f >> 5] >> (f & 31)) & 1u;
                    const int32_t cn = k < 3 ? c[u][k + 1] : nxt;
                    if (!start && cn <= c[u][k]) code = code ? code : 5;
                }
                if (wsrc && wv[u][k] < 0) code = code ? code : 6;
            }
            if (!dst) {
                // checks only
            } else if (full) {
                *reinterpret_cast<int4 *>(dst + e0) = make_int4(c[u][0], c[u][1], c[u][2], c[u][3]);
                if (wsrc)
                    *reinterpret_cast<int4 *>(wdst + e0) =
                        make_int4(wv[u][0], wv[u][1], wv[u][2], wv[u][3]);
            } else {
                for (int k = 0; k < 4; ++k)
                    if (e0 + k < m) {
                        dst[e0 + k] = c[u][k];
                        if (wsrc) wdst[e0 + k] = wv[u][k];
                    }
            }
            if (code) atomicExch(bad, code);
        }
    }
}

__global__ void k_coo_src(const int32_t *rowptr, int32_t n, int32_t *src) {
    // warp per vertex so long lists are written cooperatively
    int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = gw; u < n; u += nw) {
        int32_t b = rowptr[u], e = rowptr[u + 1];
        for (int32_t k = b + lane; k < e; k += 32) src[k] = (int32_t)u;
    }
}

// --- scan: tiles of kScanTile items
constexpr int kScanPer = 8;
constexpr int kScanTile = kCta * kScanPer;

__global__ void __launch_bounds__(kCta) k_scan_tile_sums(const int32_t *in, int32_t count,
                                                         int32_t *partial) {
    int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
    for (int j = 0; j < kScanPer; ++j) {
        int64_t i = t0 + (int64_t)j * kCta + threadIdx.x;
        if (i < count) s += in[i];
    }
    __shared__ int s_warp[kWarps];
    int total;
    block_incl_scan(s, s_warp, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kCta) k_scan_partials(int32_t *partial, int32_t ntiles) {
    __shared__ int s_warp[kWarps];
    int carry = 0;
    for (int32_t b = 0; b < ntiles; b += kCta) {
        int32_t i = b + threadIdx.x;
        int x = i < ntiles ? partial[i] : 0;
        int total;
        int incl = block_incl_scan(x, s_warp, &total);
        if (i < ntiles) partial[i] = carry + incl - x;  // exclusive
        carry += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCta) k_scan_apply(const int32_t *in, int32_t count,
                                                     const int32_t *partial, int32_t *out) {
    // each thread scans kScanPer consecutive items
    __shared__ int s_warp[kWarps];
    int64_t t0 = (int64_t)blockIdx.x * kScanTile;
    int64_t i0 = t0 + (int64_t)threadIdx.x * kScanPer;
    int vals[kScanPer];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        vals[j] = (i0 + j < count) ? in[i0 + j] : 0;
        s += vals[j];
    }
    int total;
    int incl = block_incl_scan(s, s_warp, &total);
    int run = partial[blockIdx.x] + incl - s;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        if (i0 + j < count) out[i0 + j] = run;
        run += vals[j];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kCta - 1) out[count] = run;
}

// --- vertexset conversions
__global__ void k_list_to_bitmap(const int32_t *q, int32_t size, uint32_t *bm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < size;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = q[i];
        atomicOr(&bm[v >> 5], 1u << (v & 31));
    }
}
__global__ void k_list_to_boolmap(const int32_t *q, int32_t size, uint8_t *b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < size;
         i += (int64_t)gridDim.x * blockDim.x)
        b[q[i]] = 1;
}
__global__ void k_bitmap_to_list(const uint32_t *bm, int32_t nwords, int32_t *q, int32_t *cnt,
                                 int32_t cap, int32_t *err) {
    int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < nwords;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + lane;
        uint32_t w = i < nwords ? bm[i] : 0u;
        int c = __popc(w);
        int incl = warp_incl_scan(c);
        int tot = __shfl_sync(G2_FULL, incl, 31);
        int b = 0;
        if (lane == 31 && tot) b = atomicAdd(cnt, tot);
        b = __shfl_sync(G2_FULL, b, 31);
        int pos = b + incl - c;
        while (w) {
            int bit = __ffs(w) - 1;
            w &= w - 1;
            if (pos < cap) q[pos] = (int32_t)(i * 32 + bit);
            else set_error(err, G2_EOVERFLOW);
            ++pos;
        }
    }
}
__global__ void k_boolmap_to_list(const uint8_t *b, int32_t n, int32_t *q, int32_t *cnt,
                                  int32_t cap, int32_t *err) {
    int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = base + lane;
        bool p = v < n && b[v];
        warp_append(q, cnt, cap, err, (int32_t)v, p);
    }
}
__global__ void k_bitmap_to_boolmap(const uint32_t *bm, int32_t n, uint8_t *b) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        b[v] = (bm[v >> 5] >> (v & 31)) & 1u;
}
__global__ void k_boolmap_to_bitmap(const uint8_t *b, int32_t n, uint32_t *bm) {
    int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = base + lane;
        unsigned m = __ballot_sync(G2_FULL, v < n && b[v]);
        if (lane == 0) bm[base >> 5] = m;
    }
}
__global__ void k_count_bitmap(const uint32_t *bm, int32_t nwords, int32_t *out) {
    int c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
         i += (int64_t)gridDim.x * blockDim.x)
        c += __popc(bm[i]);
    unsigned s = __reduce_add_sync(G2_FULL, (unsigned)c);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, (int)s);
}
__global__ void k_count_boolmap(const uint8_t *b, int32_t n, int32_t *out) {
    int c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        c += b[v] != 0;
    unsigned s = __reduce_add_sync(G2_FULL, (unsigned)c);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, (int)s);
}

// --- EdgeBlocking (Algorithm 1) on the device.  For vertex u and segment s
// the arcs of u with destination in segment s are one contiguous run of u's
// ascending list; cnt[s*n+u] is its length and beg[s*n+u] its first CSR
// position.  An exclusive scan of cnt in segment-major order gives every
// run's place in the blocked array, which is therefore the stable counting
// sort by segment that Algorithm 1 produces.
__global__ void k_eb_runs(const int32_t *rowptr, const int32_t *col, int32_t n, int32_t N,
                          int32_t nseg, int32_t *cnt, int32_t *beg) {
    int64_t total = (int64_t)n * nseg;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = (int32_t)(p / n), u = (int32_t)(p % n);
        int32_t b = rowptr[u], e = rowptr[u + 1];
        int64_t lo_key = (int64_t)s * N, hi_key = lo_key + N;
        int32_t lo = b, hi = e;  // first arc with col >= lo_key
        while (lo < hi) {
            int32_t mid = (lo + hi) >> 1;
            if (col[mid] < lo_key) lo = mid + 1;
            else hi = mid;
        }
        int32_t a = lo;
        hi = e;
        while (lo < hi) {
            int32_t mid = (lo + hi) >> 1;
            if (col[mid] < hi_key) lo = mid + 1;
            else hi = mid;
        }
        cnt[p] = lo - a;
        beg[p] = a;
    }
}

__global__ void k_eb_scatter(const int32_t *coo_src, const int32_t *col, int32_t m, int32_t n,
                             int32_t N, const int32_t *off, const int32_t *beg, int32_t *out_src,
                             int32_t *out_dst) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t u = coo_src[e], v = col[e];
        int64_t p = (int64_t)(v / N) * n + u;
        int32_t pos = off[p] + (int32_t)(e - beg[p]);
        out_src[pos] = u;
        out_dst[pos] = v;
    }
}

__global__ void k_eb_seg_end(const int32_t *off, int32_t n, int32_t nseg, int32_t m,
                             int64_t *seg_end) {
    int32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nseg) seg_end[s] = off[(int64_t)(s + 1) * n];
    if (s == nseg) seg_end[s] = m;
}

__global__ void k_wait_flag(const unsigned *flag, uint64_t limit_ns, int32_t *err) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (!bounded_wait_flag(flag, limit_ns)) set_error(err, G2_ETIMEOUT);
    }
}

// ================================================================ host helpers
int grid_for(const g2_graph *g, int64_t items, int items_per_cta) {
    int64_t b = (items + items_per_cta - 1) / items_per_cta;
    int64_t cap = (int64_t)g->topo->sm_count * 32;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices];
int g_pool_state[kMaxDevices];  // 0 unknown, 1 pool, 2 no pool support

// pool of the current device, or nullptr where pools are unsupported
cudaMemPool_t current_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_state[dev] == 0) {
        int ok = 0;
        cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, dev);
        cudaMemPool_t pool = nullptr;
        if (ok) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) pool = nullptr;
        }
        if (pool) {
            uint64_t keep = UINT64_MAX;  // never hand freed blocks back to the driver
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            g_pool[dev] = pool;
            g_pool_state[dev] = 1;
        } else {
            cudaGetLastError();
            g_pool_state[dev] = 2;
        }
    }
    return g_pool_state[dev] == 1 ? g_pool[dev] : nullptr;
}
}  // namespace

cudaError_t dmalloc_bytes(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes < 16) bytes = 16;
    cudaMemPool_t pool = current_pool();
    if (!pool) return cudaMalloc(p, bytes);
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void dfree(void *p, cudaStream_t st) {
    if (!p) return;
    if (!current_pool()) {
        cudaFree(p);
        return;
    }
    cudaFreeAsync(p, st);
}

g2_status ws_get(g2_graph *g, Buf b, size_t bytes, void **out) {
    if (bytes == 0) bytes = 16;
    if (g->cap[b] < bytes) {
        // the old block may still be read by work queued on g->st: its
        // release is ordered after that work
        if (g->buf[b]) dfree(g->buf[b], g->st);
        g->buf[b] = nullptr;
        g->cap[b] = 0;
        void *p = nullptr;
        cudaError_t e = dmalloc_bytes(&p, bytes, g->st);
        if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
        g->buf[b] = p;
        g->cap[b] = bytes;
    }
    *out = g->buf[b];
    return G2_OK;
}

g2_status sync_and_check(g2_graph *g, cudaStream_t st, int32_t *d_err) {
    G2_CK(cudaGetLastError());
    if (d_err) {
        G2_CK(cudaMemcpyAsync(g->h_ctr + 63, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    }
    G2_CK(cudaStreamSynchronize(st));
    if (d_err && g->h_ctr[63] != 0) {
        int code = g->h_ctr[63];
        const char *what = code == G2_ETIMEOUT ? "device-side wait timed out"
                           : code == G2_EOVERFLOW ? "queue or value overflow on the device"
                                                  : "device error";
        return fail((g2_status)code, what);
    }
    return G2_OK;
}

g2_status begin_call(g2_graph *g, cudaStream_t st, int32_t **d_err) {
    stats() = g2_stats{};
    g->st = st;
    int32_t *ctrs;
    G2_TRY(ws(g, B_CTR, 64, &ctrs));
    G2_CK(cudaMemsetAsync(ctrs, 0, 64 * sizeof(int32_t), st));
    if (count_arcs_enabled()) {
        unsigned long long *a;
        G2_TRY(ws(g, B_ARCS, 2, &a));
        G2_CK(cudaMemsetAsync(a, 0, 8, st));
    }
    *d_err = ctrs + 62;
    return G2_OK;
}

g2_status end_call(g2_graph *g, cudaStream_t st, int32_t *d_err) {
    G2_TRY(sync_and_check(g, st, d_err));
    ktime_resolve();
    if (count_arcs_enabled()) {
        unsigned long long *a;
        G2_TRY(ws(g, B_ARCS, 2, &a));
        unsigned long long h = 0;
        G2_CK(cudaMemcpy(&h, a, 8, cudaMemcpyDeviceToHost));
        stats().arcs_examined = (int64_t)h;
    }
    return G2_OK;
}

g2_status read_counters(g2_graph *g, const int32_t *d, int count, cudaStream_t st, int32_t *d_err) {
    G2_CK(cudaMemcpyAsync(g->h_ctr, d, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    return sync_and_check(g, st, d_err);
}

struct PutArgs {
    int32_t *dst[kPutMax];
    int32_t val[kPutMax];
};
struct PutArrayArgs {
    int32_t *dst;
    int32_t count;
    int32_t val[kPutArrayMax];
};
__global__ void k_put(PutArgs a) {
    const int i = threadIdx.x;
    if (i < kPutMax && a.dst[i]) *a.dst[i] = a.val[i];
}
__global__ void k_put_array(PutArrayArgs a) {
    for (int i = threadIdx.x; i < a.count; i += blockDim.x) a.dst[i] = a.val[i];
}

g2_status put_i32(cudaStream_t st, std::initializer_list<PutItem> items) {
    if (items.size() > (size_t)kPutMax) return fail(G2_EINVAL, "too many values for put_i32");
    PutArgs a;
    memset(&a, 0, sizeof(a));
    int i = 0;
    for (const PutItem &it : items) {
        a.dst[i] = it.dst;
        a.val[i] = it.val;
        ++i;
    }
    k_put<<<1, 32, 0, st>>>(a);
    G2_CK(cudaGetLastError());
    return G2_OK;
}

g2_status put_array(int32_t *dst, const int32_t *src, int count, cudaStream_t st) {
    if (count < 0 || count > kPutArrayMax) return fail(G2_EINVAL, "too many values for put_array");
    if (count == 0) return G2_OK;
    PutArrayArgs a;
    a.dst = dst;
    a.count = count;
    memcpy(a.val, src, (size_t)count * 4);
    k_put_array<<<1, 256, 0, st>>>(a);
    G2_CK(cudaGetLastError());
    return G2_OK;
}

g2_status exclusive_scan_i32(g2_graph *g, const int32_t *in, int32_t *out, int32_t count,
                             cudaStream_t st) {
    int32_t ntiles = (int32_t)((count + (int64_t)kScanTile - 1) / kScanTile);
    if (ntiles < 1) ntiles = 1;
    int32_t *partial;
    G2_TRY(ws(g, B_SCANTMP, (size_t)ntiles, &partial));
    k_scan_tile_sums<<<ntiles, kCta, 0, st>>>(in, count, partial);
    k_scan_partials<<<1, kCta, 0, st>>>(partial, ntiles);
    k_scan_apply<<<ntiles, kCta, 0, st>>>(in, count, partial, out);
    stats().launches += 3;
    G2_CK(cudaGetLastError());
    return G2_OK;
}

__global__ void k_max_degree(const int32_t *rowptr, int32_t n, int32_t *out) {
    int32_t best = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        best = max(best, rowptr[v + 1] - rowptr[v]);
    best = __reduce_max_sync(G2_FULL, best);
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(out, best);
}

g2_status max_out_degree(g2_graph *g, cudaStream_t st, int32_t *out) {
    Topology *t = g->topo;
    std::lock_guard<std::recursive_mutex> lk(t->layout_mu);
    if (t->max_out_deg < 0) {
        int32_t *d;
        G2_TRY(ws(g, B_CTR, 64, &d));
        G2_CK(cudaMemsetAsync(d + 48, 0, 4, st));
        if (t->n > 0) k_max_degree<<<grid_for(g, t->n, 256), 256, 0, st>>>(t->rowptr, t->n, d + 48);
        G2_CK(cudaMemcpyAsync(g->h_ctr + 48, d + 48, 4, cudaMemcpyDeviceToHost, st));
        G2_CK(cudaStreamSynchronize(st));
        t->max_out_deg = g->h_ctr[48];
    }
    *out = t->max_out_deg;
    return G2_OK;
}

g2_status ensure_coo(g2_graph *g, cudaStream_t st) {
    Topology *t = g->topo;
    std::lock_guard<std::recursive_mutex> lk(t->layout_mu);
    if (t->coo_src || t->m == 0) return G2_OK;
    G2_CK(dmalloc(&t->coo_src, (size_t)t->m * sizeof(int32_t), st));
    k_coo_src<<<grid_for(g, (int64_t)t->n * 32, kCta), kCta, 0, st>>>(t->rowptr, t->n, t->coo_src);
    G2_CK(cudaGetLastError());
    return G2_OK;
}

int32_t default_block_size(const g2_graph *g, int bytes_per_vertex) {
    // half of L2 for the destination range of one segment
    int64_t N = g->topo->l2_bytes / 2 / (bytes_per_vertex > 0 ? bytes_per_vertex : 4);
    if (N < 1024) N = 1024;
    if (N > g->topo->n) N = g->topo->n > 0 ? g->topo->n : 1;
    return (int32_t)N;
}

g2_status ensure_edge_block(g2_graph *g, int32_t N, cudaStream_t st) {
    Topology *t = g->topo;
    std::lock_guard<std::recursive_mutex> lk(t->layout_mu);
    if (N <= 0) N = default_block_size(g, 4);
    if (t->eb_src && t->eb_N == N) return G2_OK;
    int32_t n = t->n, m = t->m;
    int64_t nseg = n > 0 ? ((int64_t)n + N - 1) / N : 0;
    if (nseg * (int64_t)n >= 2147483647LL)
        return fail(G2_EUNSUPPORTED, "EdgeBlocking: segments x vertices must stay below 2^31");
    if (t->eb_src) {
        dfree(t->eb_src, st); dfree(t->eb_dst, st); dfree(t->eb_seg, st);
        delete[] t->h_eb_seg;
        t->eb_src = t->eb_dst = nullptr; t->eb_seg = nullptr; t->h_eb_seg = nullptr;
    }
    G2_TRY(ensure_coo(g, st));
    int64_t runs = nseg * n;
    int32_t *cnt = nullptr, *off = nullptr, *beg = nullptr;
    G2_CK(dmalloc(&t->eb_src, (size_t)std::max<int64_t>(m, 1) * 4, st));
    G2_CK(dmalloc(&t->eb_dst, (size_t)std::max<int64_t>(m, 1) * 4, st));
    G2_CK(dmalloc(&t->eb_seg, (size_t)(nseg + 1) * 8, st));
    G2_CK(dmalloc(&cnt, (size_t)(runs + 1) * 4, st));
    G2_CK(dmalloc(&off, (size_t)(runs + 1) * 4, st));
    G2_CK(dmalloc(&beg, (size_t)(runs + 1) * 4, st));
    if (runs > 0) {
        k_eb_runs<<<grid_for(g, runs, kCta), kCta, 0, st>>>(t->rowptr, t->col, n, N, (int32_t)nseg,
                                                            cnt, beg);
        G2_TRY(exclusive_scan_i32(g, cnt, off, (int32_t)runs, st));
        if (m > 0)
            k_eb_scatter<<<grid_for(g, m, kCta), kCta, 0, st>>>(t->coo_src, t->col, m, n, N, off,
                                                                beg, t->eb_src, t->eb_dst);
    }
    k_eb_seg_end<<<(int)((nseg + 1 + kCta - 1) / kCta), kCta, 0, st>>>(off, n, (int32_t)nseg, m,
                                                                       t->eb_seg);
    G2_CK(cudaGetLastError());
    t->h_eb_seg = new int64_t[nseg + 1];
    G2_CK(cudaMemcpyAsync(t->h_eb_seg, t->eb_seg, (size_t)(nseg + 1) * 8, cudaMemcpyDeviceToHost,
                          st));
    G2_CK(cudaStreamSynchronize(st));
    dfree(cnt, st); dfree(off, st); dfree(beg, st);
    t->eb_N = N;
    t->eb_nseg = (int32_t)nseg;
    return G2_OK;
}

// ------------------------------------------------------------- conversions
g2_status vset_convert(g2_graph *g, const VSet &src, int rep, VSet &dst, cudaStream_t st) {
    const int32_t n = g->topo->n;
    const int32_t nwords = (n + 31) / 32;
    if (src.rep == rep) {
        dst = src;
        return G2_OK;
    }
    dst.rep = rep;
    dst.size = src.size;
    int grid_v = grid_for(g, n, kCta);
    if (rep == OUT_SPARSE) {
        G2_CK(cudaMemsetAsync(dst.cnt, 0, sizeof(int32_t), st));
        if (src.rep == OUT_BITMAP)
            k_bitmap_to_list<<<grid_for(g, nwords, kCta), kCta, 0, st>>>(src.bitmap, nwords, dst.q,
                                                                         dst.cnt, dst.qcap, nullptr);
        else if (src.rep == OUT_BOOLMAP)
            k_boolmap_to_list<<<grid_v, kCta, 0, st>>>(src.boolmap, n, dst.q, dst.cnt, dst.qcap,
                                                       nullptr);
        else
            return fail(G2_EINVAL, "vertexset conversion from all-vertices");
    } else if (rep == OUT_BITMAP) {
        if (src.rep == OUT_SPARSE) {
            G2_CK(cudaMemsetAsync(dst.bitmap, 0, (size_t)nwords * 4, st));
            if (src.size > 0)
                k_list_to_bitmap<<<grid_for(g, src.size, kCta), kCta, 0, st>>>(src.q, src.size,
                                                                               dst.bitmap);
        } else if (src.rep == OUT_BOOLMAP) {
            k_boolmap_to_bitmap<<<grid_v, kCta, 0, st>>>(src.boolmap, n, dst.bitmap);
        } else {
            return fail(G2_EINVAL, "vertexset conversion from all-vertices");
        }
    } else if (rep == OUT_BOOLMAP) {
        if (src.rep == OUT_SPARSE) {
            G2_CK(cudaMemsetAsync(dst.boolmap, 0, (size_t)n, st));
            if (src.size > 0)
                k_list_to_boolmap<<<grid_for(g, src.size, kCta), kCta, 0, st>>>(src.q, src.size,
                                                                                dst.boolmap);
        } else if (src.rep == OUT_BITMAP) {
            k_bitmap_to_boolmap<<<grid_v, kCta, 0, st>>>(src.bitmap, n, dst.boolmap);
        } else {
            return fail(G2_EINVAL, "vertexset conversion from all-vertices");
        }
    } else {
        return fail(G2_EINVAL, "bad vertexset representation");
    }
    stats().launches += 1;
    G2_CK(cudaGetLastError());
    return G2_OK;
}

g2_status vset_count(g2_graph *g, const VSet &v, int32_t *d_out, cudaStream_t st) {
    const int32_t n = g->topo->n;
    G2_CK(cudaMemsetAsync(d_out, 0, sizeof(int32_t), st));
    if (v.rep == OUT_BITMAP)
        k_count_bitmap<<<grid_for(g, (n + 31) / 32, kCta), kCta, 0, st>>>(v.bitmap, (n + 31) / 32,
                                                                          d_out);
    else if (v.rep == OUT_BOOLMAP)
        k_count_boolmap<<<grid_for(g, n, kCta), kCta, 0, st>>>(v.boolmap, n, d_out);
    else
        return fail(G2_EINVAL, "count of a list vertexset");
    stats().launches += 1;
    G2_CK(cudaGetLastError());
    return G2_OK;
}

static void topo_release(Topology *t) {
    if (!t) return;
    if (--t->refs > 0) return;
    pr_prepare_wait(t);  // a background preparation still running finishes first
    // every call on the topology has returned (calls synchronise their
    // stream before returning), so the blocks are idle: release them to the pool
    void *blocks[] = {t->rowptr, t->col, t->w, t->symmetric ? nullptr : t->crowptr,
                      t->symmetric ? nullptr : t->ccol, t->symmetric ? nullptr : t->cw,
                      t->coo_src, t->eb_src, t->eb_dst, t->eb_seg, t->pr_slot_of, t->pr_ccol,
                      t->seg_head, t->seg_nzrow, t->seg_chunk_rank, t->blk_loc, t->blk_lane_heads,
                      t->blk_chunk_rank, t->blk_nzrow, t->blk_bchunk, t->blk_order, t->blk_deg,
                      t->blk_cta};
    for (void *b : blocks) dfree(b, nullptr);
    delete[] t->h_eb_seg;
    delete t;
}

static g2_graph *new_handle(Topology *t) {
    g2_graph *g = new g2_graph();
    g->topo = t;
    for (int i = 0; i < B_COUNT; ++i) { g->buf[i] = nullptr; g->cap[i] = 0; }
    g->h_ctr = nullptr;
    g->round = 0;
    g->round2 = 0;
    g->st = nullptr;
    return g;
}

// Pinned host counter blocks of freed handles are kept for the next handle
// (pinning and unpinning host memory are slow driver calls).
static std::mutex g_ctr_mu;
static std::vector<int32_t *> g_ctr_free;

static g2_status finish_handle(g2_graph *g) {
    {
        std::lock_guard<std::mutex> lk(g_ctr_mu);
        if (!g_ctr_free.empty()) {
            g->h_ctr = g_ctr_free.back();
            g_ctr_free.pop_back();
        }
    }
    if (!g->h_ctr) {
        cudaError_t e = cudaMallocHost(&g->h_ctr, 64 * sizeof(int32_t));
        if (e != cudaSuccess) {
            g->h_ctr = nullptr;
            return cuda_fail(e, "cudaMallocHost counters");
        }
    }
    memset(g->h_ctr, 0, 64 * sizeof(int32_t));
    return G2_OK;
}

// Host transpose (CSC with ascending lists) for non-symmetric graphs.
static void host_transpose(int32_t n, int32_t m, const int32_t *rp, const int32_t *cl,
                           const int32_t *w, std::vector<int32_t> &crp, std::vector<int32_t> &ccl,
                           std::vector<int32_t> &cw) {
    crp.assign((size_t)n + 1, 0);
    for (int32_t e = 0; e < m; ++e) crp[(size_t)cl[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) crp[(size_t)v + 1] += crp[v];
    std::vector<int32_t> pos(crp.begin(), crp.end() - 1);
    ccl.assign((size_t)std::max(m, 1), 0);
    if (w) cw.assign((size_t)std::max(m, 1), 0);
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = rp[u]; e < rp[u + 1]; ++e) {
            int32_t p = pos[cl[e]]++;
            ccl[p] = u;  // u ascending, so every list is ascending
            if (w) cw[p] = w[e];
        }
}

// A handle's own resources (workspace, counter block), not its topology.
static void handle_release(g2_graph *g) {
    // calls synchronise before returning, so the workspace is idle
    for (int i = 0; i < B_COUNT; ++i) dfree(g->buf[i], nullptr);
    if (g->h_ctr) {
        std::lock_guard<std::mutex> lk(g_ctr_mu);
        g_ctr_free.push_back(g->h_ctr);
    }
    delete g;
}

g2_status pr_prepare_start(g2_graph *g, cudaStream_t load_stream) {
    Topology *t = g->topo;
    std::lock_guard<std::mutex> lk(t->prep_mu);
    if (t->prep.joinable()) return G2_OK;
    g2_graph *h = new_handle(t);  // holds no reference: the topology joins it before it goes
    if (finish_handle(h) != G2_OK) {
        handle_release(h);
        return G2_ENOMEM;
    }
    // the preparation runs at the priority of the load's stream
    int prio = 0;
    if (cudaStreamGetPriority(load_stream, &prio) != cudaSuccess) {
        cudaGetLastError();
        prio = 0;
    }
    cudaStream_t s2 = nullptr;
    cudaError_t e = cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, prio);
    if (e != cudaSuccess) {
        handle_release(h);
        return cuda_fail(e, "stream for the background preparation");
    }
    t->prep_handle = h;
    t->prep_stream = s2;
    t->prep_status = G2_OK;
    const int dev = t->device;
    t->prep = std::thread([t, h, s2, dev]() {
        cudaSetDevice(dev);
        g2_status s = pr_build_layouts(h, s2);
        if (s == G2_OK && cudaStreamSynchronize(s2) != cudaSuccess) s = G2_ECUDA;
        if (s != G2_OK) t->prep_error = g2_last_error();
        t->prep_status = s;
    });
    return G2_OK;
}

g2_status pr_prepare_wait(Topology *t) {
    std::lock_guard<std::mutex> lk(t->prep_mu);
    if (!t->prep.joinable()) return G2_OK;
    t->prep.join();
    handle_release(t->prep_handle);
    t->prep_handle = nullptr;
    cudaStreamDestroy(t->prep_stream);
    t->prep_stream = nullptr;
    const g2_status s = t->prep_status;
    t->prep_status = G2_OK;
    if (s != G2_OK) return fail(s, "background PageRank preparation: " + t->prep_error);
    return G2_OK;
}

}  // namespace g2

using namespace g2;

// ============================================================== public C ABI
extern "C" {

const char *g2_last_error(void) { return t_err.c_str(); }
const char *g2_version(void) { return "g2 0.1 (sm_103a)"; }

g2_status g2_last_stats(g2_stats *out) {
    if (!out) return fail(G2_EINVAL, "null stats pointer");
    *out = t_stats;
    return G2_OK;
}
void g2_set_count_arcs(int32_t enable) { t_count_arcs = enable != 0; }

void g2_set_kernel_timing(int32_t enable) { t_ktime = enable != 0; }

g2_status g2_kernel_time(const char *name, double *ms, int64_t *launches, int32_t reset) {
    if (!name || !ms || !launches) return fail(G2_EINVAL, "null argument");
    *ms = 0.0;
    *launches = 0;
    for (const KTotal &x : t_ktotals)
        if (x.name == name) {
            *ms = x.ms;
            *launches = x.launches;
        }
    if (reset) t_ktotals.clear();
    return G2_OK;
}

// Address at which kernels may read the caller's array p, or nullptr when
// they cannot (then it is copied with cudaMemcpy): device memory (flag
// G2_DEVICE_PTRS), pinned host memory, or pageable host memory on a device
// that reads it through the host's page tables (the coherent link of a
// Grace-Blackwell system; no page migration).  16-byte alignment required.
static const int32_t *device_readable(const int32_t *p, bool dev, int device) {
    if (!p || (reinterpret_cast<uintptr_t>(p) & 15u)) return nullptr;
    if (dev) return p;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer &&
        !(reinterpret_cast<uintptr_t>(a.devicePointer) & 15u))
        return static_cast<const int32_t *>(a.devicePointer);
    if (a.type != cudaMemoryTypeUnregistered) return nullptr;
    int pageable = 0, host_tables = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
    cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device);
    return pageable && host_tables ? p : nullptr;
}

// Whether a copy engine reads p directly: device memory or pinned host
// memory (pageable memory goes through the driver's staging buffers, which
// holds up the other host threads' CUDA calls meanwhile).
static bool copy_engine_source(const void *p, bool dev) {
    if (!p || dev) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice ||
           a.type == cudaMemoryTypeManaged;
}

g2_status g2_load_csr(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *col,
                      const int32_t *w, uint32_t flags, void *stream, g2_graph **out) {
    if (!out) return fail(G2_EINVAL, "null output handle");
    *out = nullptr;
    if (n < 0 || n >= 2147483647 || m < 0 || m >= 2147483647LL)
        return fail(G2_EINVAL, "n or m out of range (must be < 2^31 - 1)");
    if (!rowptr || (m > 0 && !col)) return fail(G2_EINVAL, "null rowptr/col");
    if (flags & ~(G2_SYMMETRIC | G2_DEVICE_PTRS | G2_PREPARE_PAGERANK | G2_LOAD_OVERLAP))
        return fail(G2_EINVAL, "unknown flags");
    cudaStream_t st = as_stream(stream);
    const bool dev = flags & G2_DEVICE_PTRS;
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    Topology *t = new Topology();
    t->refs = 1;
    t->n = n;
    t->m = (int32_t)m;
    t->symmetric = flags & G2_SYMMETRIC;
    t->rowptr = t->col = t->w = t->crowptr = t->ccol = t->cw = t->coo_src = nullptr;
    t->eb_N = 0; t->eb_nseg = 0; t->eb_src = t->eb_dst = nullptr; t->eb_seg = nullptr;
    t->h_eb_seg = nullptr;
    t->max_out_deg = -1;
    t->pr_hot = -1; t->pr_hot_min_deg = 0; t->pr_slot_of = t->pr_ccol = nullptr;
    t->seg_head = nullptr; t->seg_nzrow = t->seg_chunk_rank = nullptr; t->seg_nnzrow = 0;
    t->blk_S = 0; t->blk_nb = 0; t->blk_nchunks = 0; t->blk_nruns = 0; t->blk_nact = 0;
    t->blk_loc = nullptr; t->blk_lane_heads = nullptr;
    t->blk_chunk_rank = t->blk_nzrow = t->blk_bchunk = t->blk_order = t->blk_deg = nullptr;
    t->blk_cta = nullptr; t->blk_G = 0;
    g2_graph *g = new_handle(t);
    auto bail = [&](g2_status s) { g2_free_graph(g); return s; };
    cudaError_t e;
    if ((e = cudaGetDevice(&t->device)) != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
    // three attribute queries (the full property query costs milliseconds)
    int sms = 0, l2 = 0, optin = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, t->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, t->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, t->device)) !=
            cudaSuccess)
        return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
    t->sm_count = sms;
    t->l2_bytes = l2;
    t->smem_optin = optin;
    t->max_coop_blocks = 0;
    if (finish_handle(g) != G2_OK) return bail(G2_ENOMEM);
    // every array carries kPad spare elements (zeroed) so that a 16-byte
    // rounded bulk copy of a slice ending at the last element stays in bounds
    size_t mb = ((size_t)std::max<int64_t>(m, 1) + kPad) * 4;
    size_t rb = ((size_t)n + 1 + kPad) * 4;
    if ((e = dmalloc(&t->rowptr, rb, st)) != cudaSuccess)
        return bail(cuda_fail(e, "allocation of rowptr"));
    if ((e = dmalloc(&t->col, mb, st)) != cudaSuccess) return bail(cuda_fail(e, "allocation of col"));
    if (w && (e = dmalloc(&t->w, mb, st)) != cudaSuccess) return bail(cuda_fail(e, "allocation of w"));
    // zero the padding past the copied elements (the copies below fill the rest)
    const size_t mcopy = (size_t)m * 4, rcopy = ((size_t)n + 1) * 4;
    cudaMemsetAsync(reinterpret_cast<char *>(t->rowptr) + rcopy, 0, rb - rcopy, st);
    cudaMemsetAsync(reinterpret_cast<char *>(t->col) + mcopy, 0, mb - mcopy, st);
    if (w) cudaMemsetAsync(reinterpret_cast<char *>(t->w) + mcopy, 0, mb - mcopy, st);
    if ((e = cudaMemcpyAsync(t->rowptr, rowptr, ((size_t)n + 1) * 4, kind, st)) != cudaSuccess)
        return bail(cuda_fail(e, "copy rowptr"));
    // the arcs are read by the validating copy kernel itself where the device
    // can address the caller's arrays; otherwise copied, then validated.  A
    // load that overlaps other work moves pinned or device arrays with a copy
    // engine and validates them in one pass afterwards: the copy kernel would
    // hold SMs for the whole transfer, and a kernel that needs whole SMs
    // (PageRank's sweep, one 1024-thread CTA per SM) would wait for them
    // (measured on RMAT-22: 7.1-7.4 ms per pipelined load + step against
    // 7.6-7.7 ms).  Pageable arrays in such a load keep the copy kernel, on a
    // quarter of the SMs with deeper reads per thread.
    const bool overlap = flags & G2_LOAD_OVERLAP;
    const int32_t *col_rd = m > 0 ? device_readable(col, dev, t->device) : nullptr;
    const int32_t *w_rd = (w && m > 0) ? device_readable(w, dev, t->device) : nullptr;
    const bool engine = overlap && copy_engine_source(col, dev) && copy_engine_source(w, dev);
    const bool fused_copy = col_rd && (!w || w_rd) && !engine;
    if (!fused_copy) {
        if (m > 0 && (e = cudaMemcpyAsync(t->col, col, (size_t)m * 4, kind, st)) != cudaSuccess)
            return bail(cuda_fail(e, "copy col"));
        if (w && m > 0 && (e = cudaMemcpyAsync(t->w, w, (size_t)m * 4, kind, st)) != cudaSuccess)
            return bail(cuda_fail(e, "copy w"));
    }
    // validation on the device
    {
        uint32_t *rowstart = nullptr;
        int32_t *bad = nullptr;
        size_t words = ((size_t)std::max<int64_t>(m, 1) + 31) / 32;
        if ((e = dmalloc(&rowstart, words * 4, st)) != cudaSuccess)
            return bail(cuda_fail(e, "allocation for validation"));
        if ((e = dmalloc(&bad, 4, st)) != cudaSuccess) {
            dfree(rowstart, st);
            return bail(cuda_fail(e, "allocation for validation"));
        }
        cudaMemsetAsync(rowstart, 0, words * 4, st);
        cudaMemsetAsync(bad, 0, 4, st);
        k_validate_rows<<<(int)((n + 1 + 255) / 256), 256, 0, st>>>(t->rowptr, n, (int32_t)m,
                                                                   rowstart, bad);
        if (m > 0 && fused_copy && overlap)
            k_load_cols<4><<<std::max(1, t->sm_count / 4), 256, 0, st>>>(
                col_rd, w_rd, t->col, t->w, n, (int32_t)m, rowstart, bad);
        else if (m > 0 && fused_copy)
            k_load_cols<1><<<t->sm_count * 8, 256, 0, st>>>(col_rd, w_rd, t->col, t->w, n,
                                                            (int32_t)m, rowstart, bad);
        else if (m > 0)  // copied above: check the device copy, 16-byte reads
            k_load_cols<2><<<t->sm_count * 8, 256, 0, st>>>(t->col, t->w, nullptr, nullptr, n,
                                                            (int32_t)m, rowstart, bad);
        // into the handle's pinned counters: a copy to pageable memory would
        // block inside the driver until the upload ends, stalling the CUDA
        // calls of other host threads meanwhile
        g->h_ctr[60] = 0;
        cudaMemcpyAsync(g->h_ctr + 60, bad, 4, cudaMemcpyDeviceToHost, st);
        e = cudaStreamSynchronize(st);
        const int32_t hbad = g->h_ctr[60];
        dfree(rowstart, st);
        dfree(bad, st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "graph validation"));
        if (hbad) {
            static const char *why[] = {"", "rowptr[0] != 0", "rowptr[n] != m",
                                        "rowptr not monotone / out of range", "arc id out of range",
                                        "adjacency list not strictly ascending",
                                        "negative weight"};
            return bail(fail(G2_EINVAL, std::string("invalid CSR: ") + why[hbad]));
        }
    }
    if (t->symmetric) {
        t->crowptr = t->rowptr;
        t->ccol = t->col;
        t->cw = t->w;
    } else {
        // transpose on the host (one-time load step)
        std::vector<int32_t> hrp((size_t)n + 1), hcl((size_t)std::max<int64_t>(m, 1)), hw;
        if (w) hw.resize((size_t)std::max<int64_t>(m, 1));
        cudaMemcpyAsync(hrp.data(), t->rowptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, st);
        if (m > 0) cudaMemcpyAsync(hcl.data(), t->col, (size_t)m * 4, cudaMemcpyDeviceToHost, st);
        if (w && m > 0) cudaMemcpyAsync(hw.data(), t->w, (size_t)m * 4, cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(e, "CSR download"));
        std::vector<int32_t> crp, ccl, cw;
        host_transpose(n, (int32_t)m, hrp.data(), hcl.data(), w ? hw.data() : nullptr, crp, ccl, cw);
        if ((e = dmalloc(&t->crowptr, rb, st)) != cudaSuccess ||
            (e = dmalloc(&t->ccol, mb, st)) != cudaSuccess ||
            (w && (e = dmalloc(&t->cw, mb, st)) != cudaSuccess))
            return bail(cuda_fail(e, "allocation of the CSC"));
        cudaMemsetAsync(t->crowptr, 0, rb, st);
        cudaMemsetAsync(t->ccol, 0, mb, st);
        if (w) cudaMemsetAsync(t->cw, 0, mb, st);
        cudaMemcpyAsync(t->crowptr, crp.data(), ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, st);
        if (m > 0) cudaMemcpyAsync(t->ccol, ccl.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st);
        if (w && m > 0) cudaMemcpyAsync(t->cw, cw.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st);
        // the host vectors must outlive the copies
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(e, "CSC upload"));
    }
    if (flags & G2_PREPARE_PAGERANK) {
        const g2_status ps = pr_prepare_start(g, st);
        if (ps != G2_OK) return bail(ps);
    }
    *out = g;
    return G2_OK;
}

void g2_free_graph(g2_graph *g) {
    if (!g) return;
    Topology *t = g->topo;
    handle_release(g);
    topo_release(t);
}


g2_status g2_graph_view(g2_graph *g, g2_graph **out) {
    if (!g || !out) return fail(G2_EINVAL, "null graph or output");
    g->topo->refs++;
    g2_graph *v = new_handle(g->topo);
    g2_status s = finish_handle(v);
    if (s != G2_OK) {
        g2_free_graph(v);
        return s;
    }
    *out = v;
    return G2_OK;
}

g2_status g2_graph_info(const g2_graph *g, int64_t *n, int64_t *m, int32_t *sm_count,
                        int64_t *l2_bytes) {
    if (!g) return fail(G2_EINVAL, "null graph");
    if (n) *n = g->topo->n;
    if (m) *m = g->topo->m;
    if (sm_count) *sm_count = g->topo->sm_count;
    if (l2_bytes) *l2_bytes = g->topo->l2_bytes;
    return G2_OK;
}

g2_status g2_edge_block(g2_graph *g, int32_t N, int32_t *num_segments, void *stream) {
    if (!g) return fail(G2_EINVAL, "null graph");
    cudaStream_t st = as_stream(stream);
    g->st = st;
    G2_TRY(ensure_edge_block(g, N, st));
    G2_CK(cudaStreamSynchronize(st));
    if (num_segments) *num_segments = g->topo->eb_nseg;
    return G2_OK;
}

g2_status g2_edge_block_export(g2_graph *g, int32_t *src, int32_t *dst, int64_t *seg_end,
                               void *stream) {
    if (!g || !src || !dst || !seg_end) return fail(G2_EINVAL, "null argument");
    Topology *t = g->topo;
    if (!t->eb_src) return fail(G2_EINVAL, "no EdgeBlocking layout built (call g2_edge_block)");
    cudaStream_t st = as_stream(stream);
    g->st = st;
    if (t->m > 0) {
        G2_CK(cudaMemcpyAsync(src, t->eb_src, (size_t)t->m * 4, cudaMemcpyDeviceToDevice, st));
        G2_CK(cudaMemcpyAsync(dst, t->eb_dst, (size_t)t->m * 4, cudaMemcpyDeviceToDevice, st));
    }
    G2_CK(cudaMemcpyAsync(seg_end, t->eb_seg, (size_t)(t->eb_nseg + 1) * 8,
                          cudaMemcpyDeviceToDevice, st));
    G2_CK(cudaStreamSynchronize(st));
    return G2_OK;
}

// ------------------------------------------------------------ frontier API
g2_status g2_frontier_create(g2_graph *g, int32_t format, g2_frontier **out) {
    if (!g || !out) return fail(G2_EINVAL, "null graph or output");
    if (format < G2_FRONTIER_SPARSE || format > G2_FRONTIER_BOOLMAP)
        return fail(G2_EINVAL, "bad frontier format");
    int32_t n = g->topo->n;
    g2_frontier *f = new g2_frontier();
    f->g = g;
    f->format = format;
    f->q = nullptr; f->cnt = nullptr; f->bitmap = nullptr; f->boolmap = nullptr;
    f->cap = 0;
    // allocated and cleared on the legacy stream, then synchronised, so that
    // the frontier is ready for a call on any stream
    cudaError_t e = dmalloc(&f->cnt, sizeof(int32_t), nullptr);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->cnt, 0, sizeof(int32_t), nullptr);
    if (e == cudaSuccess && format == G2_FRONTIER_SPARSE) {
        f->cap = std::max(n, 1);
        e = dmalloc(&f->q, (size_t)f->cap * 4, nullptr);
    } else if (e == cudaSuccess && format == G2_FRONTIER_BITMAP) {
        e = dmalloc(&f->bitmap, ((size_t)(n + 31) / 32 + 1) * 4, nullptr);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(f->bitmap, 0, ((size_t)(n + 31) / 32 + 1) * 4, nullptr);
    } else if (e == cudaSuccess) {
        e = dmalloc(&f->boolmap, (size_t)std::max(n, 1), nullptr);
        if (e == cudaSuccess) e = cudaMemsetAsync(f->boolmap, 0, (size_t)std::max(n, 1), nullptr);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        g2_frontier_free(f);
        return cuda_fail(e, "frontier allocation");
    }
    *out = f;
    return G2_OK;
}

void g2_frontier_free(g2_frontier *f) {
    if (!f) return;
    // calls synchronise before returning, so the frontier's blocks are idle
    dfree(f->q, nullptr);
    dfree(f->cnt, nullptr);
    dfree(f->bitmap, nullptr);
    dfree(f->boolmap, nullptr);
    delete f;
}

g2_status g2_frontier_set(g2_frontier *f, const int32_t *verts, int32_t k, void *stream) {
    if (!f || k < 0 || (k > 0 && !verts)) return fail(G2_EINVAL, "bad frontier_set arguments");
    g2_graph *g = f->g;
    int32_t n = g->topo->n;
    for (int32_t i = 0; i < k; ++i)
        if (verts[i] < 0 || verts[i] >= n) return fail(G2_EINVAL, "vertex id out of range");
    cudaStream_t st = as_stream(stream);
    g->st = st;
    int32_t *tmp;
    G2_TRY(ws(g, B_I1, (size_t)std::max(k, 1), &tmp));
    if (k > 0) G2_CK(cudaMemcpyAsync(tmp, verts, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    VSet src{OUT_SPARSE, tmp, k, nullptr, nullptr, nullptr, k};
    if (f->format == G2_FRONTIER_SPARSE) {
        if (k > f->cap) {
            dfree(f->q, st);
            f->q = nullptr;
            G2_CK(dmalloc(&f->q, (size_t)k * 4, st));
            f->cap = k;
        }
        if (k > 0) G2_CK(cudaMemcpyAsync(f->q, tmp, (size_t)k * 4, cudaMemcpyDeviceToDevice, st));
        G2_TRY(put_i32(st, {{f->cnt, src.size}}));
    } else {
        VSet dst{f->format == G2_FRONTIER_BITMAP ? (int)OUT_BITMAP : (int)OUT_BOOLMAP, nullptr, 0,
                 nullptr, f->bitmap, f->boolmap, 0};
        G2_TRY(vset_convert(g, src, dst.rep, dst, st));
    }
    return sync_and_check(g, st, nullptr);
}

g2_status g2_frontier_size(g2_frontier *f, int32_t *size, void *stream) {
    if (!f || !size) return fail(G2_EINVAL, "null argument");
    g2_graph *g = f->g;
    cudaStream_t st = as_stream(stream);
    g->st = st;
    if (f->format == G2_FRONTIER_SPARSE) {
        G2_CK(cudaMemcpyAsync(g->h_ctr, f->cnt, 4, cudaMemcpyDeviceToHost, st));
    } else {
        VSet v{f->format == G2_FRONTIER_BITMAP ? (int)OUT_BITMAP : (int)OUT_BOOLMAP, nullptr, 0,
               nullptr, f->bitmap, f->boolmap, 0};
        int32_t *d;
        G2_TRY(ws(g, B_CTR, 64, &d));
        G2_TRY(vset_count(g, v, d + 32, st));
        G2_CK(cudaMemcpyAsync(g->h_ctr, d + 32, 4, cudaMemcpyDeviceToHost, st));
    }
    G2_CK(cudaStreamSynchronize(st));
    *size = g->h_ctr[0];
    return G2_OK;
}

g2_status g2_frontier_list(g2_frontier *f, int32_t *verts, int32_t cap, int32_t *k, void *stream) {
    if (!f || !verts || !k || cap < 0) return fail(G2_EINVAL, "null argument");
    g2_graph *g = f->g;
    cudaStream_t st = as_stream(stream);
    g->st = st;
    int32_t size = 0;
    G2_TRY(g2_frontier_size(f, &size, stream));
    if (size > cap) return fail(G2_EOVERFLOW, "frontier larger than the output capacity");
    if (f->format == G2_FRONTIER_SPARSE) {
        if (size > 0)
            G2_CK(cudaMemcpyAsync(verts, f->q, (size_t)size * 4, cudaMemcpyDeviceToDevice, st));
    } else {
        int32_t *d;
        G2_TRY(ws(g, B_CTR, 64, &d));
        VSet src{f->format == G2_FRONTIER_BITMAP ? (int)OUT_BITMAP : (int)OUT_BOOLMAP, nullptr, 0,
                 nullptr, f->bitmap, f->boolmap, size};
        VSet dst{OUT_SPARSE, verts, cap, d + 33, nullptr, nullptr, 0};
        G2_TRY(vset_convert(g, src, OUT_SPARSE, dst, st));
    }
    *k = size;
    return sync_and_check(g, st, nullptr);
}

g2_status g2_selftest_wait_timeout(int64_t limit_ns, void *stream) {
    if (limit_ns <= 0 || limit_ns > 10000000000LL) return fail(G2_EINVAL, "limit out of range");
    cudaStream_t st = as_stream(stream);
    unsigned *flag = nullptr;
    int32_t *err = nullptr;
    G2_CK(dmalloc(&flag, 4, st));
    cudaError_t ea = dmalloc(&err, 4, st);
    if (ea != cudaSuccess) {
        dfree(flag, st);
        return cuda_fail(ea, "selftest allocation");
    }
    cudaMemsetAsync(flag, 0, 4, st);
    cudaMemsetAsync(err, 0, 4, st);
    k_wait_flag<<<1, 32, 0, st>>>(flag, (uint64_t)limit_ns, err);
    int32_t h = 0;
    cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    dfree(flag, st);
    dfree(err, st);
    if (e != cudaSuccess) return cuda_fail(e, "selftest");
    if (h == G2_ETIMEOUT) return fail(G2_ETIMEOUT, "bounded wait expired as expected");
    return G2_OK;
}

}  // extern "C"
