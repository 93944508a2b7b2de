// g2_noalloc.cu — a BFS entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// runtime which has reserved the device memory for its own pool (a fresh
// allocation would fail or bypass that pool's accounting), and latency-bound
// callers that cannot afford the implicit device synchronisation that
// allocating and freeing can cause.  g2_bfs_csr_static serves them: the
// caller passes the graph and the outputs in its own device memory, and the
// only scratch the traversal needs (two frontier queues, their counters, the
// grid-barrier words and the error word) lives in the fixed array below,
// which every GPU that loads this library holds until the process exits.
// (With CUDA's lazy module loading, the module that holds the array is loaded
// on a device at this file's first use there, the first call: that call
// reserves the array's device memory and may synchronise the device, so a
// caller that cannot afford it makes one call at set-up time.)
//
// The caller's CSR is never copied, so it is checked on the device before
// the traversal reads it (row offsets monotone within [0, m], rowptr[0] = 0,
// rowptr[n] = m, every column id in [0, n)): a bad graph returns G2_EINVAL
// instead of sending the traversal out of bounds.
//
// The traversal is the fused persistent BFS: one cooperative kernel runs the
// whole frontier loop, warp-mapped load balancing, with a time-bounded grid
// barrier between rounds.
#include <cuda_runtime.h>

#include <mutex>

#include "g2_host.h"
#include "g2_lb.cuh"

namespace g2 {
namespace {

// Largest graph the fixed scratch serves, and its layout (int32 words):
// [0..2] rotating queue lengths, [4] rounds, [8..9] grid-barrier words,
// [12] error word, then two queues of kStaticMaxN vertices each.
constexpr int32_t kStaticMaxN = 1 << 20;
constexpr int32_t kHdr = 64;
static __device__ __align__(256) int32_t g_scratch[kHdr + 2 * (int64_t)kStaticMaxN];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t *g_scratch_ptr[kMaxDevices];  // device address of g_scratch, per device

// Resolve (once per device, with that device current) the device address of
// the scratch array.  In host code `g_scratch` names a host-side stand-in,
// not device memory, so kernels must get this address instead.
g2_status scratch_address(int32_t **out) {
    int dev = 0;
    G2_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(G2_EUNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_ptr[dev] = static_cast<int32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return G2_OK;
}

// Every call starts from a cleared header (counters, barrier words, error),
// since the array keeps whatever the previous call left in it.
__global__ void k_static_init(int32_t *s, int32_t *depth, int32_t *parent, int32_t n, int32_t src) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        depth[v] = v == src ? 0 : -1;
        if (parent) parent[v] = v == src ? src : -1;
    }
    if (blockIdx.x == 0 && threadIdx.x < kHdr) s[threadIdx.x] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s[kHdr] = src;  // queue 0 holds the source
        s[0] = 1;
    }
}

// The caller's CSR: on any violation the error word becomes G2_EINVAL.
__global__ void k_static_check(const int32_t *rowptr, const int32_t *col, int32_t n, int64_t m,
                               int32_t *err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t v = i0; v <= n; v += stride) {
        const int64_t r = rowptr[v];
        if (r < 0 || r > m || (v == 0 && r != 0) || (v == n && r != m)) bad = true;
        else if (v < n && rowptr[v + 1] < r) bad = true;
    }
    for (int64_t e = i0; e < m; e += stride)
        if ((uint32_t)col[e] >= (uint32_t)n) bad = true;
    if (bad) atomicCAS(err, 0, (int32_t)G2_EINVAL);
}

struct StaticBfsArgs {
    DevGraph g;
    int32_t *depth;
    int32_t *parent;
    int32_t *s;
    uint64_t limit_ns;
};

__global__ void __launch_bounds__(kCta) k_static_bfs(StaticBfsArgs a) {
    int32_t *cnt = a.s;
    int32_t *err = a.s + 12;
    int32_t *q[2] = {a.s + kHdr, a.s + kHdr + kStaticMaxN};
    GridBarrier bar{reinterpret_cast<unsigned long long *>(a.s + 8)};
    OpBFS op{a.depth, a.parent};
    OutCtx out;
    memset(&out, 0, sizeof(out));
    out.mode = OUT_SPARSE;
    out.dedup = DD_NONE;  // the compare-and-swap on depth admits each vertex once
    out.cap = kStaticMaxN;
    out.err = err;
    // a graph the check rejected is not traversed (every CTA reads the word
    // the check kernel, which ran before, left)
    if (ld_relaxed_i32(err) != 0) return;
    int d = 0;
    for (;; ++d) {
        int32_t size = ld_relaxed_i32(cnt + d % 3);
        if (size == 0) break;
        FrontierIn fin{q[d & 1], size, nullptr};
        out.q = q[(d + 1) & 1];
        out.cnt = cnt + (d + 1) % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt[(d + 2) % 3] = 0;
        lb_warp(a.g, fin, size, op, out, blockIdx.x, gridDim.x, nullptr);
        if (!grid_sync(bar, err, a.limit_ns)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.s[4] = d;
}

}  // namespace
}  // namespace g2

using namespace g2;

extern "C" g2_status g2_bfs_csr_static(int32_t n, int64_t m, const int32_t *rowptr,
                                       const int32_t *col, int32_t src, int32_t *depth,
                                       int32_t *parent, void *stream) {
    if (n < 1 || n > kStaticMaxN)
        return fail(G2_EINVAL, "g2_bfs_csr_static: n must be in [1, 1048576] (the static scratch "
                               "holds two queues of 1048576 vertices)");
    if (m < 0 || m >= 2147483647LL) return fail(G2_EINVAL, "g2_bfs_csr_static: m out of range");
    if (!rowptr || (m > 0 && !col) || !depth) return fail(G2_EINVAL, "g2_bfs_csr_static: null pointer");
    if (src < 0 || src >= n) return fail(G2_EINVAL, "g2_bfs_csr_static: source out of range");
    cudaStream_t st = as_stream(stream);
    int32_t *s = nullptr;
    G2_TRY(scratch_address(&s));
    int dev = 0, sms = 0, per_sm = 0;
    G2_CK(cudaGetDevice(&dev));
    G2_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    G2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_static_bfs, kCta, 0));
    if (per_sm < 1) return fail(G2_EUNSUPPORTED, "g2_bfs_csr_static: kernel does not fit on an SM");
    int init_grid = (int)std::min<int64_t>((n + kCta - 1) / kCta, (int64_t)sms * 8);
    k_static_init<<<init_grid, kCta, 0, st>>>(s, depth, parent, n, src);
    const int check_grid = (int)std::min<int64_t>((std::max<int64_t>(m, n) + kCta - 1) / kCta,
                                                  (int64_t)sms * 8);
    k_static_check<<<check_grid, kCta, 0, st>>>(rowptr, col, n, m, s + 12);
    G2_CK(cudaGetLastError());
    StaticBfsArgs a;
    a.g.n = n;
    a.g.m = (int32_t)m;
    a.g.rowptr = rowptr;
    a.g.col = col;
    a.g.w = nullptr;
    a.g.crowptr = rowptr;
    a.g.ccol = col;
    a.g.cw = nullptr;
    a.depth = depth;
    a.parent = parent;
    a.s = s;
    a.limit_ns = 2000000000ULL;
    void *params[] = {&a};
    G2_CK(cudaLaunchCooperativeKernel((const void *)k_static_bfs, dim3(per_sm * sms), dim3(kCta),
                                      params, 0, st));
    // the header comes back to host stack memory (a pageable copy: nothing is
    // allocated for it, pinned memory included)
    int32_t hdr[16];
    G2_CK(cudaMemcpyAsync(hdr, s, sizeof(hdr), cudaMemcpyDeviceToHost, st));
    G2_CK(cudaStreamSynchronize(st));
    if (hdr[12] == G2_EINVAL)
        return fail(G2_EINVAL, "g2_bfs_csr_static: invalid CSR (row offsets or a column id out of range)");
    if (hdr[12] == G2_ETIMEOUT) return fail(G2_ETIMEOUT, "g2_bfs_csr_static: grid barrier timed out");
    if (hdr[12] != 0) return fail((g2_status)hdr[12], "g2_bfs_csr_static: device error");
    return G2_OK;
}
