// g2_host.h — host-side internals of libg2: the graph handle, its device
// workspace, error and statistics plumbing, and the internal launchers shared
// by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <initializer_list>
#include <mutex>
#include <thread>
#include <cstdlib>
#include <string>

#include "g2.h"
#include "g2_device.cuh"

namespace g2 {

// ------------------------------------------------------------ errors, stats
void set_error_msg(const std::string &msg);
g2_status fail(g2_status st, const std::string &msg);
g2_status cuda_fail(cudaError_t e, const char *what);
g2_stats &stats();           // thread-local stats of the current call
bool count_arcs_enabled();   // thread-local

#define G2_CK(call)                                          \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ::g2::cuda_fail(e_, #call); \
    } while (0)

#define G2_TRY(expr)                    \
    do {                                \
        g2_status s_ = (expr);          \
        if (s_ != G2_OK) return s_;     \
    } while (0)

// --------------------------------------------------------------- workspace
// Named device buffers owned by a graph handle, allocated on first use and
// reused by every later call (the frontier reuse the paper's liveness analysis
// enables, Sec. VI-A: no cudaMalloc/cudaFree inside the iteration loops).
enum Buf {
    B_Q0, B_Q1, B_Q2, B_Q3,        // sparse queues (capacity n, or m when dedup is off)
    B_BM0, B_BM1,                  // bitmaps
    B_BOOL0, B_BOOL1,              // boolmaps
    B_STAMP, B_STAMP2,             // monotonic-counter dedup stamps
    B_DDBM, B_DDBOOL,              // bitmap / boolmap dedup flags
    B_SCAN, B_SCANTMP,             // STRICT prefix sums, scan partials
    B_TWC_S, B_TWC_M, B_TWC_L,     // TWC buckets
    B_CTR,                         // small device counters (int32[64])
    B_ARCS,                        // 64-bit arc counter
    B_F0, B_F1, B_F2,              // float/int scratch arrays of n (PR, CC)
    B_D0, B_D1,                    // double arrays of n (BC)
    B_LVL,                         // BC level queue (int32[n])
    B_I0, B_I1,                    // int32 arrays of n
    B_BIG,                         // dedup-disabled overflow queue (capacity m + n)
    B_MS0, B_MS1, B_MS2,           // multi-source masks (uint64[n])
    B_COUNT
};

struct Topology;  // shared by views (reference counted)

}  // namespace g2

struct g2_graph {
    g2::Topology *topo;
    void *buf[g2::B_COUNT];
    size_t cap[g2::B_COUNT];
    int32_t *h_ctr;   // pinned host mirror of B_CTR
    int32_t round;    // monotonic-counter stamp (advances every apply round)
    int32_t round2;
    cudaStream_t st;  // stream of the call in progress (set at every entry)
};

struct g2_frontier {
    g2_graph *g;
    int32_t format;
    int32_t *q;       // SPARSE: list (capacity cap)
    int32_t cap;
    int32_t *cnt;     // device int32 length (SPARSE)
    uint32_t *bitmap; // BITMAP
    uint8_t *boolmap; // BOOLMAP
};

namespace g2 {

struct Topology {
    std::atomic<int> refs;
    // serialise the lazy layout builders (views on several threads share
    // the topology); recursive because one builder may call another.
    // PageRank's layouts have a lock of their own, so that building them in
    // the background does not hold up the other builders.
    std::recursive_mutex layout_mu;
    std::recursive_mutex pr_mu;
    // background preparation of PageRank's layouts (G2_PREPARE_PAGERANK):
    // a host thread driving a handle of its own (own workspace, no reference
    // on the topology) on a non-blocking stream
    std::mutex prep_mu;
    std::thread prep;
    g2_graph *prep_handle = nullptr;
    cudaStream_t prep_stream = nullptr;
    g2_status prep_status = G2_OK;
    std::string prep_error;
    int32_t n;
    int32_t m;
    bool symmetric;
    int device;
    int sm_count;
    int64_t l2_bytes;
    int32_t smem_optin;   // largest dynamic shared memory a CTA may opt into
    int max_coop_blocks;  // resident CTAs of kCta threads for the fused kernels
    int32_t *rowptr, *col, *w;     // CSR
    int32_t *crowptr, *ccol, *cw;  // CSC (== CSR pointers when symmetric)
    int32_t *coo_src;              // lazily built source of every CSR arc
    // EdgeBlocking (Algorithm 1) layout
    int32_t eb_N;
    int32_t eb_nseg;
    int32_t *eb_src, *eb_dst;
    int64_t *eb_seg;     // device [nseg+1]
    int64_t *h_eb_seg;   // host copy
    // PageRank share-cache layout: the share slot of every vertex, the least
    // out-degree of the cached vertices, the CSC column ids as share slots
    int32_t max_out_deg;  // largest out-degree (-1: not computed yet)
    int32_t pr_hot;
    int32_t pr_hot_min_deg;
    int32_t *pr_slot_of, *pr_ccol;
    // segmented-sweep layout: row-head flags per arc, rows with in-arcs in
    // order, head count before every 128-arc chunk
    uint32_t *seg_head;
    int32_t *seg_nzrow;
    int32_t *seg_chunk_rank;
    int32_t seg_nnzrow;
    // source-blocked sweep layout (g2_pr_blk.cu): sources per block (0 = not
    // built), blocks, 256-arc chunks, runs; per arc the source's rank within
    // its block; per lane of a chunk its head flags and the heads before it;
    // runs before every chunk; destination rank of every run; first chunk of
    // every block; vertex of every rank and its out-degree
    int32_t blk_S;
    int32_t blk_nb;
    int32_t blk_G;            // CTAs of the sweep (one per SM)
    int64_t blk_nchunks;
    int32_t blk_nruns;
    int32_t blk_nact;         // ranks with out-arcs (they come first)
    uint16_t *blk_loc;
    uint16_t *blk_lane_heads;
    int32_t *blk_chunk_rank, *blk_nzrow, *blk_bchunk, *blk_order, *blk_deg;
    int32_t *blk_cta;         // first chunk of every CTA of the sweep (blk_G + 1)
    DevGraph view() const {
        DevGraph d;
        d.n = n; d.m = m;
        d.rowptr = rowptr; d.col = col; d.w = w;
        d.crowptr = crowptr; d.ccol = ccol; d.cw = cw;
        return d;
    }
};

// ------------------------------------------------------------ device memory
// Every device allocation of the library comes from one stream-ordered pool
// per device whose release threshold is unlimited: freed blocks stay with the
// pool and later allocations reuse them without a driver round trip and
// without the device-wide synchronisation a cudaFree implies.  A graph that
// is loaded, queried and freed once per request pays for its memory once per
// process, not once per request.  (Devices without memory-pool support fall
// back to cudaMalloc/cudaFree.)
//  dmalloc: the block is ordered on `st` (null = legacy stream); other
//           streams may use it once the host has synchronised with `st`.
//  dfree:   the release is ordered after the work already queued on `st`;
//           the block must not be in use by work on any other stream.
cudaError_t dmalloc_bytes(void **p, size_t bytes, cudaStream_t st);
void dfree(void *p, cudaStream_t st);
template <class T>
inline cudaError_t dmalloc(T **p, size_t bytes, cudaStream_t st) {
    return dmalloc_bytes(reinterpret_cast<void **>(p), bytes, st);
}

// Device buffer of at least `bytes` bytes for slot b (grown if needed; old
// contents are NOT kept when it grows).  Allocation and release are ordered
// on g->st, the stream of the call in progress on this handle.
g2_status ws_get(g2_graph *g, Buf b, size_t bytes, void **out);
template <class T>
inline g2_status ws(g2_graph *g, Buf b, size_t count, T **out) {
    return ws_get(g, b, count * sizeof(T), reinterpret_cast<void **>(out));
}

// Stream helpers.
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
g2_status sync_and_check(g2_graph *g, cudaStream_t st, int32_t *d_err);
int grid_for(const g2_graph *g, int64_t items, int items_per_cta);

// Kernel timing: ktime_begin/ktime_end bracket one launch with CUDA events
// when timing is enabled (no-ops otherwise); durations are collected by
// end_call after the stream has synchronised.
struct KTime {
    const char *name;
    cudaEvent_t e0, e1;
};
void ktime_begin(KTime &k, const char *name, cudaStream_t st);
void ktime_end(KTime &k, cudaStream_t st);

// Start of a public call: reset the thread's stats, zero the device error
// word (returned in *d_err, B_CTR slot 62) and the arc counter.
g2_status begin_call(g2_graph *g, cudaStream_t st, int32_t **d_err);
// End of a public call: synchronise, report device errors, collect counters.
g2_status end_call(g2_graph *g, cudaStream_t st, int32_t *d_err);
// Read `count` device int32 counters into g->h_ctr (synchronises) and check
// the error word.
g2_status read_counters(g2_graph *g, const int32_t *d, int count, cudaStream_t st, int32_t *d_err);

// Small host values stored to device memory by a one-warp kernel that takes
// them as launch arguments: no copy reads host memory, so nothing waits for a
// pageable staging copy or for a copy engine busy with another call's
// transfer.  put_i32: up to kPutMax (address, value) pairs (null addresses
// skipped); put_array: count <= kPutArrayMax consecutive values.
constexpr int kPutMax = 8;
constexpr int kPutArrayMax = 256;
struct PutItem {
    int32_t *dst;
    int32_t val;
};
g2_status put_i32(cudaStream_t st, std::initializer_list<PutItem> items);
g2_status put_array(int32_t *dst, const int32_t *src, int count, cudaStream_t st);

// COO source array of the CSR arcs (built on first use).
g2_status ensure_coo(g2_graph *g, cudaStream_t st);
// EdgeBlocking layout for segment size N (Algorithm 1), built on the device.
g2_status ensure_edge_block(g2_graph *g, int32_t N, cudaStream_t st);
int32_t default_block_size(const g2_graph *g, int bytes_per_vertex);

// PageRank layouts for handle h, built on stream st (defined with PageRank).
g2_status pr_build_layouts(g2_graph *h, cudaStream_t st);
// Source-blocked PageRank (g2_pr_blk.cu): whether its layout applies with
// blocks of S sources, the layout itself, and `iters` rounds over it.
bool pr_blk_applies(const Topology *t, int32_t S);
g2_status ensure_blk_layout(g2_graph *g, int32_t S, cudaStream_t st);
g2_status pagerank_blk_run(g2_graph *g, float damping, int32_t iters, float *rank, int32_t S,
                           cudaStream_t st);
// Start the background preparation for g's topology / wait for it (joins the
// thread, releases its handle and stream; returns its status).
g2_status pr_prepare_start(g2_graph *g, cudaStream_t load_stream);
g2_status pr_prepare_wait(Topology *t);

// Largest out-degree of the graph (computed on the device once, then kept).
g2_status max_out_degree(g2_graph *g, cudaStream_t st, int32_t *out);
// Bounded-degree graphs (road networks, meshes: largest out-degree <= 32)
// run BFS, SSSP and BC with kernel fusion when the caller gives no schedule:
// their many small levels cost more in launches and host round trips than in
// arcs.
constexpr int32_t kBoundedDegree = 32;

// Time limit of one grid-barrier wait in the fused kernels (2 s;
// G2_BARRIER_TIMEOUT_NS overrides).
inline uint64_t barrier_limit_ns() {
    static uint64_t lim = 0;
    if (lim == 0) {
        const char *e = getenv("G2_BARRIER_TIMEOUT_NS");
        long long v = e ? atoll(e) : 0;
        lim = v > 0 ? (uint64_t)v : 2000000000ULL;
    }
    return lim;
}

// Cooperative launch of a fused kernel taking one argument struct: resident
// CTAs only (co-residency is what makes its grid barriers safe).
template <class K, class A>
inline g2_status launch_coop(g2_graph *g, K kernel, A &args, cudaStream_t st, int want = 0) {
    int per_sm = 0;
    G2_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kCta, 0));
    if (per_sm < 1) return fail(G2_EUNSUPPORTED, "fused kernel does not fit on an SM");
    // fewer resident CTAs make every grid barrier cheaper; the round's work
    // is spread over the virtual CTAs either way.  One CTA per SM measured
    // best on road grids (G2_FUSED_CTAS_PER_SM overrides for sweeps); a
    // caller whose rounds sweep every vertex asks for more (`want`).
    static int cap = -1;
    if (cap < 0) {
        const char *e = getenv("G2_FUSED_CTAS_PER_SM");
        cap = e ? atoi(e) : 1;
    }
    const int use = want > 0 ? want : cap;
    if (use > 0 && use < per_sm) per_sm = use;
    int grid = per_sm * g->topo->sm_count;
    void *params[] = {&args};
    G2_CK(cudaLaunchCooperativeKernel((const void *)kernel, dim3(grid), dim3(kCta), params, 0, st));
    stats().launches += 1;
    return G2_OK;
}

// Device-wide exclusive scan of int32 (out[0..count], out[count] = total).
g2_status exclusive_scan_i32(g2_graph *g, const int32_t *in, int32_t *out, int32_t count,
                             cudaStream_t st);

// ------------------------------------------------------------- frontiers
// Internal vertexset: which representation is live and its size (host copy,
// valid after the round that produced it).
struct VSet {
    int rep;           // OUT_SPARSE (list), OUT_BITMAP, OUT_BOOLMAP; or -1 = all vertices
    int32_t *q;        // list
    int32_t qcap;
    int32_t *cnt;      // device length of the list
    uint32_t *bitmap;
    uint8_t *boolmap;
    int32_t size;      // host-known size
};

// Convert a vertexset to the representation `rep` using buffers `dst`
// (which must not alias the source's live buffer).
g2_status vset_convert(g2_graph *g, const VSet &src, int rep, VSet &dst, cudaStream_t st);
// Exact member count of a bitmap / boolmap on the device into *d_out.
g2_status vset_count(g2_graph *g, const VSet &v, int32_t *d_out, cudaStream_t st);

// ------------------------------------------------------------- apply engine
enum OpKind { K_BFS, K_RELAX, K_LABEL, K_PR, K_SIGMA, K_HOOK, K_DELTA };

struct OpArgs {
    OpKind kind;
    int32_t *i0;       // depth / dist / label
    int32_t *i1;       // parent
    const float *f0;   // contrib
    float *f1;         // acc
    double *d0;        // sigma
    int32_t threshold; // RELAX near/far split (INT32_MAX: everything near)
    int32_t *err;
};

struct OutArgs {
    int rep;            // OUT_NONE / OUT_SPARSE / OUT_BITMAP / OUT_BOOLMAP
    int32_t *q;
    int32_t qcap;
    int32_t *cnt;       // device counter of q (zeroed by the caller)
    uint32_t *bitmap;   // zeroed by the caller
    uint8_t *boolmap;   // zeroed by the caller
    int dedup;          // DD_*
    // far pile (RELAX only)
    int32_t *q2;
    int32_t q2cap;
    int32_t *cnt2;
    int32_t *stamp2;
    int32_t round2;
};

// One edgeset.apply round with a simple schedule.  `in` must already be in
// the representation the schedule's direction needs: a list (or all
// vertices) for PUSH, a bitmap / boolmap (or all vertices) for PULL.
g2_status apply_round(g2_graph *g, const g2_schedule &s, const OpArgs &op, const VSet &in,
                      const OutArgs &out, cudaStream_t st);

// Check that a simple schedule is valid and implemented for op/direction.
g2_status check_schedule(const g2_graph *g, const g2_schedule &s, OpKind op, bool all_vertices);

// Pick s1/s2 of a hybrid schedule for an input frontier of `size` vertices.
const g2_schedule &pick_schedule(const g2_hybrid &h, int32_t size, int32_t n);
g2_hybrid default_hybrid();

}  // namespace g2
