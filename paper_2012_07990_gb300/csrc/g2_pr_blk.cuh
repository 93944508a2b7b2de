// g2_pr_blk.cuh — the source-blocked PageRank arc sweep (Sec. VII: one PULL
// + EDGE_ONLY round; EdgeBlocking, Sec. VI-D and Algorithms 1-2, applied to
// the sources of the pull instead of the destinations of the push).
// Kept in a file of its own so that a profile of this kernel can name the
// exact source it was taken on.
//
// Layout (built once per topology in g2_pr_blk.cu).  Vertices are numbered
// by rank: a stable order by degree bucket, highest first.  The sources are
// cut into blocks of S consecutive ranks, S sized so that one block's shares
// fill a CTA's shared memory.  The CSC arcs are partitioned stably by the
// block of their source, so inside a block the arcs of one destination stay
// contiguous (a run); each block is padded to whole chunks of kBlkArcs arcs.
// Per arc: the source's rank within its block (16 bits).  Per lane of a
// chunk (8 arcs): its head flags (bit k: arc k is the first of a run, or of a
// block) and the heads before it in the chunk, in one 16-bit word.  Per run:
// its destination's rank (nzrow1, one entry later than the run's number:
// entry 0, which the run before the first stands for, and the padding runs
// point at the spare slot n).
// Per chunk: the number of runs that start before it.
//
// One CTA per SM takes an equal range of chunks.  For each block its range
// touches it copies that block's shares into shared memory once, then its
// warps sweep the block's chunks: every gather is a shared-memory load, and a
// run costs one reduction into y.  On a power-law graph a block's arcs
// concentrate on few destinations (RMAT-22, S = 49,152: 12.3M runs for
// 128.3M arcs), so the scattered L2 traffic per arc falls by an order of
// magnitude against a gather per arc.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "g2_device.cuh"
#include "g2_pr_seg.cuh"

namespace g2 {

constexpr int kBlkArcs = 256;               // arcs per warp chunk, 8 per lane
constexpr int kBlkHeadWords = kBlkArcs / 32;
constexpr int kBlkCta = 1024;               // one CTA per SM, 32 warps
// largest block: 16-bit ranks within a block, and the shares of one block
// within a CTA's shared memory (227 KB on sm_103)
constexpr int kBlkMaxS = 57344;
// default block: 192 KB of shares, measured best on RMAT-22
constexpr int kBlkDefaultS = 49152;

// Cost of a chunk for the division of the sweep among CTAs: its arcs plus
// kBlkRunCost per run (a run costs a row lookup and a reduction into y, about
// four arcs' worth of gathers and sums, measured on RMAT-21).  Sparse blocks
// (low-degree sources, a run per arc or two) would otherwise leave the CTAs
// that draw them several times behind the others.  (4-5 measured best on
// RMAT-22.)
constexpr int kBlkRunCost = 5;

// shared memory of a launch with blocks of S sources
__host__ __device__ constexpr size_t blk_smem_bytes(int S) { return (size_t)S * 4; }

// Arguments of the sweep.  nzrow1 holds the destination of run r at r + 1;
// entry 0 and the entries past the last run hold the spare slot n.
struct BlkSweepArgs {
    const uint4 *loc4;
    const uint16_t *lane_heads;
    const int32_t *chunk_rank;
    const int32_t *nzrow1;
    const int32_t *bchunk;
    int32_t nb;
    const int32_t *cta_chunk;
    int32_t S;
    int64_t nshare;
    const float *share;
    float *y;
    double *dslots;
    double *dfin;
};

// streams read once: kept out of L1, which holds the run rows
__device__ __forceinline__ uint4 ld_stream_u4(const uint4 *p) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ uint32_t ld_stream_u16(const uint16_t *p) {
    unsigned short r;
    asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return r;
}

template <int CTA>
__global__ void __launch_bounds__(CTA, 1) k_pr_blk(BlkSweepArgs a) {
    extern __shared__ __align__(16) float s_sh[];
    // The previous vertex pass left D in kDSlots slots: the first warp of
    // block 0 adds them into *dfin and zeroes them.
    if (a.dslots && blockIdx.x == 0 && threadIdx.x < 32) fold_dslots(a.dslots, a.dfin);
    constexpr int W = CTA / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this CTA's chunks: an equal share of the cost (arcs + runs); chunk
    // indices fit 32 bits (fewer than 2^31 arcs, 256 per chunk)
    int32_t c0 = a.cta_chunk[blockIdx.x];
    const int32_t c1 = a.cta_chunk[blockIdx.x + 1];
    if (c0 >= c1) return;
    // block of chunk c0: the last b with bchunk[b] <= c0 (bchunk[0] = 0)
    int lo = 0, hi = a.nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.bchunk[mid] <= c0) lo = mid;
        else hi = mid - 1;
    }
    int b = lo;
    while (c0 < c1) {
        const int32_t cend = min(c1, a.bchunk[b + 1]);
        if (cend > c0) {
            __syncthreads();  // every warp is done with the previous block's shares
            const int64_t s0 = (int64_t)b * a.S;
            const int32_t len4 = (int32_t)(min((int64_t)a.S, a.nshare - s0) >> 2);
            const float4 *src = reinterpret_cast<const float4 *>(a.share + s0);
            float4 *dst = reinterpret_cast<float4 *>(s_sh);
            for (int i = threadIdx.x; i < len4; i += CTA) {
                const uint4 u = ld_stream_u4(reinterpret_cast<const uint4 *>(src + i));
                dst[i] = make_float4(__uint_as_float(u.x), __uint_as_float(u.y),
                                     __uint_as_float(u.z), __uint_as_float(u.w));
            }
            __syncthreads();
            // software pipeline: the next chunk's ids, head word and run base
            // are loaded while this chunk is summed.  Ids, head words and
            // shares are read once per sweep and bypass L1, which keeps the
            // run rows (read by neighbouring chunks of the same lines).
            int32_t c = c0 + warp;
            const uint4 *lp = a.loc4 + (size_t)c * 32 + lane;
            const uint16_t *hp = a.lane_heads + (size_t)c * 32 + lane;
            uint4 nl = make_uint4(0, 0, 0, 0);
            uint32_t nh = 0;
            int32_t nrk = 0;
            if (c < cend) {
                nl = ld_stream_u4(lp);
                nh = ld_stream_u16(hp);
                nrk = a.chunk_rank[c];
            }
            for (; c < cend; c += W) {
                const uint4 l = nl;
                const uint32_t hf = nh & 0xFFu;             // heads among this lane's arcs
                const int32_t prefix = (int32_t)(nh >> 8);  // heads before this lane
                const int32_t base_rank = nrk;
                lp += W * 32;
                hp += W * 32;
                if (c + W < cend) {
                    nl = ld_stream_u4(lp);
                    nh = ld_stream_u16(hp);
                    nrk = a.chunk_rank[c + W];
                }
                float v[8];
                v[0] = s_sh[l.x & 0xFFFFu];
                v[1] = s_sh[l.x >> 16];
                v[2] = s_sh[l.y & 0xFFFFu];
                v[3] = s_sh[l.y >> 16];
                v[4] = s_sh[l.z & 0xFFFFu];
                v[5] = s_sh[l.z >> 16];
                v[6] = s_sh[l.w & 0xFFFFu];
                v[7] = s_sh[l.w >> 16];
                const int32_t total_heads = __shfl_sync(G2_FULL, prefix + __popc(hf), 31);
                // run r's row is nzb[r - base_rank]: the run open at the
                // chunk's start is r = base_rank - 1
                const int32_t *nzb = a.nzrow1 + base_rank;
                // lane-local pieces: A = arcs before the lane's first head (all
                // of them without a head), inner runs closed by a later head of
                // the lane (one reduction each), run = arcs from the last head on
                float A = 0.f, run = 0.f;
                const int f = hf ? __ffs(hf) - 1 : 8;  // first head (8: none)
                if (!__any_sync(G2_FULL, __popc(hf) >= 2)) {
                    // no lane of the chunk closes a run inside itself (the usual
                    // case in the blocks of high-degree sources)
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        if (k < f) A += v[k];
                        else run += v[k];
                    }
                } else {
                    // head number prefix + j closes run prefix + j - 1
                    int j = prefix;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const bool h = (hf >> k) & 1u;
                        if (h && k > f) atomicAdd(a.y + nzb[j], run);
                        if (k == f) A = run;
                        j += h;
                        run = h ? v[k] : run + v[k];
                    }
                    if (f == 8) A = run;
                }
                const bool has_head = hf != 0;
                // segmented inclusive scan over lanes.  Sums are >= 0, so the
                // segment flag travels in the sign bit; lane 0 always starts a
                // segment, so before the step of distance d lanes 0 .. d-1 are
                // flagged and no lane needs a bounds test.
                uint32_t enc = __float_as_uint(has_head ? run : A) |
                               ((has_head || lane == 0) ? 0x80000000u : 0u);
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t o = __shfl_up_sync(G2_FULL, enc, d);
                    const float sum = __uint_as_float(enc) + fabsf(__uint_as_float(o));
                    if ((int32_t)enc >= 0) enc = __float_as_uint(sum) | (o & 0x80000000u);
                }
                const float q = __uint_as_float(enc & 0x7fffffffu);
                float qprev = __shfl_up_sync(G2_FULL, q, 1);
                if (lane == 0) qprev = 0.f;
                // the run that ends at this lane's first head (run prefix - 1)
                // and the run that reaches the end of the chunk (it may go on
                // in the next chunk of the same block)
                if (has_head) {
                    const float tot = qprev + A;
                    if (tot != 0.f) atomicAdd(a.y + nzb[prefix], tot);
                }
                if (lane == 31 && q != 0.f) atomicAdd(a.y + nzb[total_heads], q);
            }
        }
        c0 = cend;
        ++b;
    }
}

}  // namespace g2
