// g2_pr_blk.cu — PageRank over the source-blocked layout (the sweep kernel is
// in g2_pr_blk.cuh).  Round t of Sec. VII's topology-driven PageRank,
//   x_t[v] = (1-d)/n + d * ( sum_{u->v} x_{t-1}[u]/outdeg(u) + D_{t-1}/n ),
// runs in rank space: every per-vertex array is indexed by the vertex's rank
// (the stable degree-bucket order of the layout), so the shares of one
// source block are contiguous and the vertex pass streams.  x_0 = 1/n needs
// no permutation; the last vertex pass writes x_t back in vertex order.
//
// The layout build is an EdgeBlocking preprocessing step (Algorithm 1: a
// stable counting sort of the arcs by block), here keyed by the source's
// block and done on the device by a warp-tiled stable partition:
//   1. rank of every vertex: stable partition of the vertices by degree
//      bucket (highest bucket first);
//   2. rank of every arc's source, its block = rank / S;
//   3. stable partition of the CSC arcs by block, every block padded to
//      whole chunks;
//   4. per arc its rank within the block (16 bits) and its destination's
//      rank (a temporary), then the run heads, the run destinations and the
//      runs before every chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "g2_host.h"
#include "g2_pr_blk.cuh"

namespace g2 {

// ------------------------------------------------------- stable partition
// Items 0..count-1 with keys vals[i] / div in [0, nkeys) get positions such
// that the items of key k occupy [start_k, start_k + size_k) in index order,
// and start_k = the sum over j < k of size_j rounded up to a multiple of pad.
// A warp owns a tile of kPartTile consecutive items and walks it 32 at a
// time; counts live in the warp's slice of shared memory (nkeys ints).
constexpr int kPartTile = 2048;
constexpr int kPartMaxKeys = 1024;
constexpr int kPartCta = 256;

// floor(x / d) for 0 <= x < 2^31 and 1 <= d < 2^24: a float estimate from the
// reciprocal, then the exact correction (the estimate is off by at most one)
__device__ __forceinline__ int32_t div_floor(int32_t x, int32_t d, float inv) {
    int32_t q = __float2int_rz((float)x * inv);
    if (q * d > x) --q;
    else if ((q + 1) * d <= x) ++q;
    return q;
}

__global__ void __launch_bounds__(kPartCta) k_part_count(const int32_t *vals, int32_t div,
                                                         int64_t count, int32_t nkeys,
                                                         int32_t ntiles, int32_t *counts) {
    extern __shared__ int32_t s_part[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *c = s_part + wid * nkeys;
    const int32_t wpc = kPartCta / 32;
    for (int32_t tile = blockIdx.x * wpc + wid; tile < ntiles; tile += gridDim.x * wpc) {
        for (int k = lane; k < nkeys; k += 32) c[k] = 0;
        __syncwarp();
        const int64_t base = (int64_t)tile * kPartTile;
        const float inv = 1.0f / (float)div;
#pragma unroll 8
        for (int s = 0; s < kPartTile / 32; ++s) {
            const int64_t i = base + s * 32 + lane;
            if (i < count) atomicAdd(&c[div_floor(vals[i], div, inv)], 1);
        }
        __syncwarp();
        for (int k = lane; k < nkeys; k += 32) counts[(int64_t)k * ntiles + tile] = c[k];
        __syncwarp();
    }
}

// scan = exclusive scan of counts (key-major); one CTA: padded key starts,
// shift[k] = padded start - unpadded start, pstart[nkeys] = padded total
__global__ void k_part_starts(const int32_t *scan, int32_t ntiles, int32_t nkeys, int32_t pad,
                              int32_t *shift, int32_t *pstart, int32_t *total) {
    __shared__ int32_t s_beg[kPartMaxKeys + 1];
    for (int k = threadIdx.x; k <= nkeys; k += blockDim.x) s_beg[k] = scan[(int64_t)k * ntiles];
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int k = 0; k < nkeys; ++k) {
            const int64_t size = s_beg[k + 1] - s_beg[k];
            pstart[k] = (int32_t)acc;
            shift[k] = (int32_t)(acc - s_beg[k]);
            acc += (size + pad - 1) / pad * pad;
        }
        pstart[nkeys] = (int32_t)acc;
        *total = (int32_t)acc;
    }
}

__global__ void __launch_bounds__(kPartCta) k_part_pos(const int32_t *vals, int32_t div,
                                                       int64_t count, int32_t nkeys, int32_t ntiles,
                                                       const int32_t *scan, const int32_t *shift,
                                                       int32_t *pos) {
    extern __shared__ int32_t s_part[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int32_t *c = s_part + wid * nkeys;
    const int32_t wpc = kPartCta / 32;
    for (int32_t tile = blockIdx.x * wpc + wid; tile < ntiles; tile += gridDim.x * wpc) {
        for (int k = lane; k < nkeys; k += 32) c[k] = scan[(int64_t)k * ntiles + tile] + shift[k];
        __syncwarp();
        const int64_t base = (int64_t)tile * kPartTile;
        for (int s = 0; s < kPartTile / 32; ++s) {
            const int64_t i = base + s * 32 + lane;
            const int key = i < count ? vals[i] / div : -1;
            const unsigned peers = __match_any_sync(G2_FULL, key);
            const int r = __popc(peers & lt);
            if (key >= 0) pos[i] = c[key] + r;
            __syncwarp();
            if (key >= 0 && r == 0) c[key] += __popc(peers);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------- layout kernels
// degree bucket key, highest bucket first (bucket 0 = no out-arcs, last)
__global__ void k_blk_vkey(const int32_t *rowptr, int32_t n, int32_t *key) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        key[v] = kDegBuckets - 1 - deg_bucket(rowptr[v + 1] - rowptr[v]);
}

// order[rank[v]] = v, deg[rank[v]] = outdeg(v)
__global__ void k_blk_order(const int32_t *rowptr, const int32_t *rank, int32_t n, int32_t *order,
                            int32_t *deg) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = rank[v];
        order[r] = (int32_t)v;
        deg[r] = rowptr[v + 1] - rowptr[v];
    }
}

// Per CSC arc: the rank of its source, and (as k_part_count) the per-tile
// counts of the partition keys srank / S, in one pass over the arcs.  Eight
// steps' gathers are issued before their counts.
__global__ void __launch_bounds__(kPartCta) k_blk_src_count(const int32_t *ccol,
                                                            const int32_t *rank, int32_t S,
                                                            int64_t count, int32_t nkeys,
                                                            int32_t ntiles, int32_t *srank,
                                                            int32_t *counts) {
    extern __shared__ int32_t s_part[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t *c = s_part + wid * nkeys;
    const int32_t wpc = kPartCta / 32;
    const float inv = 1.0f / (float)S;
    for (int32_t tile = blockIdx.x * wpc + wid; tile < ntiles; tile += gridDim.x * wpc) {
        for (int k = lane; k < nkeys; k += 32) c[k] = 0;
        __syncwarp();
        const int64_t base = (int64_t)tile * kPartTile;
        constexpr int kB = 8;
        for (int s0 = 0; s0 < kPartTile / 32; s0 += kB) {
            int32_t sr[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int64_t i = base + (s0 + j) * 32 + lane;
                sr[j] = i < count ? rank[ccol[i]] : -1;
            }
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int64_t i = base + (s0 + j) * 32 + lane;
                if (i < count) {
                    srank[i] = sr[j];
                    atomicAdd(&c[div_floor(sr[j], S, inv)], 1);
                }
            }
        }
        __syncwarp();
        for (int k = lane; k < nkeys; k += 32) counts[(int64_t)k * ntiles + tile] = c[k];
        __syncwarp();
    }
}

// Per CSC arc of row v: the rank of v.  The rows are taken 32 at a time (a
// group); a group's arcs are cut into pieces of kDstPiece positions, and
// every piece is one work item (hub rows make a few groups hold millions of
// arcs).  k_blk_dst_pieces counts the pieces of every group; after their
// exclusive scan, a warp takes an equal range of consecutive items, finds
// the group of its first item by one binary search and walks on from there.
// For an item the warp loads the 32 rows' ends and ranks (one coalesced load
// each) and writes the piece's positions in coalesced steps of 32, each lane
// finding its position's row among the 32 by a binary search over the lanes.
constexpr int kDstPiece = 2048;

__global__ void k_blk_dst_pieces(const int32_t *crowptr, int32_t n, int32_t *pieces) {
    const int64_t groups = ((int64_t)n + 31) / 32;
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < groups;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = (int64_t)crowptr[min((int64_t)n, gi * 32 + 32)] - crowptr[gi * 32];
        pieces[gi] = (int32_t)((len + kDstPiece - 1) / kDstPiece);
    }
}

__global__ void k_blk_dst_ranks(const int32_t *crowptr, const int32_t *rank, int32_t n,
                                const int32_t *piece_start, int32_t *drank) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t groups = (int32_t)(((int64_t)n + 31) / 32);
    const int64_t items = piece_start[groups];
    const int64_t per = (items + nw - 1) / nw;
    const int64_t it0 = gw * per, it1 = min(items, it0 + per);
    if (it0 >= it1) return;
    // the group of item it0: the last g with piece_start[g] <= it0
    int32_t g = 0, hi = groups - 1;
    while (g < hi) {
        const int32_t mid = (int32_t)(((int64_t)g + hi + 1) >> 1);
        if (piece_start[mid] <= it0) g = mid;
        else hi = mid - 1;
    }
    int32_t gbeg = piece_start[g], gend = piece_start[g + 1];
    int32_t end = 0, rk = 0, start = 0, stop = 0, loaded = -1;
    for (int64_t it = it0; it < it1; ++it) {
        while (it >= gend) {  // groups without pieces (no arcs) are passed over
            ++g;
            gbeg = gend;
            gend = piece_start[g + 1];
        }
        if (loaded != g) {
            const int32_t v0 = g * 32;
            const int32_t vl = min(v0 + lane, n - 1);
            end = crowptr[vl + 1];  // end of row v0 + lane (rows past n: m)
            rk = rank[vl];
            start = crowptr[v0];
            stop = __shfl_sync(G2_FULL, end, 31);
            loaded = g;
        }
        const int32_t pb = start + (int32_t)(it - gbeg) * kDstPiece;
        const int32_t pe = min(stop, pb + kDstPiece);
        for (int32_t p0 = pb; p0 < pe; p0 += 32) {
            const int32_t p = p0 + lane;
            // k = the number of the 32 rows that end at or before arc p
            // (at most 31 for p < stop)
            int k = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (__shfl_sync(G2_FULL, end, k + step - 1) <= p) k += step;
            const int32_t r = __shfl_sync(G2_FULL, rk, k);
            if (p < pe) drank[p] = r;
        }
    }
}

// The position pass of the stable partition of the arcs by source block
// (keys srank / S), placing every arc directly: its source's rank within the
// block and its destination's rank go to its position.  A warp's stores
// fall into one contiguous run per block present among its 32 arcs.  Warps
// take tiles from a counter (equal tiles, uneven costs).  Within a tile,
// the first lane of each key's group among a step's 32 arcs claims the
// group's positions with one shared-memory atomic that returns the key's
// running count; eight steps' claims are issued back to back, and the warp's
// claims to one counter are served in the order of its instructions, so the
// tile's arcs of one key keep their order (were two steps' claims ever
// served the other way round, a run would only split in two: positions stay
// disjoint and every one is filled).
__global__ void __launch_bounds__(kPartCta) k_blk_place(const int32_t *srank, const int32_t *drank,
                                                        int32_t S, int64_t count, int32_t nkeys,
                                                        int32_t ntiles, const int32_t *scan,
                                                        const int32_t *shift, int32_t *tile_ctr,
                                                        uint16_t *loc, int32_t *dst) {
    extern __shared__ int32_t s_part[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int32_t *c = s_part + wid * nkeys;
    const float inv = 1.0f / (float)S;
    for (;;) {
        int32_t tile = 0;
        if (lane == 0) tile = atomicAdd(tile_ctr, 1);
        tile = __shfl_sync(G2_FULL, tile, 0);
        if (tile >= ntiles) break;
        for (int k = lane; k < nkeys; k += 32) c[k] = scan[(int64_t)k * ntiles + tile] + shift[k];
        __syncwarp();
        const int64_t base = (int64_t)tile * kPartTile;
        constexpr int kB = 8;
        for (int s0 = 0; s0 < kPartTile / 32; s0 += kB) {
            int32_t sr[kB], dr[kB], got[kB], who[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int64_t i = base + (s0 + j) * 32 + lane;
                sr[j] = i < count ? srank[i] : -1;
                dr[j] = i < count ? drank[i] : 0;
            }
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int key = sr[j] >= 0 ? div_floor(sr[j], S, inv) : -1;
                const unsigned peers = __match_any_sync(G2_FULL, key);
                const int lead = __ffs(peers) - 1;
                got[j] = 0;
                if (key >= 0 && lane == lead) got[j] = atomicAdd(&c[key], __popc(peers));
                who[j] = (lead << 8) | __popc(peers & lt);
            }
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                const int32_t p = __shfl_sync(G2_FULL, got[j], who[j] >> 8) + (who[j] & 0xFF);
                if (sr[j] >= 0) {
                    const int key = div_floor(sr[j], S, inv);
                    loc[p] = (uint16_t)(sr[j] - key * S);
                    dst[p] = dr[j];
                }
            }
        }
        __syncwarp();  // the tile's claims are done before the counters are reset
    }
}

// The padding of every block (after its arcs, up to the next whole chunk):
// source rank 0 of the block and the spare destination slot n.  A CTA per
// block.
__global__ void k_blk_fill_pad(const int32_t *scan, int32_t ntiles, const int32_t *pstart,
                               int32_t nb, int32_t n, uint16_t *loc, int32_t *dst) {
    for (int32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t size = (int64_t)scan[(int64_t)(b + 1) * ntiles] - scan[(int64_t)b * ntiles];
        for (int64_t p = pstart[b] + size + threadIdx.x; p < pstart[b + 1]; p += blockDim.x) {
            loc[p] = 0;
            dst[p] = n;
        }
    }
}

static __global__ void k_fill_i32_blk(int32_t *p, int64_t count, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// First chunk of every block (blocks start on chunk boundaries) and a flag
// per chunk that starts a block with arcs.
__global__ void k_blk_mark_starts(const int32_t *pstart, int32_t nb, int64_t total,
                                  uint8_t *chunk_start, int32_t *bchunk) {
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x) {
        const int32_t p = pstart[b];
        bchunk[b] = p / kBlkArcs;
        if (b < nb && p < total && pstart[b + 1] > p) chunk_start[p / kBlkArcs] = 1;
    }
}

// The head flags of a chunk and what the sweep reads of them, a warp per
// chunk: lane l holds arcs 8l .. 8l + 7 (two 16-byte loads of destinations);
// arc k is a head where its destination differs from the arc before it, or
// where it starts a block.  Out: the chunk's 8 head words (bit j of word w:
// arc 32w + j), per lane (heads before the lane in the chunk << 8) | its 8
// flags, and the chunk's head count.
__global__ void k_blk_heads(const int32_t *dst, int64_t nchunks, const uint8_t *chunk_start,
                            uint32_t *head, uint16_t *lane_heads, int32_t *ccount) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int64_t c = gw; c < nchunks; c += nw) {
        const int64_t p = c * kBlkArcs + lane * 8;
        const int4 d0 = *reinterpret_cast<const int4 *>(dst + p);
        const int4 d1 = *reinterpret_cast<const int4 *>(dst + p + 4);
        int32_t prev = __shfl_up_sync(G2_FULL, d1.w, 1);
        if (lane == 0) prev = (p > 0 && !chunk_start[c]) ? dst[p - 1] : -1;
        const int32_t d[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
        uint32_t hf = (uint32_t)(d[0] != prev);
#pragma unroll
        for (int k = 1; k < 8; ++k) hf |= (uint32_t)(d[k] != d[k - 1]) << k;
        // heads before this lane: exclusive scan of the lanes' counts
        const int cnt = __popc(hf);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(G2_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        lane_heads[c * 32 + lane] = (uint16_t)(((incl - cnt) << 8) | hf);
        // head word w = the flags of lanes 4w .. 4w + 3
        uint32_t word = hf << (8 * (lane & 3));
        word |= __shfl_xor_sync(G2_FULL, word, 1);
        word |= __shfl_xor_sync(G2_FULL, word, 2);
        if ((lane & 3) == 0) head[c * kBlkHeadWords + (lane >> 2)] = word;
        if (lane == 31) ccount[c] = incl;
    }
}

// nzrow1[k + 1] = destination rank of the k-th run
__global__ void k_blk_nzrow(const uint32_t *head, const int32_t *chunk_rank, const int32_t *dst,
                            int64_t words, int32_t *nzrow1) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = w / kBlkHeadWords;
        int32_t r = chunk_rank[c];
        for (int64_t j = c * kBlkHeadWords; j < w; ++j) r += __popc(head[j]);
        uint32_t bits = head[w];
        while (bits) {
            const int j = __ffs(bits) - 1;
            bits &= bits - 1;
            nzrow1[++r] = dst[w * 32 + j];
        }
    }
}

// cta_chunk[i] = the first chunk of CTA i: the least c with
// kBlkArcs * c + runcost * (runs before c) >= i / G of the sweep's total cost
__global__ void k_blk_cta_split(const int32_t *chunk_rank, int64_t nchunks, int32_t G,
                                int32_t runcost, int32_t *cta_chunk) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > G) return;
    const int64_t total = kBlkArcs * nchunks + (int64_t)runcost * chunk_rank[nchunks];
    const int64_t target = total * i / G;
    int64_t lo = 0, hi = nchunks;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (kBlkArcs * mid + (int64_t)runcost * chunk_rank[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    cta_chunk[i] = (int32_t)lo;
}

// --------------------------------------------------------- vertex passes
// The first shares in rank order (x0 = 1/n), D0 = (#vertices without
// out-arcs)/n into the slots (one reduction per CTA), and x0 in the caller's
// array where there are no rounds to write it (x: the same value everywhere).
__global__ void __launch_bounds__(kCta) k_pr_blk_init(const int32_t *deg, int32_t n, float *share,
                                                      double *dslots, float *x, double inv_n) {
    __shared__ float s_d[kCta / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const float x0 = (float)inv_n;
    float dangling = 0.f;
    if (r0 + 4 <= n) {
        const int4 d4 = *reinterpret_cast<const int4 *>(deg + r0);
        const int32_t od[4] = {d4.x, d4.y, d4.z, d4.w};
        float sh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sh[k] = od[k] > 0 ? x0 / (float)od[k] : 0.f;
            dangling += od[k] == 0 ? 1.f : 0.f;
        }
        *reinterpret_cast<float4 *>(share + r0) = make_float4(sh[0], sh[1], sh[2], sh[3]);
        if (x) *reinterpret_cast<float4 *>(x + r0) = make_float4(x0, x0, x0, x0);
    } else {
        for (int k = 0; k < 4; ++k) {
            const int64_t r = r0 + k;
            if (r >= n) break;
            const int32_t od = deg[r];
            share[r] = od > 0 ? x0 / (float)od : 0.f;
            if (od == 0) dangling += 1.f;
            if (x) x[r] = x0;
        }
    }
    // at most 1,024 per CTA: exact in fp32; scaled by 1/n in fp64
    for (int o = 16; o > 0; o >>= 1) dangling += __shfl_xor_sync(G2_FULL, dangling, o);
    if (lane == 0) s_d[warp] = dangling;
    __syncthreads();
    if (warp == 0) {
        float v = lane < kCta / 32 ? s_d[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(G2_FULL, v, o);
        if (lane == 0 && v != 0.f)
            atomicAdd(dslots + (blockIdx.x % kDSlots) * kDStride, (double)v * inv_n);
    }
}

// After a sweep: x_t from y, the next shares, the next D; y back to zero,
// over ranks [0, n).  A thread takes U groups of four consecutive ranks
// (16-byte loads and stores), the groups of a CTA adjacent, all U groups'
// loads issued before their arithmetic; the last round also writes x_t to
// the caller's array in vertex order.  D's partial sums meet in shared
// memory: one fp64 reduction per CTA.  ntail isolated vertices ranked after
// n (no arc in or out: y = 0, no share) are left out, their x_t being the
// same for all: CTA 0 adds ntail * x_t to D.
template <bool WRITE_X, int U>
__global__ void __launch_bounds__(kCta) k_pr_blk_vertex(const int32_t *deg, const int32_t *order,
                                                        int32_t n, int32_t ntail, float *y,
                                                        float *share_next, float *x,
                                                        const double *dprev, double *dslots,
                                                        float base, float damp, double inv_n) {
    __shared__ float s_d[kCta / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cta0 = (int64_t)blockIdx.x * (kCta * 4 * U);
    int32_t od[U][4];
    float yv[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t r0 = cta0 + ((int64_t)u * kCta + threadIdx.x) * 4;
        if (r0 + 4 <= n) {
            const int4 d4 = *reinterpret_cast<const int4 *>(deg + r0);
            const float4 y4 = *reinterpret_cast<const float4 *>(y + r0);
            od[u][0] = d4.x; od[u][1] = d4.y; od[u][2] = d4.z; od[u][3] = d4.w;
            yv[u][0] = y4.x; yv[u][1] = y4.y; yv[u][2] = y4.z; yv[u][3] = y4.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                od[u][k] = r0 + k < n ? deg[r0 + k] : 0;
                yv[u][k] = r0 + k < n ? y[r0 + k] : 0.f;
            }
        }
    }
    const float dterm = (float)(*dprev * inv_n);
    float dsum = 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t r0 = cta0 + ((int64_t)u * kCta + threadIdx.x) * 4;
        if (r0 >= n) continue;
        const bool full = r0 + 4 <= n;
        float xs[4], sh[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            xs[k] = base + damp * (yv[u][k] + dterm);
            sh[k] = 0.f;
            if (r0 + k >= n) continue;
            if (od[u][k] > 0) sh[k] = xs[k] / (float)od[u][k];
            else dsum += xs[k];
        }
        if (full) {
            *reinterpret_cast<float4 *>(share_next + r0) = make_float4(sh[0], sh[1], sh[2], sh[3]);
            *reinterpret_cast<float4 *>(y + r0) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            for (int k = 0; k < 4; ++k)
                if (r0 + k < n) {
                    share_next[r0 + k] = sh[k];
                    y[r0 + k] = 0.f;
                }
        }
        if (WRITE_X) {
            if (full) {
                const int4 o4 = *reinterpret_cast<const int4 *>(order + r0);
                x[o4.x] = xs[0];
                x[o4.y] = xs[1];
                x[o4.z] = xs[2];
                x[o4.w] = xs[3];
            } else {
                for (int k = 0; k < 4; ++k)
                    if (r0 + k < n) x[order[r0 + k]] = xs[k];
            }
        }
    }
    if (ntail > 0 && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(dslots, (double)ntail * (double)(base + damp * (0.f + dterm)));
    // D partial of the CTA into one of the fp64 slots; the next sweep folds them
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(G2_FULL, dsum, o);
    if (lane == 0) s_d[warp] = dsum;
    __syncthreads();
    if (warp == 0) {
        float v = lane < kCta / 32 ? s_d[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(G2_FULL, v, o);
        if (lane == 0 && v != 0.f) atomicAdd(dslots + (blockIdx.x % kDSlots) * kDStride, (double)v);
    }
}

// ------------------------------------------------------------ host side
static int part_grid(const g2_graph *g, int32_t ntiles) {
    const int wpc = kPartCta / 32;
    int64_t b = ((int64_t)ntiles + wpc - 1) / wpc;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)g->topo->sm_count * 8));
}

// The count and scan of a stable partition (see k_part_count): the scan of
// the per-tile counts, the padded key starts (pstart, nkeys + 1 entries; the
// padded total also in *total) and the launch shape of the position pass.
struct PartTable {
    int32_t *counts = nullptr, *scan = nullptr, *shift = nullptr;
    int32_t ntiles = 0;
    int grid = 1;
    size_t smem = 0;
    void release(cudaStream_t st) {
        dfree(counts, st);
        dfree(scan, st);
        dfree(shift, st);
        counts = scan = shift = nullptr;
    }
};

// The tables of a stable partition of count items into nkeys keys, and the
// launch shape of its count and position passes.
static g2_status partition_alloc(g2_graph *g, int64_t count, int32_t nkeys, PartTable *pt,
                                 cudaStream_t st) {
    pt->ntiles = (int32_t)std::max<int64_t>(1, (count + kPartTile - 1) / kPartTile);
    const int64_t cells = (int64_t)nkeys * pt->ntiles;
    if (cells >= 2147483647LL) return fail(G2_EUNSUPPORTED, "partition table too large");
    G2_CK(dmalloc(&pt->counts, (size_t)(cells + 1) * 4, st));
    G2_CK(dmalloc(&pt->scan, (size_t)(cells + 1) * 4, st));
    G2_CK(dmalloc(&pt->shift, (size_t)nkeys * 4, st));
    pt->smem = (size_t)(kPartCta / 32) * nkeys * 4;
    pt->grid = part_grid(g, pt->ntiles);
    return G2_OK;
}

// After the count pass: the scan, the padded key starts and the total.
static g2_status partition_starts(g2_graph *g, int32_t nkeys, int32_t pad, int32_t *pstart,
                                  int64_t *total, PartTable *pt, cudaStream_t st) {
    int32_t *d_total;
    G2_TRY(ws(g, B_CTR, 64, &d_total));
    d_total += 50;
    G2_TRY(exclusive_scan_i32(g, pt->counts, pt->scan, (int32_t)((int64_t)nkeys * pt->ntiles), st));
    k_part_starts<<<1, 1024, 0, st>>>(pt->scan, pt->ntiles, nkeys, pad, pt->shift, pstart, d_total);
    G2_CK(cudaGetLastError());
    G2_CK(cudaMemcpyAsync(g->h_ctr + 50, d_total, 4, cudaMemcpyDeviceToHost, st));
    G2_CK(cudaStreamSynchronize(st));
    *total = g->h_ctr[50];
    stats().launches += 1;
    return G2_OK;
}

static g2_status partition_table(g2_graph *g, const int32_t *vals, int32_t div, int64_t count,
                                 int32_t nkeys, int32_t pad, int32_t *pstart, int64_t *total,
                                 PartTable *pt, cudaStream_t st) {
    G2_TRY(partition_alloc(g, count, nkeys, pt, st));
    k_part_count<<<pt->grid, kPartCta, pt->smem, st>>>(vals, div, count, nkeys, pt->ntiles,
                                                       pt->counts);
    stats().launches += 1;
    return partition_starts(g, nkeys, pad, pstart, total, pt, st);
}

// Positions of a stable partition: pos[i] for every item.
static g2_status stable_partition(g2_graph *g, const int32_t *vals, int32_t div, int64_t count,
                                  int32_t nkeys, int32_t pad, int32_t *pos, int32_t *pstart,
                                  int64_t *total, cudaStream_t st) {
    PartTable pt;
    G2_TRY(partition_table(g, vals, div, count, nkeys, pad, pstart, total, &pt, st));
    k_part_pos<<<pt.grid, kPartCta, pt.smem, st>>>(vals, div, count, nkeys, pt.ntiles, pt.scan, pt.shift,
                                                   pos);
    G2_CK(cudaGetLastError());
    stats().launches += 1;
    pt.release(st);
    return G2_OK;
}

static void free_blk(Topology *t, cudaStream_t st) {
    void *blocks[] = {t->blk_loc, t->blk_lane_heads, t->blk_chunk_rank, t->blk_nzrow, t->blk_bchunk,
                      t->blk_order, t->blk_deg, t->blk_cta};
    for (void *p : blocks) dfree(p, st);
    t->blk_loc = nullptr;
    t->blk_lane_heads = nullptr;
    t->blk_chunk_rank = t->blk_nzrow = t->blk_bchunk = t->blk_order = t->blk_deg = nullptr;
    t->blk_cta = nullptr;
    t->blk_S = 0;
}

// Whether the source-blocked layout applies to t with blocks of S sources.
bool pr_blk_applies(const Topology *t, int32_t S) {
    if (S < 256 || S > kBlkMaxS || (S & 3)) return false;
    if (blk_smem_bytes(S) > (size_t)t->smem_optin) return false;
    const int64_t nb = ((int64_t)t->n + S - 1) / S;
    if (t->n == 0 || nb > kPartMaxKeys) return false;
    // padded arcs must stay int32-addressable
    return (int64_t)t->m + nb * kBlkArcs + kPad < 2147483647LL;
}

g2_status ensure_blk_layout(g2_graph *g, int32_t S, cudaStream_t st) {
    Topology *t = g->topo;
    std::lock_guard<std::recursive_mutex> lk(t->pr_mu);
    if (t->blk_S == S) return G2_OK;
    if (!pr_blk_applies(t, S)) return fail(G2_EUNSUPPORTED, "source-blocked layout does not apply");
    free_blk(t, st);
    const int32_t n = t->n, m = t->m;
    const int32_t nb = (int32_t)(((int64_t)n + S - 1) / S);
    const int grid = grid_for(g, n, kCta);
    int32_t *vkey = nullptr, *rank = nullptr, *vstart = nullptr;
    G2_CK(dmalloc(&vkey, (size_t)n * 4, st));
    G2_CK(dmalloc(&rank, (size_t)n * 4, st));
    G2_CK(dmalloc(&vstart, (size_t)(kDegBuckets + 1) * 4, st));
    G2_CK(dmalloc(&t->blk_order, ((size_t)n + kPad) * 4, st));
    G2_CK(dmalloc(&t->blk_deg, ((size_t)n + kPad) * 4, st));
    G2_CK(dmalloc(&t->blk_bchunk, ((size_t)nb + 1) * 4, st));
    // one CTA per SM; the sweep's chunks are divided among them by cost
    const int32_t G = std::max(1, t->sm_count);
    G2_CK(dmalloc(&t->blk_cta, ((size_t)G + 1) * 4, st));
    // 1. vertex ranks
    k_blk_vkey<<<grid, kCta, 0, st>>>(t->rowptr, n, vkey);
    int64_t vtotal = 0;
    G2_TRY(stable_partition(g, vkey, 1, n, kDegBuckets, 1, rank, vstart, &vtotal, st));
    // the first rank without out-arcs (bucket 0 is ranked last)
    G2_CK(cudaMemcpyAsync(g->h_ctr + 52, vstart + (kDegBuckets - 1), 4, cudaMemcpyDeviceToHost, st));
    k_blk_order<<<grid, kCta, 0, st>>>(t->rowptr, rank, n, t->blk_order, t->blk_deg);
    G2_CK(cudaMemsetAsync(t->blk_order + n, 0, kPad * 4, st));
    G2_CK(cudaMemsetAsync(t->blk_deg + n, 0, kPad * 4, st));
    stats().launches += 2;
    dfree(vkey, st);
    dfree(vstart, st);
    int64_t total = 0;
    int32_t *pstart = nullptr;
    G2_CK(dmalloc(&pstart, ((size_t)nb + 1) * 4, st));
    if (m > 0) {
        // 2-4. source ranks of every arc with the counts of its block key,
        // destination ranks, the stable partition by source block with
        // every arc placed in the position pass; the padding keeps rank 0 of
        // its block and points at the spare slot n
        int32_t *srank = nullptr, *drank = nullptr, *dst = nullptr;
        G2_CK(dmalloc(&srank, (size_t)m * 4, st));
        G2_CK(dmalloc(&drank, (size_t)m * 4, st));
        PartTable pt;
        G2_TRY(partition_alloc(g, m, nb, &pt, st));
        k_blk_src_count<<<pt.grid, kPartCta, pt.smem, st>>>(t->ccol, rank, S, m, nb, pt.ntiles,
                                                             srank, pt.counts);
        {
            const int32_t groups = (int32_t)(((int64_t)n + 31) / 32);
            int32_t *pieces = nullptr, *pstart_d = nullptr;
            G2_CK(dmalloc(&pieces, ((size_t)groups + 1) * 4, st));
            G2_CK(dmalloc(&pstart_d, ((size_t)groups + 1) * 4, st));
            k_blk_dst_pieces<<<grid_for(g, groups, kCta), kCta, 0, st>>>(t->crowptr, n, pieces);
            G2_TRY(exclusive_scan_i32(g, pieces, pstart_d, groups, st));
            k_blk_dst_ranks<<<(int)std::max(1, t->sm_count * 8), kCta, 0, st>>>(
                t->crowptr, rank, n, pstart_d, drank);
            dfree(pieces, st);
            dfree(pstart_d, st);
        }
        stats().launches += 3;
        G2_TRY(partition_starts(g, nb, kBlkArcs, pstart, &total, &pt, st));
        G2_CK(dmalloc(&t->blk_loc, ((size_t)total + kPad) * 2, st));
        G2_CK(dmalloc(&dst, (size_t)total * 4, st));
        G2_CK(cudaMemsetAsync(t->blk_loc + total, 0, (size_t)kPad * 2, st));
        k_blk_fill_pad<<<std::min(nb, 1024), kCta, 0, st>>>(pt.scan, pt.ntiles, pstart, nb, n,
                                                             t->blk_loc, dst);
        int32_t *tile_ctr = nullptr;
        G2_TRY(ws(g, B_CTR, 64, &tile_ctr));
        tile_ctr += 52;
        G2_CK(cudaMemsetAsync(tile_ctr, 0, 4, st));
        k_blk_place<<<pt.grid, kPartCta, pt.smem, st>>>(srank, drank, S, m, nb, pt.ntiles, pt.scan,
                                                         pt.shift, tile_ctr, t->blk_loc, dst);
        stats().launches += 2;
        G2_CK(cudaGetLastError());
        pt.release(st);
        dfree(srank, st);
        dfree(drank, st);
        const int64_t words = total / 32, nchunks = total / kBlkArcs;
        uint32_t *head = nullptr;
        uint8_t *cstart = nullptr;
        int32_t *ccount = nullptr;
        G2_CK(dmalloc(&head, ((size_t)words + kPad) * 4, st));
        G2_CK(cudaMemsetAsync(head + words, 0, kPad * 4, st));
        G2_CK(dmalloc(&cstart, (size_t)nchunks + 16, st));
        G2_CK(cudaMemsetAsync(cstart, 0, (size_t)nchunks + 16, st));
        G2_CK(dmalloc(&ccount, (size_t)nchunks * 4, st));
        G2_CK(dmalloc(&t->blk_chunk_rank, ((size_t)nchunks + kPad) * 4, st));
        const int64_t lanes = nchunks * 32;
        G2_CK(dmalloc(&t->blk_lane_heads, ((size_t)lanes + kPad) * 2, st));
        k_blk_mark_starts<<<(nb + 1 + kCta - 1) / kCta, kCta, 0, st>>>(pstart, nb, total, cstart,
                                                                       t->blk_bchunk);
        k_blk_heads<<<grid_for(g, lanes, kCta), kCta, 0, st>>>(dst, nchunks, cstart, head,
                                                               t->blk_lane_heads, ccount);
        G2_TRY(exclusive_scan_i32(g, ccount, t->blk_chunk_rank, (int32_t)nchunks, st));
        G2_CK(cudaMemcpyAsync(g->h_ctr + 51, t->blk_chunk_rank + nchunks, 4, cudaMemcpyDeviceToHost,
                              st));
        G2_CK(cudaStreamSynchronize(st));
        const int32_t nruns = g->h_ctr[51];
        // run r's row at r + 1; entry 0 and the kPad entries past the last
        // run point at the spare slot n
        G2_CK(dmalloc(&t->blk_nzrow, ((size_t)nruns + 1 + kPad) * 4, st));
        k_fill_i32_blk<<<1, 32, 0, st>>>(t->blk_nzrow, 1, n);
        k_fill_i32_blk<<<1, kPad, 0, st>>>(t->blk_nzrow + (size_t)nruns + 1, kPad, n);
        k_blk_nzrow<<<grid_for(g, words, kCta), kCta, 0, st>>>(head, t->blk_chunk_rank, dst, words,
                                                               t->blk_nzrow);
        int32_t runcost = kBlkRunCost;
        if (const char *e = getenv("G2_PR_BLK_RUNCOST")) runcost = std::max(0, atoi(e));
        k_blk_cta_split<<<(G + 1 + kCta - 1) / kCta, kCta, 0, st>>>(t->blk_chunk_rank, nchunks, G,
                                                                    runcost, t->blk_cta);
        stats().launches += 9;
        dfree(ccount, st);
        dfree(cstart, st);
        dfree(dst, st);
        dfree(head, st);
        t->blk_nruns = nruns;
    } else {
        G2_CK(cudaMemsetAsync(t->blk_bchunk, 0, ((size_t)nb + 1) * 4, st));
        G2_CK(cudaMemsetAsync(t->blk_cta, 0, ((size_t)G + 1) * 4, st));
        t->blk_nruns = 0;
    }
    G2_CK(cudaGetLastError());
    G2_CK(cudaStreamSynchronize(st));
    dfree(rank, st);
    dfree(pstart, st);
    t->blk_nb = nb;
    t->blk_G = G;
    t->blk_nchunks = total / kBlkArcs;
    t->blk_nact = g->h_ctr[52];
    t->blk_S = S;
    return G2_OK;
}

g2_status pagerank_blk_run(g2_graph *g, float damping, int32_t iters, float *rank, int32_t S,
                           cudaStream_t st) {
    Topology *t = g->topo;
    const int32_t n = t->n;
    G2_TRY(ensure_blk_layout(g, S, st));
    const double inv_n = 1.0 / (double)n;
    const float base = (float)((1.0 - damping) * inv_n);
    // shares in rank order, padded with zeros to whole blocks; y in rank
    // order with the spare slot n (the padding runs' target)
    const size_t nshare_alloc = (size_t)t->blk_nb * S + 4;
    float *cbuf[2], *y;
    G2_TRY(ws(g, B_F0, nshare_alloc, &cbuf[0]));
    G2_TRY(ws(g, B_F1, nshare_alloc, &cbuf[1]));
    G2_TRY(ws(g, B_F2, (size_t)n + 4, &y));
    // In a symmetric graph a vertex without out-arcs has no in-arcs either:
    // the non-final vertex passes leave those ranks (the last ones) out.
    const int32_t nact = t->symmetric ? t->blk_nact : n;
    for (int i = 0; i < 2; ++i)
        G2_CK(cudaMemsetAsync(cbuf[i] + nact, 0, (nshare_alloc - nact) * 4, st));
    G2_CK(cudaMemsetAsync(y, 0, ((size_t)n + 4) * 4, st));
    constexpr size_t R = (size_t)kDSlots * kDStride;
    double *dd;
    G2_TRY(ws(g, B_D1, 8 + R, &dd));
    G2_CK(cudaMemsetAsync(dd, 0, (8 + R) * sizeof(double), st));
    const int qblocks = (int)((((int64_t)n + 3) / 4 + kCta - 1) / kCta);
    k_pr_blk_init<<<qblocks, kCta, 0, st>>>(t->blk_deg, n, cbuf[0], dd + 8,
                                            iters <= 0 ? rank : nullptr, inv_n);
    stats().launches += 1;
    if (iters <= 0) return G2_OK;
    const size_t smem = blk_smem_bytes(S);
    auto kern = k_pr_blk<kBlkCta>;
    G2_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // one CTA per SM (the block's shares take most of its shared memory),
    // each with the range of chunks the layout assigned it; launched even
    // without arcs: its first warp folds the dangling mass
    const int grid = t->blk_G;
    const int64_t nshare = ((int64_t)n + 3) & ~(int64_t)3;
    constexpr int kVtxGroups = 2;  // 1: 14.9-15.1 us, 2: 13.5-13.8 us, 4: 14.7 us on RMAT-22
    constexpr int64_t kVtxSpan = (int64_t)kCta * 4 * kVtxGroups;
    const int vgrid = (int)(((int64_t)n + kVtxSpan - 1) / kVtxSpan);
    const int vgrid_act = std::max(1, (int)(((int64_t)nact + kVtxSpan - 1) / kVtxSpan));
    for (int32_t it = 0; it < iters; ++it) {
        double *dprev = dd + 2 + (it & 1);
        KTime kt;
        ktime_begin(kt, "pr_round", st);
        BlkSweepArgs a;
        a.loc4 = reinterpret_cast<const uint4 *>(t->blk_loc);
        a.lane_heads = t->blk_lane_heads;
        a.chunk_rank = t->blk_chunk_rank;
        a.nzrow1 = t->blk_nzrow;
        a.bchunk = t->blk_bchunk;
        a.nb = t->blk_nb;
        a.cta_chunk = t->blk_cta;
        a.S = S;
        a.nshare = nshare;
        a.share = cbuf[it & 1];
        a.y = y;
        a.dslots = dd + 8;
        a.dfin = dprev;
        kern<<<grid, kBlkCta, smem, st>>>(a);
        ktime_end(kt, st);
        KTime kv;
        ktime_begin(kv, "pr_vertex", st);
        float *sn = cbuf[(it + 1) & 1];
        if (it == iters - 1)
            k_pr_blk_vertex<true, kVtxGroups><<<vgrid, kCta, 0, st>>>(
                t->blk_deg, t->blk_order, n, 0, y, sn, rank, dprev, dd + 8, base, damping, inv_n);
        else
            k_pr_blk_vertex<false, kVtxGroups><<<vgrid_act, kCta, 0, st>>>(
                t->blk_deg, t->blk_order, nact, n - nact, y, sn, rank, dprev, dd + 8, base,
                damping, inv_n);
        ktime_end(kv, st);
        stats().launches += 2;
        stats().iterations++;
        stats().pull_rounds++;
    }
    G2_CK(cudaGetLastError());
    return G2_OK;
}

}  // namespace g2
