// g2_pr_seg.cuh — the PageRank arc sweep (Sec. VII: one PULL + EDGE_ONLY
// round over the CSC; the vertex pass in g2_pr.cu finishes the rank update).
// Kept in a file of its own so that a profile of this kernel can name the
// exact source it was taken on.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "g2_device.cuh"

namespace g2 {

// ------------------------------------------------ segmented arc sweep
// A warp takes 128 consecutive CSC arcs (one int4 of column ids per lane),
// gathers their shares, and sums them per row with a warp segmented scan
// whose segment starts are precomputed row-head flags (bit e set iff arc e is
// the first in-arc of its row).  Row ids come from the rank of each head:
// the k-th head overall starts row nzrow[k].  Sums are added with
// fire-and-forget reductions into y (zeroed again by the vertex pass), so no
// block barrier or search is needed anywhere.
constexpr int kSegArcs = 128;  // arcs per warp chunk

// The dangling mass D of a vertex pass is accumulated in kDSlots slots (one
// per 128-byte line) instead of one word, so the warps' atomics spread over
// many L2 lines instead of serialising on one address.
constexpr int kDSlots = 64;
constexpr int kDStride = 16;  // doubles between slots

// One warp: *fin = the sum of the slots, which are zeroed for the next pass.
__device__ __forceinline__ void fold_dslots(double *slots, double *fin) {
    const int lane = threadIdx.x & 31;
    double v = slots[lane * kDStride] + slots[(lane + 32) * kDStride];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(G2_FULL, v, o);
    slots[lane * kDStride] = 0.0;
    slots[(lane + 32) * kDStride] = 0.0;
    if (lane == 0) *fin = v;
}

__device__ __forceinline__ float ld_evict_last(const float *p) {
    float v;
    asm volatile("ld.global.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// Share of slot u: the hottest slots from shared memory, an optional next
// tier [hot, warm) through L1 with evict-last priority, the rest through the
// read-only path.  (Loading the cold rest without L1 allocation was measured
// to lower the L2 hit rate and raise DRAM reads by half, so it is not used.)
template <bool HOT>
__device__ __forceinline__ float seg_gather(const float *contrib, const float *s_hot, int32_t hot,
                                            int32_t warm, int32_t u) {
    if (HOT && u < hot) return s_hot[u];
    if (u < warm) return ld_evict_last(contrib + u);
    return __ldg(contrib + u);
}

template <int CTA, bool HOT>
__global__ void __launch_bounds__(CTA) k_pr_seg(const int32_t *pcol, const uint32_t *head,
                                                const int32_t *chunk_rank, const int32_t *nzrow,
                                                int32_t m, int64_t nchunks, const float *contrib,
                                                int32_t hot, int32_t warm, float *y,
                                                double *dslots, double *dfin) {
    extern __shared__ float s_hot[];
    // The previous vertex pass left D in kDSlots slots: the first warp of
    // block 0 adds them into *dfin (read by the next vertex pass) and zeroes
    // them (dslots null: nothing to fold).
    if (dslots && blockIdx.x == 0 && threadIdx.x < 32) fold_dslots(dslots, dfin);
    if (HOT) {
        for (int32_t i = threadIdx.x; i < hot; i += CTA) s_hot[i] = __ldg(contrib + i);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    // chunk indices fit 32 bits: m < 2^31 arcs, 128 arcs per chunk
    const int32_t nch = (int32_t)nchunks;
    const int32_t gw = (int32_t)((blockIdx.x * CTA + threadIdx.x) >> 5);
    const int32_t nw = (int32_t)((gridDim.x * CTA) >> 5);
    const int sh = (lane & 7) * 4;
    const unsigned below = (1u << sh) - 1u;
    const int4 *pcol4 = reinterpret_cast<const int4 *>(pcol) + lane;
    const uint4 *head4 = reinterpret_cast<const uint4 *>(head);
    // software pipeline: the next chunk's column ids and head words are
    // loaded while this chunk's gathers are in flight
    int4 nu4 = make_int4(0, 0, 0, 0);
    uint4 nh = make_uint4(0, 0, 0, 0);
    if (gw < nch) {
        nu4 = pcol4[(int64_t)gw * (kSegArcs / 4)];
        nh = head4[gw];
    }
    for (int32_t c = gw; c < nch; c += nw) {
        const int4 u4 = nu4;
        const uint32_t w0 = nh.x, w1 = nh.y, w2 = nh.z, w3 = nh.w;
        if (c + nw < nch) {
            nu4 = pcol4[(int64_t)(c + nw) * (kSegArcs / 4)];
            nh = head4[c + nw];
        }
        float v0, v1, v2, v3;
        if ((int64_t)(c + 1) * kSegArcs <= m) {
            v0 = seg_gather<HOT>(contrib, s_hot, hot, warm, u4.x);
            v1 = seg_gather<HOT>(contrib, s_hot, hot, warm, u4.y);
            v2 = seg_gather<HOT>(contrib, s_hot, hot, warm, u4.z);
            v3 = seg_gather<HOT>(contrib, s_hot, hot, warm, u4.w);
        } else {
            // the last, partial chunk
            const int64_t a0 = (int64_t)c * kSegArcs + 4 * lane;
            v0 = a0 + 0 < m ? seg_gather<HOT>(contrib, s_hot, hot, warm, u4.x) : 0.f;
            v1 = a0 + 1 < m ? seg_gather<HOT>(contrib, s_hot, hot, warm, u4.y) : 0.f;
            v2 = a0 + 2 < m ? seg_gather<HOT>(contrib, s_hot, hot, warm, u4.z) : 0.f;
            v3 = a0 + 3 < m ? seg_gather<HOT>(contrib, s_hot, hot, warm, u4.w) : 0.f;
        }
        const int wi = lane >> 3;
        const uint32_t mine = wi == 0 ? w0 : wi == 1 ? w1 : wi == 2 ? w2 : w3;
        const uint32_t hf = (mine >> sh) & 0xFu;
        // heads before this lane in the chunk
        int prefix = __popc(mine & below);
        if (wi > 0) prefix += __popc(w0);
        if (wi > 1) prefix += __popc(w1);
        if (wi > 2) prefix += __popc(w2);
        const int total_heads = __popc(w0) + __popc(w1) + __popc(w2) + __popc(w3);
        const int32_t base_rank = chunk_rank[c];
        // lane-local pieces: A = arcs before the first head, inner complete
        // segments, T = arcs from the last head on
        float vals[4] = {v0, v1, v2, v3};
        float A = 0.f, run = 0.f;
        int seen = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if ((hf >> k) & 1u) {
                if (seen == 0) {
                    A = run;
                } else if (run != 0.f) {
                    // complete segment inside this lane: its head is the (seen-1)-th
                    atomicAdd(y + nzrow[base_rank + prefix + seen - 1], run);
                }
                run = 0.f;
                ++seen;
            }
            run += vals[k];
        }
        if (seen == 0) A = run;
        const bool has_head = seen > 0;
        const float T = has_head ? run : 0.f;
        // segmented inclusive scan over lanes: q = T at a headed lane, else
        // q(previous lane) + A.  Shares are >= 0, so the partial sums are too
        // and the head flag travels in the sign bit: one shuffle per step.
        float q = has_head ? T : A;
        bool f = has_head;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t enc = __float_as_uint(q) | (f ? 0x80000000u : 0u);
            const uint32_t o = __shfl_up_sync(G2_FULL, enc, d);
            if (lane >= d && !f) {
                q += __uint_as_float(o & 0x7fffffffu);
                f = (o >> 31) != 0u;
            }
        }
        float qprev = __shfl_up_sync(G2_FULL, q, 1);
        if (lane == 0) qprev = 0.f;
        if (has_head) {
            // the segment that ends just before this lane's first head
            float tot = qprev + A;
            int32_t rk = base_rank + prefix - 1;
            if (tot != 0.f && rk >= 0) atomicAdd(y + nzrow[rk], tot);
        }
        if (lane == 31) {
            // the segment that runs to the end of the chunk (may continue)
            int32_t rk = base_rank + total_heads - 1;
            if (q != 0.f && rk >= 0) atomicAdd(y + nzrow[rk], q);
        }
    }
}

}  // namespace g2
