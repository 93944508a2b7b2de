// g2_cluster.cuh — building blocks of the one-cluster fused loops (the
// small-frontier rounds of kernel fusion, Sec. VI-C, run inside one
// thread-block cluster): the cluster barrier, reads of a peer CTA's shared
// memory, warp-aggregated appends to shared-memory lists, and the host side
// (does a cluster of a kernel fit, launch one cluster).
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>

#include "g2_host.h"

namespace g2 {

constexpr int kClCta = 1024;  // threads per cluster CTA

// Why a one-cluster launch ended.
enum { CL_DONE = 0, CL_TO_GRID = 1, CL_OVERFLOW = 2 };

// Arrive at and wait on the cluster barrier (release / acquire at cluster
// scope: what a CTA wrote before it is visible to every CTA of the cluster
// after it).  Every thread of every CTA must take it.
__device__ __forceinline__ void cl_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
                 ::: "memory");
}

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// The value at `local` (a shared-memory address of this CTA) in the shared
// memory of cluster CTA `rank`.
__device__ __forceinline__ int32_t cl_read(const int32_t *local, uint32_t rank) {
    uint32_t ra;
    int32_t v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(ra)
                 : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return v;
}

// Warp-aggregated append of the lanes with `pred` to a shared-memory list:
// one shared atomic per warp; entries past `cap` are counted, not stored.
// Called by all 32 lanes.
__device__ __forceinline__ void cta_append(int32_t *q, int32_t *cnt, int32_t cap, int32_t v,
                                           bool pred, int lane) {
    const unsigned mask = __ballot_sync(G2_FULL, pred);
    if (mask == 0) return;
    const int leader = __ffs(mask) - 1;
    int32_t pos = 0;
    if (lane == leader) pos = atomicAdd(cnt, __popc(mask));
    pos = __shfl_sync(G2_FULL, pos, leader) + __popc(mask & lanemask_lt());
    if (pred && pos < cap) q[pos] = v;
}

// The cluster CTA that holds entry i of the concatenated list, where CTA r
// holds entries [off[r], off[r + 1]) (off: the CL + 1 prefix sums of the
// CTAs' list lengths).
template <int CL>
__device__ __forceinline__ int cl_owner(const int32_t *off, int32_t i) {
    int r = 0;
#pragma unroll
    for (int j = 1; j < CL; ++j) r += i >= off[j];
    return r;
}

// The vertices at depth `lvl`, appended to q (the frontier of a level the
// cluster loop could not hold).
static __global__ void k_level_list(const int32_t *depth, int32_t n, int32_t lvl, int32_t *q,
                                    int32_t *cnt, int32_t *err) {
    const int lane = threadIdx.x & 31;
    for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = base + lane;
        const bool p = v < n && depth[v] == lvl;
        warp_append(q, cnt, n, err, (int32_t)v, p);
    }
}

// ------------------------------------------------------------------ host
// Whether one cluster of CL CTAs of `kernel` (kClCta threads, `smem` bytes
// of dynamic shared memory) fits on the current device.
template <class K>
inline bool cluster_fits(K kernel, int CL, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kClCta);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    bool ok = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem) == cudaSuccess;
    if (ok && CL > 8)
        ok = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
             cudaSuccess;
    ok = ok && cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) == cudaSuccess &&
         clusters >= 1;
    cudaGetLastError();
    return ok;
}

// Cluster size for one-cluster loop `slot` (a small id per kernel family) on
// the current device: 16 CTAs where a cluster that large fits, else 8; 0 when
// none fits or G2_FUSED_CLUSTER=0 (read on every call; G2_FUSED_CLUSTER=8 or
// 16 asks for that size).  k16 / k8 are the kernel's two instances.
template <class K16, class K8>
inline int cluster_size(int slot, K16 k16, K8 k8, size_t smem) {
    const char *e = getenv("G2_FUSED_CLUSTER");
    const int want = e ? atoi(e) : -1;
    if (want == 0) return 0;
    constexpr int kMaxDev = 64, kSlots = 8;
    static std::mutex mu;
    static int fits[kMaxDev][kSlots][2];  // 16 / 8 CTAs: 0 unknown, 1 fits, 2 does not
    int dev = 0;
    if (slot < 0 || slot >= kSlots || cudaGetDevice(&dev) != cudaSuccess || dev < 0 ||
        dev >= kMaxDev) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lock(mu);
    int *f = fits[dev][slot];
    if (f[0] == 0) f[0] = cluster_fits(k16, 16, smem) ? 1 : 2;
    if (f[1] == 0) f[1] = cluster_fits(k8, 8, smem) ? 1 : 2;
    if (want != 8 && f[0] == 1) return 16;
    if (want != 16 && f[1] == 1) return 8;
    return 0;
}

// A tuning knob read from the environment on every call.
inline int32_t env_i32(const char *name, int32_t dflt) {
    const char *e = getenv(name);
    return e ? (int32_t)atoi(e) : dflt;
}

// One cluster of CL CTAs of `kernel` on `st`.
template <class K, class A>
inline g2_status launch_cluster(K kernel, int CL, size_t smem, const A &a, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kClCta);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    G2_CK(cudaLaunchKernelEx(&cfg, kernel, a));
    stats().launches += 1;
    return G2_OK;
}

}  // namespace g2
