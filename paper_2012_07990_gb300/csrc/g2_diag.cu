// g2_diag.cu — diagnostics that measure the memory system the kernels run
// on, so that their rooflines can be stated against what this GPU does
// rather than against nominal bandwidth.
//
// g2_diag_gather: one pass of out[t] = sum of x[idx[e]] over the elements a
// thread strides through, with the access shape of the PageRank arc sweep
// (16-byte loads of four consecutive indices per thread, two such quads in
// flight, then their gathers).  Fed with a CSC's column ids it is the share
// gather of a round without the sums per row, the shared-memory cache or the
// atomics: a floor for the sweep on that order of indices.  mode 1 streams
// idx alone (the column bytes, no gather).  The indices are checked in a
// separate pass first; the pass that is timed loads without checks.
#include <cuda_runtime.h>

#include "g2_diag.h"
#include "g2_host.h"

namespace g2 {

__global__ void k_diag_check(const int32_t *idx, int64_t m, uint32_t n, int32_t *bad) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        if ((uint32_t)idx[e] >= n) atomicExch(bad, 1);
}

template <int MODE>
__device__ __forceinline__ float diag_quad(const int4 u, const float *__restrict__ x) {
    if (MODE == 1) return (float)u.x + (float)u.y + (float)u.z + (float)u.w;
    return __ldg(x + u.x) + __ldg(x + u.y) + __ldg(x + u.z) + __ldg(x + u.w);
}

// idx 16-byte aligned; m4 = m / 4 full quads, the tail of m % 4 by thread 0
template <int MODE>
__global__ void __launch_bounds__(256) k_diag_gather(const int32_t *__restrict__ idx,
                                                     const float *__restrict__ x, int64_t m,
                                                     float *out) {
    const int4 *idx4 = reinterpret_cast<const int4 *>(idx);
    const int64_t m4 = m / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.f;
    for (; q + stride < m4; q += 2 * stride) {
        const int4 a = idx4[q], b = idx4[q + stride];
        s += diag_quad<MODE>(a, x) + diag_quad<MODE>(b, x);
    }
    for (; q < m4; q += stride) s += diag_quad<MODE>(idx4[q], x);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t e = m4 * 4; e < m; ++e) s += MODE == 1 ? (float)idx[e] : __ldg(x + idx[e]);
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace g2

using namespace g2;

extern "C" g2_status g2_diag_gather(const int32_t *idx, int64_t m, const float *x, int32_t n,
                                    int32_t mode, float *out, int32_t grid, float *ms,
                                    void *stream) {
    if (!idx || !out || m < 0 || n < 0 || grid < 1 || mode < 0 || mode > 1 ||
        (mode == 0 && !x) || (reinterpret_cast<uintptr_t>(idx) & 15u))
        return fail(G2_EINVAL, "bad g2_diag_gather arguments (idx must be 16-byte aligned)");
    cudaStream_t st = as_stream(stream);
    int32_t *bad = nullptr, h = 0;
    G2_CK(dmalloc(&bad, 4, st));
    cudaError_t e = cudaMemsetAsync(bad, 0, 4, st);
    if (e == cudaSuccess && mode == 0 && m > 0)
        k_diag_check<<<grid, 256, 0, st>>>(idx, m, (uint32_t)n, bad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(bad, st);
    if (e != cudaSuccess) return cuda_fail(e, "g2_diag_gather check");
    if (h) return fail(G2_EINVAL, "index outside [0, n)");
    cudaEvent_t e0, e1;
    G2_CK(cudaEventCreate(&e0));
    G2_CK(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    if (mode == 0) k_diag_gather<0><<<grid, 256, 0, st>>>(idx, x, m, out);
    else k_diag_gather<1><<<grid, 256, 0, st>>>(idx, x, m, out);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "g2_diag_gather");
    if (ms) *ms = t;
    return G2_OK;
}
