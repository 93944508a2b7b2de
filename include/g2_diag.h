/*
 * g2_diag.h — measurement probes of libg2.so that are not part of the
 * traversal library: they time access patterns of its kernels on their own,
 * to find the floor a kernel runs against.  Same conventions as g2.h.
 */
#ifndef G2_DIAG_H
#define G2_DIAG_H

#include <stdint.h>

#include "g2.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Diagnostic: one pass of out[t] = sum of x[idx[e]] over the elements e
 * thread t of a grid of `grid` CTAs x 256 threads strides through, with the
 * access shape of the PageRank arc sweep (16-byte loads of four consecutive
 * indices, two quads in flight per thread) (mode 0), or of the idx values
 * alone (mode 1: streams idx, no gather).  idx int32[m] (16-byte aligned),
 * x float[n] and out float[grid * 256] are device arrays; every idx must lie
 * in [0, n): a checking pass runs first and returns G2_EINVAL before any
 * gather.  *ms (host, may be NULL) receives the gather pass's device time
 * from CUDA events on `stream`.  Fed with a CSC's column ids it is the share
 * gather of a PageRank round without sums, cache or atomics: a floor for the
 * arc sweep on that index order.  Synchronises `stream` before returning. */
g2_status g2_diag_gather(const int32_t *idx, int64_t m, const float *x, int32_t n, int32_t mode,
                         float *out, int32_t grid, float *ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* G2_DIAG_H */
