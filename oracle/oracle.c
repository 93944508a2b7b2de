/*
 * oracle.c — plain, slow, obviously-correct CPU reference for the g2
 * frontier-traversal path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this file's library.  It
 * shares no code, header, table or helper with the CUDA path.  Single thread,
 * no blocking or fusion: each function is the textbook definition or the
 * paper's algorithm written out step by step.
 *
 * Graph input everywhere: CSR, int32 rowptr[n+1] and col[m]; arcs u->v for
 * col[rowptr[u] .. rowptr[u+1]-1].
 *
 * Functions and what they follow:
 *   oracle_bfs        BFS of the paper's Fig. 2 program (Sec. IV): hop depth,
 *                     and the parent array with the canonical reading
 *                     "minimum-id in-neighbour one level up" (the paper's
 *                     parent is any winner of the compare-and-swap race).
 *   oracle_cc         connected components (Sec. VII, the Soman et al. CC):
 *                     label = minimum vertex id of the component, computed by
 *                     union-find over the undirected edges.
 *   oracle_sssp       single-source shortest paths (Sec. VII, delta-stepping):
 *                     the exact distances, computed by Dijkstra's algorithm;
 *                     delta-stepping reaches the same distances for any delta.
 *   oracle_pagerank   PageRank (Sec. VII, topology-driven, fixed rounds):
 *                     power iteration with uniform redistribution of the mass
 *                     of vertices without out-arcs, fp64.
 *   oracle_bc         betweenness centrality (Sec. VII): Brandes' dependency
 *                     accumulation summed over the given sources, path counts
 *                     in long double, no normalisation or halving.
 *   oracle_edgeblock  EdgeBlocking preprocessing, Algorithm 1 (Sec. VI-D).
 *   oracle_etwc_split the per-vertex three-way edge split of Algorithm 3
 *                     (Sec. VI-D, ETWC).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ENOMEM 1
#define ORACLE_EOVERFLOW 2

/* ---------------------------------------------------------------- BFS ---- */
/* depth[v] = number of arcs on a shortest path src -> v, -1 if unreachable.
 * parent[v] (optional) = smallest u with an arc u->v and depth[u] = depth[v]-1;
 * parent[src] = src; -1 if unreachable. */
int oracle_bfs(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t src,
               int32_t *depth, int32_t *parent) {
    int32_t *queue = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!queue) return ORACLE_ENOMEM;
    for (int32_t v = 0; v < n; ++v) depth[v] = -1;
    int32_t head = 0, tail = 0;
    depth[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (depth[v] == -1) {
                depth[v] = depth[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    if (parent) {
        for (int32_t v = 0; v < n; ++v) parent[v] = -1;
        parent[src] = src;
        for (int32_t u = 0; u < n; ++u) {
            if (depth[u] < 0) continue;
            for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                int32_t v = col[e];
                if (v == src || depth[v] != depth[u] + 1) continue;
                if (parent[v] == -1 || u < parent[v]) parent[v] = u;
            }
        }
    }
    return ORACLE_OK;
}

/* ----------------------------------------------------------------- CC ---- */
static int32_t uf_find(int32_t *p, int32_t x) {
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

/* label[v] = min vertex id in v's connected component, arcs taken as
 * undirected edges. */
int oracle_cc(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t *label) {
    for (int32_t v = 0; v < n; ++v) label[v] = v;
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            int32_t a = uf_find(label, u), b = uf_find(label, col[e]);
            if (a == b) continue;
            /* the root of every set is its smallest member */
            if (a < b) label[b] = a;
            else label[a] = b;
        }
    }
    for (int32_t v = 0; v < n; ++v) label[v] = uf_find(label, v);
    return ORACLE_OK;
}

/* --------------------------------------------------------------- SSSP ---- */
typedef struct { int64_t d; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *size, heap_item x) {
    int64_t i = (*size)++;
    h[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, int64_t *size) {
    heap_item top = h[0];
    h[0] = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *size && h[l].d < h[s].d) s = l;
        if (r < *size && h[r].d < h[s].d) s = r;
        if (s == i) break;
        heap_item t = h[s]; h[s] = h[i]; h[i] = t;
        i = s;
    }
    return top;
}

/* dist[v] = min over src->v paths of the sum of arc weights (w >= 1);
 * INT32_MAX if unreachable.  Returns ORACLE_EOVERFLOW if a finite distance
 * does not fit below INT32_MAX. */
int oracle_sssp(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *w,
                int32_t src, int32_t *dist) {
    int64_t m = rowptr[n];
    int64_t *d = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    heap_item *h = (heap_item *)malloc((size_t)(m + 1) * sizeof(heap_item));
    char *done = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!d || !h || !done) { free(d); free(h); free(done); return ORACLE_ENOMEM; }
    const int64_t INF = INT64_MAX;
    for (int32_t v = 0; v < n; ++v) d[v] = INF;
    int64_t hs = 0;
    d[src] = 0;
    heap_push(h, &hs, (heap_item){0, src});
    while (hs > 0) {
        heap_item it = heap_pop(h, &hs);
        int32_t u = it.v;
        if (done[u]) continue;
        done[u] = 1;
        for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            int32_t v = col[e];
            int64_t nd = d[u] + (int64_t)w[e];
            if (nd < d[v]) {
                d[v] = nd;
                heap_push(h, &hs, (heap_item){nd, v});
            }
        }
    }
    int rc = ORACLE_OK;
    for (int32_t v = 0; v < n; ++v) {
        if (d[v] == INF) dist[v] = INT32_MAX;
        else if (d[v] >= INT32_MAX) { dist[v] = INT32_MAX; rc = ORACLE_EOVERFLOW; }
        else dist[v] = (int32_t)d[v];
    }
    free(d); free(h); free(done);
    return rc;
}

/* ----------------------------------------------------------- PageRank ---- */
/* x^0 = 1/n; for t = 1..iters:
 *   D = sum of x^{t-1}[u] over u with no out-arc,
 *   x^t[v] = (1-damping)/n + damping * ( sum_{u->v} x^{t-1}[u]/outdeg(u) + D/n ).
 * Output x^iters. */
int oracle_pagerank(int32_t n, const int32_t *rowptr, const int32_t *col, double damping,
                    int32_t iters, double *x) {
    double *y = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!y) return ORACLE_ENOMEM;
    for (int32_t v = 0; v < n; ++v) x[v] = 1.0 / n;
    for (int32_t t = 0; t < iters; ++t) {
        double D = 0.0;
        for (int32_t u = 0; u < n; ++u)
            if (rowptr[u + 1] == rowptr[u]) D += x[u];
        for (int32_t v = 0; v < n; ++v) y[v] = 0.0;
        for (int32_t u = 0; u < n; ++u) {
            int32_t deg = rowptr[u + 1] - rowptr[u];
            if (deg == 0) continue;
            double share = x[u] / deg;
            for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) y[col[e]] += share;
        }
        for (int32_t v = 0; v < n; ++v) x[v] = (1.0 - damping) / n + damping * (y[v] + D / n);
    }
    free(y);
    return ORACLE_OK;
}

/* ----------------------------------------------------------------- BC ---- */
/* bc[v] = sum over sources s of delta_s(v), with
 *   delta_s(v) = sum over w with v->w and depth_s(w) = depth_s(v)+1 of
 *                sigma_s(v)/sigma_s(w) * (1 + delta_s(w)),
 * sigma_s = number of shortest s->v paths, delta_s(s) not added.
 * (Brandes, "A faster algorithm for betweenness centrality", 2001.) */
int oracle_bc(int32_t n, const int32_t *rowptr, const int32_t *col, const int32_t *srcs,
              int32_t k, double *bc) {
    int32_t *depth = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *order = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    long double *sigma = (long double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(long double));
    long double *delta = (long double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(long double));
    long double *acc = (long double *)calloc((size_t)(n > 0 ? n : 1), sizeof(long double));
    if (!depth || !order || !sigma || !delta || !acc) {
        free(depth); free(order); free(sigma); free(delta); free(acc);
        return ORACLE_ENOMEM;
    }
    for (int32_t i = 0; i < k; ++i) {
        int32_t s = srcs[i];
        for (int32_t v = 0; v < n; ++v) { depth[v] = -1; sigma[v] = 0.0L; delta[v] = 0.0L; }
        int32_t head = 0, tail = 0;
        depth[s] = 0; sigma[s] = 1.0L; order[tail++] = s;
        while (head < tail) {
            int32_t u = order[head++];
            for (int32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
                int32_t v = col[e];
                if (depth[v] == -1) { depth[v] = depth[u] + 1; order[tail++] = v; }
                if (depth[v] == depth[u] + 1) sigma[v] += sigma[u];
            }
        }
        for (int32_t j = tail - 1; j >= 0; --j) {
            int32_t v = order[j];
            long double dv = 0.0L;
            for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int32_t w = col[e];
                if (depth[w] == depth[v] + 1) dv += sigma[v] / sigma[w] * (1.0L + delta[w]);
            }
            delta[v] = dv;
            if (v != s) acc[v] += dv;
        }
    }
    for (int32_t v = 0; v < n; ++v) bc[v] = (double)acc[v];
    free(depth); free(order); free(sigma); free(delta); free(acc);
    return ORACLE_OK;
}

/* --------------------------------------------------- EdgeBlocking (Alg. 1) */
/* Input: COO edges (src[e], dst[e]) for e < m, n vertices, N vertices per
 * segment.  Output: the edges regrouped by segment floor(dst/N), keeping
 * their input order inside a segment (out_src, out_dst), and the array the
 * algorithm leaves in its prefix-sum variable: seg_end[s] = one past the last
 * output index of segment s, for s < numberOfSegments, and seg_end[numSeg] =
 * m.  Returns the number of segments. */
int32_t oracle_edgeblock(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int32_t N,
                         int32_t *out_src, int32_t *out_dst, int64_t *seg_end) {
    int32_t num_seg = (n + N - 1) / N;
    int64_t *segment_size = (int64_t *)calloc((size_t)num_seg + 1, sizeof(int64_t));
    if (!segment_size) return -1;
    /* first pass: count the edges of each subgraph */
    for (int64_t e = 0; e < m; ++e) segment_size[dst[e] / N] += 1;
    /* exclusive prefix sum: the start of each subgraph */
    int64_t run = 0;
    for (int32_t s = 0; s <= num_seg; ++s) {
        int64_t c = segment_size[s];
        seg_end[s] = run;
        run += c;
    }
    /* second pass: place every edge, advancing its subgraph's cursor */
    for (int64_t e = 0; e < m; ++e) {
        int32_t s = dst[e] / N;
        int64_t idx = seg_end[s];
        out_src[idx] = src[e];
        out_dst[idx] = dst[e];
        seg_end[s] = idx + 1;
    }
    free(segment_size);
    return num_seg;
}

/* ------------------------------------------------ ETWC split (Alg. 3) ---- */
/* The three queue entries ETWC makes from one frontier vertex whose arcs are
 * [start, end): a chunk that is a multiple of the CTA granularity `cta`, then
 * a multiple of the warp granularity `warp`, then the rest.  ranges[2*i],
 * ranges[2*i+1] = [begin, end) of stage i (i = 0 thread, 1 warp, 2 CTA); an
 * empty stage has begin == end. */
void oracle_etwc_split(int64_t start, int64_t end, int32_t warp, int32_t cta, int64_t *ranges) {
    int64_t size = end - start;
    int64_t pos = start;
    int64_t cta_part = (size / cta) * cta;
    ranges[4] = pos; ranges[5] = pos + cta_part;
    pos += cta_part; size -= cta_part;
    int64_t warp_part = (size / warp) * warp;
    ranges[2] = pos; ranges[3] = pos + warp_part;
    pos += warp_part; size -= warp_part;
    ranges[0] = pos; ranges[1] = size > 0 ? end : pos;
}
