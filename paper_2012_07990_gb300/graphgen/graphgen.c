/*
 * graphgen.c — seeded synthetic graph generators (RMAT power-law graphs and
 * road-like perturbed 2D grids) and the CSR assembly they need.
 *
 * This module prepares INPUTS only.  It holds none of the traversal
 * arithmetic (no BFS, no relaxation, no PageRank, no blocking); both the CUDA
 * path and the CPU oracle consume what it produces.
 *
 * Random numbers come from one counter-based generator, SplitMix64 (Steele,
 * Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
 * 2014): every draw is a pure function of (seed, stream tag, counter), so the
 * output does not depend on the thread count or the order of work.
 *
 * Output convention: CSR with int32 offsets and ids, adjacency lists sorted
 * ascending, no self-loops, no duplicate arcs.  Arrays are malloc'd here and
 * released with g2gen_free().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* draw(seed, tag, i): 64 random bits for counter i of stream `tag`. */
static inline uint64_t draw(uint64_t seed, uint64_t tag, uint64_t i) {
    return splitmix64(splitmix64(seed ^ (tag * 0xD1B54A32D192ED03ULL)) ^ i);
}

void g2gen_free(void *p) { free(p); }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Assemble a CSR from an arc list (both directions already present when the
 * graph is meant to be symmetric).  Sorts each list, drops self-loops and
 * duplicates.  Returns 0 on success, -1 on allocation failure, -2 if the arc
 * count does not fit int32. */
static int csr_from_arcs(int64_t n, int64_t na, const int32_t *asrc, const int32_t *adst,
                         int32_t **rowptr_out, int32_t **col_out, int64_t *m_out) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t e = 0; e < na; ++e)
        if (asrc[e] != adst[e]) cnt[asrc[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    int64_t total = cnt[n];
    int32_t *tmp = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    int64_t *pos = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!tmp || !pos) { free(cnt); free(tmp); free(pos); return -1; }
    memcpy(pos, cnt, (size_t)(n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < na; ++e)
        if (asrc[e] != adst[e]) tmp[pos[asrc[e]]++] = adst[e];
    free(pos);
    /* sort + unique each list; record the unique length */
    int64_t *ulen = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!ulen) { free(cnt); free(tmp); return -1; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v) {
        int32_t *lst = tmp + cnt[v];
        int64_t len = cnt[v + 1] - cnt[v];
        if (len > 1) qsort(lst, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t k = 0;
        for (int64_t i = 0; i < len; ++i)
            if (k == 0 || lst[i] != lst[k - 1]) lst[k++] = lst[i];
        ulen[v] = k;
    }
    int64_t m = 0;
    for (int64_t v = 0; v < n; ++v) m += ulen[v];
    if (m > 2147483647LL || n > 2147483646LL) { free(cnt); free(tmp); free(ulen); return -2; }
    int32_t *rowptr = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t *col = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!rowptr || !col) { free(cnt); free(tmp); free(ulen); free(rowptr); free(col); return -1; }
    rowptr[0] = 0;
    for (int64_t v = 0; v < n; ++v) rowptr[v + 1] = (int32_t)(rowptr[v] + ulen[v]);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; ++v)
        memcpy(col + rowptr[v], tmp + cnt[v], (size_t)ulen[v] * sizeof(int32_t));
    free(cnt); free(tmp); free(ulen);
    *rowptr_out = rowptr; *col_out = col; *m_out = m;
    return 0;
}

/*
 * RMAT (Chakrabarti, Zhan, Faloutsos 2004).  n = 2^scale vertices,
 * edge_factor * n samples.  Each sample descends `scale` levels of the
 * adjacency matrix, choosing quadrant (0,0),(0,1),(1,0),(1,1) with
 * probability a,b,c,1-a-b-c from 32 random bits per level, most significant
 * bit first.  No vertex-id permutation.  symmetric != 0 adds the reverse of
 * every sample.  Self-loops and duplicates are dropped in CSR assembly.
 */
int g2gen_rmat(int scale, int edge_factor, double a, double b, double c, uint64_t seed,
               int symmetric, int64_t *n_out, int64_t *m_out, int32_t **rowptr, int32_t **col) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -3;
    int64_t n = (int64_t)1 << scale;
    int64_t ns = (int64_t)edge_factor * n;
    int64_t na = symmetric ? 2 * ns : ns;
    int32_t *asrc = (int32_t *)malloc((size_t)na * sizeof(int32_t));
    int32_t *adst = (int32_t *)malloc((size_t)na * sizeof(int32_t));
    if (!asrc || !adst) { free(asrc); free(adst); return -1; }
    const double t1 = a, t2 = a + b, t3 = a + b + c;
    const uint64_t T1 = (uint64_t)(t1 * 4294967296.0);
    const uint64_t T2 = (uint64_t)(t2 * 4294967296.0);
    const uint64_t T3 = (uint64_t)(t3 * 4294967296.0);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ns; ++i) {
        uint32_t u = 0, v = 0;
        uint64_t bits = 0;
        for (int l = 0; l < scale; ++l) {
            if ((l & 1) == 0) bits = draw(seed, 1, (uint64_t)i * 32 + (uint64_t)(l >> 1));
            uint64_t r = (l & 1) ? (bits >> 32) : (bits & 0xFFFFFFFFULL);
            uint32_t bu, bv;
            if (r < T1) { bu = 0; bv = 0; }
            else if (r < T2) { bu = 0; bv = 1; }
            else if (r < T3) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        asrc[i] = (int32_t)u; adst[i] = (int32_t)v;
        if (symmetric) { asrc[ns + i] = (int32_t)v; adst[ns + i] = (int32_t)u; }
    }
    int rc = csr_from_arcs(n, na, asrc, adst, rowptr, col, m_out);
    free(asrc); free(adst);
    *n_out = n;
    return rc;
}

/*
 * Road-like graph: a W x H 4-neighbour lattice (vertex id = y*W + x), each
 * lattice edge deleted independently with probability p_delete, plus
 * `n_shortcuts` local shortcuts u -> u + (dx, dy) with dx, dy uniform in
 * [-reach, reach] (clamped to the grid; a shortcut that lands on u is
 * skipped).  Always symmetric.
 */
int g2gen_grid(int W, int H, double p_delete, int64_t n_shortcuts, int reach, uint64_t seed,
               int64_t *n_out, int64_t *m_out, int32_t **rowptr, int32_t **col) {
    if (W < 1 || H < 1 || reach < 0) return -3;
    int64_t n = (int64_t)W * H;
    int64_t nh = (int64_t)(W - 1) * H, nv = (int64_t)W * (H - 1);
    int64_t cap = 2 * (nh + nv + n_shortcuts);
    int32_t *asrc = (int32_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    int32_t *adst = (int32_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    if (!asrc || !adst) { free(asrc); free(adst); return -1; }
    /* lattice edges: ids [0, nh) horizontal, [nh, nh+nv) vertical */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nh + nv; ++e) {
        int64_t u, v;
        if (e < nh) { int64_t y = e / (W - 1), x = e % (W - 1); u = y * W + x; v = u + 1; }
        else { int64_t k = e - nh; u = k; v = k + W; }
        int keep = (double)(draw(seed, 2, (uint64_t)e) >> 11) * 0x1.0p-53 >= p_delete;
        asrc[2 * e] = keep ? (int32_t)u : 0;  adst[2 * e] = keep ? (int32_t)v : 0;
        asrc[2 * e + 1] = keep ? (int32_t)v : 0; adst[2 * e + 1] = keep ? (int32_t)u : 0;
    }
    int64_t base = 2 * (nh + nv);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_shortcuts; ++j) {
        uint64_t r0 = draw(seed, 3, (uint64_t)j);
        uint64_t r1 = draw(seed, 4, (uint64_t)j);
        int64_t u = (int64_t)(r0 % (uint64_t)n);
        int64_t x = u % W, y = u / W;
        int64_t dx = (int64_t)((r1 & 0xFFFFFFFFULL) % (uint64_t)(2 * reach + 1)) - reach;
        int64_t dy = (int64_t)((r1 >> 32) % (uint64_t)(2 * reach + 1)) - reach;
        int64_t x2 = x + dx, y2 = y + dy;
        if (x2 < 0) x2 = 0;
        if (x2 >= W) x2 = W - 1;
        if (y2 < 0) y2 = 0;
        if (y2 >= H) y2 = H - 1;
        int64_t v = y2 * W + x2;
        /* a skipped shortcut is written as a self-loop, dropped in assembly */
        asrc[base + 2 * j] = (int32_t)u; adst[base + 2 * j] = (int32_t)v;
        asrc[base + 2 * j + 1] = (int32_t)v; adst[base + 2 * j + 1] = (int32_t)u;
    }
    int rc = csr_from_arcs(n, cap, asrc, adst, rowptr, col, m_out);
    free(asrc); free(adst);
    *n_out = n;
    return rc;
}

/*
 * Edge weights: w({u,v}) = 1 + draw(seed, 5, min*n + max) mod wmax, a pure
 * function of the unordered pair, so both arcs of an undirected edge carry the
 * same weight whatever order the arcs are stored in.
 */
void g2gen_pair_weights(int64_t n, const int32_t *rowptr, const int32_t *col, uint64_t seed,
                        int32_t wmax, int32_t *w) {
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            int64_t v = col[e];
            int64_t lo = u < v ? u : v, hi = u < v ? v : u;
            w[e] = (int32_t)(1 + draw(seed, 5, (uint64_t)(lo * n + hi)) % (uint64_t)wmax);
        }
    }
}

/* CSR assembly from a caller-supplied arc list (used for small hand-made and
 * random test graphs). */
int g2gen_csr_from_arcs(int64_t n, int64_t na, const int32_t *asrc, const int32_t *adst,
                        int64_t *m_out, int32_t **rowptr, int32_t **col) {
    return csr_from_arcs(n, na, asrc, adst, rowptr, col, m_out);
}

int g2gen_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
