/*
 * Seeded synthetic graph generators (input only).
 *
 * This module produces the CSR inputs that both the CPU oracle and the CUDA
 * path consume.  It holds none of the partition-centric method's arithmetic:
 * only random-number generation, edge sampling, sorting, de-duplication and
 * CSR assembly.
 *
 * Random numbers come from splitmix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used counter-style: the n-th
 * draw of a stream with seed s is mix(s + (n + 1) * 0x9E3779B97F4A7C15).
 * Being counter based, every draw is independent of thread scheduling, so the
 * same (seed, sizes) gives the same graph on any host.
 *
 * RMAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each edge descends `scale`
 * levels of the adjacency matrix; at each level it picks quadrant
 * (0,0),(0,1),(1,0),(1,1) with probabilities a, b, c, d = 1-a-b-c.  The
 * paper's RMAT graphs use the generator's default settings and degree 16
 * (evaluation setup, datasets paragraph); defaults here are a/b/c/d =
 * 0.57/0.19/0.19/0.05 and edge factor 16, with self loops and duplicate
 * edges removed and no vertex relabelling.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n-th output (n >= 0) of the splitmix64 stream seeded with `seed`. */
static inline uint64_t sm64_at(uint64_t seed, uint64_t n) {
    return sm64_mix(seed + (n + 1) * GOLDEN);
}

uint64_t gg_splitmix64_at(uint64_t seed, uint64_t n) { return sm64_at(seed, n); }

void gg_splitmix64_fill(uint64_t seed, uint64_t start, uint64_t count, uint64_t *out) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)count; ++i) out[i] = sm64_at(seed, start + (uint64_t)i);
}

/* Edge sampling ------------------------------------------------------------ */

/* Samples `m` RMAT edges of a 2^scale-vertex graph.  Edge i, level j uses the
 * draw with counter i*scale + j; level 0 decides the most significant bit.
 * Quadrant thresholds are compared on the top 53 bits as a double in [0,1). */
void gg_rmat_edges(int scale, uint64_t m, double a, double b, double c,
                   uint64_t seed, uint32_t *src, uint32_t *dst) {
    const double ab = a + b, abc = a + b + c;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)m; ++i) {
        uint32_t u = 0, v = 0;
        uint64_t base = (uint64_t)i * (uint64_t)scale;
        for (int j = 0; j < scale; ++j) {
            double r = (double)(sm64_at(seed, base + (uint64_t)j) >> 11) * (1.0 / 9007199254740992.0);
            uint32_t bit = 1u << (scale - 1 - j);
            if (r < a) {
            } else if (r < ab) {
                v |= bit;
            } else if (r < abc) {
                u |= bit;
            } else {
                u |= bit;
                v |= bit;
            }
        }
        src[i] = u;
        dst[i] = v;
    }
}

/* Samples `m` edges with both endpoints uniform in [0, n): edge i uses draw
 * 2i for the source and 2i+1 for the destination (multiply-shift reduction). */
void gg_uniform_edges(uint32_t n, uint64_t m, uint64_t seed, uint32_t *src, uint32_t *dst) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)m; ++i) {
        uint64_t x = sm64_at(seed, 2 * (uint64_t)i), y = sm64_at(seed, 2 * (uint64_t)i + 1);
        src[i] = (uint32_t)(((x >> 32) * (uint64_t)n) >> 32);
        dst[i] = (uint32_t)(((y >> 32) * (uint64_t)n) >> 32);
    }
}

/* CSR assembly ------------------------------------------------------------- */

static int cmp_u32(const void *x, const void *y) {
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return (a > b) - (a < b);
}

static void sort_u32(uint32_t *p, uint64_t n) {
    /* insertion sort for short rows, qsort otherwise */
    if (n < 32) {
        for (uint64_t i = 1; i < n; ++i) {
            uint32_t x = p[i];
            uint64_t j = i;
            while (j > 0 && p[j - 1] > x) { p[j] = p[j - 1]; --j; }
            p[j] = x;
        }
    } else {
        qsort(p, (size_t)n, sizeof(uint32_t), cmp_u32);
    }
}

/* Builds a CSR over n vertices from m (src, dst) pairs.  Rows are sorted by
 * destination.  If drop_self, self loops are removed; if dedup, repeated
 * (src, dst) pairs are kept once.  If symmetrize, every pair also contributes
 * its reverse.  row_ptr must hold n+1 entries; col must hold m (or 2m when
 * symmetrizing) entries.  Returns the final edge count. */
uint64_t gg_build_csr(uint32_t n, uint64_t m, const uint32_t *src, const uint32_t *dst,
                      int drop_self, int dedup, int symmetrize,
                      uint64_t *row_ptr, uint32_t *col) {
    uint64_t *cnt = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < m; ++i) {
        if (drop_self && src[i] == dst[i]) continue;
        cnt[src[i] + 1]++;
        if (symmetrize) cnt[dst[i] + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    uint64_t *cur = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    memcpy(cur, cnt, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; ++i) {
        if (drop_self && src[i] == dst[i]) continue;
        col[cur[src[i]]++] = dst[i];
        if (symmetrize) col[cur[dst[i]]++] = src[i];
    }
    free(cur);
    /* sort each row, count unique entries */
    uint64_t *keep = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    int64_t v;
#pragma omp parallel for schedule(dynamic, 1024)
    for (v = 0; v < (int64_t)n; ++v) {
        uint64_t b = cnt[v], e = cnt[v + 1];
        sort_u32(col + b, e - b);
        uint64_t k = 0;
        for (uint64_t i = b; i < e; ++i) {
            if (dedup && k > 0 && col[b + k - 1] == col[i]) continue;
            col[b + k++] = col[i];
        }
        keep[v + 1] = k;
    }
    row_ptr[0] = 0;
    for (uint32_t u = 0; u < n; ++u) row_ptr[u + 1] = row_ptr[u] + keep[u + 1];
    /* compact in place: destination offsets never exceed source offsets */
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t b = cnt[u], o = row_ptr[u], k = keep[u + 1];
        if (o != b) memmove(col + o, col + b, (size_t)k * sizeof(uint32_t));
    }
    uint64_t total = row_ptr[n];
    free(cnt);
    free(keep);
    return total;
}

/* Edge weights in [1, hi]: w[e] = 1 + (draw_e mod hi), in CSR order. */
void gg_weights(uint64_t m, uint64_t seed, uint32_t hi, int32_t *w) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)m; ++i) w[i] = (int32_t)(1 + sm64_at(seed, (uint64_t)i) % hi);
}

/* Picks `count` distinct vertices with out-degree >= 1 by rejection from the
 * stream `seed`.  Returns how many were found (fewer only if the graph has
 * fewer such vertices or the draw budget runs out). */
uint32_t gg_roots(uint32_t n, const uint64_t *row_ptr, uint32_t count, uint64_t seed, uint32_t *out) {
    uint32_t found = 0;
    uint64_t draws = 0, budget = 64ull * n + 1024;
    while (found < count && draws < budget) {
        uint32_t v = (uint32_t)(((sm64_at(seed, draws++) >> 32) * (uint64_t)n) >> 32);
        if (row_ptr[v + 1] == row_ptr[v]) continue;
        int dup = 0;
        for (uint32_t i = 0; i < found; ++i) dup |= (out[i] == v);
        if (!dup) out[found++] = v;
    }
    return found;
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
