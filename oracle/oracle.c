/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, serial, obviously-correct CPU implementations of what the GPOP
 * scatter/gather path computes (Lakhotia et al., "GPOP: A cache- and
 * memory-efficient framework for Graph Processing Over Partitions").  Only the
 * test suite, the smoke check and the bench's CPU-baseline leg may load this
 * file; the CUDA library never links or calls it, and the two share no code.
 *
 * Floating point is FP64 throughout.  Two tiers:
 *
 *  Tier 1 -- plain definitions that the bulk-synchronous method reaches
 *            exactly (BFS/CC/SSSP) or up to rounding order (PageRank/PPR):
 *              orc_pagerank   Alg. 6 (PageRank user functions) written as the
 *                             power iteration it performs, sinks not redistributed
 *              orc_ppr        seeded personalised PageRank (restart alpha) in
 *                             the same form, seed re-injected every iteration
 *              orc_nibble     parallel Nibble (Alg. 4): its user functions run
 *                             in Alg. 2's order; an approximation (eps
 *                             truncation), so this follows the algorithm's steps
 *              orc_bfs        queue BFS (Alg. 5 computes a BFS tree); parent =
 *                             minimum-ID in-neighbour one level up
 *              orc_cc         union-find; label = minimum vertex ID of the
 *                             component (fixed point of label propagation, Sec. 5 CC)
 *              orc_sssp       Dijkstra with a binary heap (Alg. 7 reaches the
 *                             same fixed point by Bellman-Ford)
 *
 *  Tier 2 -- orc_gpop: the serial GPOP engine following Alg. 2 (scatter,
 *            reInit, gather, filter), Alg. 3 (partition-centric scatter over
 *            the PNG layout) and Eq. (mode) (Sec. 3.2) step by step, with
 *            index partitions of P consecutive vertices (Sec. 3.1.1), bins
 *            bin[p][q] holding (value, id list) messages (Sec. 3.1.2).
 *            It records per-iteration frontier sizes and per-partition modes.
 *
 * Readings of points the paper leaves open (each also in the design notes):
 *  - a partition-centric message from an inactive source carries NULL and the
 *    gather ignores it (Sec. 3.1.2 says all of V^p is scattered but never how
 *    gather treats inactive senders);
 *  - BFS parent = smallest candidate among the messages of the discovering
 *    iteration (Alg. 5's "first message wins" is order dependent);
 *  - the "r" without superscript in Eq. (PC) is r^p;
 *  - Eq. (mode) ties go to PC ("<="), evaluated exactly in integers;
 *  - a partition with no active vertex or no out-edge is not scattered.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

#define U32_INF 0xFFFFFFFFu
#define U64_INF 0xFFFFFFFFFFFFFFFFull

/* ------------------------------------------------------------------------ */
/* Tier 1                                                                    */
/* ------------------------------------------------------------------------ */

/* PageRank as Alg. 6 computes it: x_0 = 1/n, and each iteration
 *   x_{t+1}[v] = (1-d)/n + d * sum_{u->v} x_t[u] / outdeg(u).
 * Sinks scatter nothing, so their mass is dropped (no redistribution).
 * Stops after max_iters iterations, or earlier once sum_v |x_{t+1}-x_t| < tol.
 * res_hist (optional, max_iters entries) receives each iteration's L1 change. */
int orc_pagerank(uint32_t n, const uint64_t *rp, const uint32_t *col, double d,
                 uint32_t max_iters, double tol, double *x, uint32_t *iters_out,
                 double *res_out, double *res_hist) {
    double *y = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!y) return -1;
    for (uint32_t v = 0; v < n; ++v) x[v] = 1.0 / n;
    uint32_t t = 0;
    double res = 0.0;
    while (t < max_iters) {
        for (uint32_t v = 0; v < n; ++v) y[v] = 0.0;
        for (uint32_t u = 0; u < n; ++u) {
            uint64_t deg = rp[u + 1] - rp[u];
            if (deg == 0) continue;
            double share = x[u] / (double)deg;
            for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) y[col[e]] += share;
        }
        res = 0.0;
        for (uint32_t v = 0; v < n; ++v) {
            double nx = (1.0 - d) / n + d * y[v];
            res += fabs(nx - x[v]);
            x[v] = nx;
        }
        if (res_hist) res_hist[t] = res;
        ++t;
        if (res < tol) break;
    }
    free(y);
    if (iters_out) *iters_out = t;
    if (res_out) *res_out = res;
    return 0;
}

/* Seeded personalised PageRank with restart probability alpha:
 *   x_0 = e_s,  x_{t+1}[v] = alpha*[v==s] + (1-alpha) * sum_{u->v} x_t[u]/outdeg(u).
 * Same stopping rule as orc_pagerank. */
int orc_ppr(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t s, double alpha,
            uint32_t max_iters, double tol, double *x, uint32_t *iters_out, double *res_out) {
    double *y = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (!y || s >= n) { free(y); return -1; }
    for (uint32_t v = 0; v < n; ++v) x[v] = 0.0;
    x[s] = 1.0;
    uint32_t t = 0;
    double res = 0.0;
    while (t < max_iters) {
        for (uint32_t v = 0; v < n; ++v) y[v] = 0.0;
        for (uint32_t u = 0; u < n; ++u) {
            uint64_t deg = rp[u + 1] - rp[u];
            if (deg == 0 || x[u] == 0.0) continue;
            double share = x[u] / (double)deg;
            for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) y[col[e]] += share;
        }
        res = 0.0;
        for (uint32_t v = 0; v < n; ++v) {
            double nx = (v == s ? alpha : 0.0) + (1.0 - alpha) * y[v];
            res += fabs(nx - x[v]);
            x[v] = nx;
        }
        ++t;
        if (res < tol) break;
    }
    free(y);
    if (iters_out) *iters_out = t;
    if (res_out) *res_out = res;
    return 0;
}

/* Parallel Nibble (Alg. 4) run through the bulk-synchronous flow of Alg. 2,
 * in FP64.  PR starts as the indicator of the seed s and the frontier is {s}.
 * Each iteration, in the paper's order:
 *   scatter  every frontier vertex v sends PR[v] / (2 deg v) along each out-edge
 *            (scatterFunc; the values are read before initFunc changes them);
 *   initFunc every frontier vertex keeps half its PR (update1) and stays on
 *            (cond1) iff PR[v] >= eps * deg v;
 *   gather   every message adds its value to PR of its destination (gatherFunc),
 *            which is thereby activated;
 *   filter   the next frontier is every vertex that stayed on or was activated
 *            and has PR[v] >= eps * deg v (cond2).
 * Reading for sinks: the paper's test is PR >= eps * 0, always true, which would
 * keep a reached sink on forever while it sends nothing; here a sink is never
 * kept (cond1 and cond2 also require deg v > 0).
 * Stops when the frontier is empty or after max_iters iterations.  frontier_out
 * (optional, max_iters entries) receives the frontier size entering each
 * iteration. */
int orc_nibble(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t s, double eps,
               uint32_t max_iters, double *pr, uint32_t *iters_out, uint64_t *frontier_out) {
    if (s >= n) return -1;
    double *msg = (double *)calloc(n, sizeof(double));
    uint8_t *front = (uint8_t *)calloc(n, 1), *nfront = (uint8_t *)calloc(n, 1), *recv = (uint8_t *)calloc(n, 1);
    if (!msg || !front || !nfront || !recv) { free(msg); free(front); free(nfront); free(recv); return -1; }
    for (uint32_t v = 0; v < n; ++v) pr[v] = 0.0;
    pr[s] = 1.0;
    front[s] = 1;
    uint64_t nf = 1;
    uint32_t t = 0;
    while (nf > 0 && t < max_iters) {
        if (frontier_out) frontier_out[t] = nf;
        for (uint32_t v = 0; v < n; ++v) { msg[v] = 0.0; recv[v] = 0; nfront[v] = 0; }
        /* scatter */
        for (uint32_t v = 0; v < n; ++v) {
            if (!front[v]) continue;
            uint64_t deg = rp[v + 1] - rp[v];
            for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
                msg[col[e]] += pr[v] / (2.0 * (double)deg);
                recv[col[e]] = 1;
            }
        }
        /* initFunc on the frontier */
        for (uint32_t v = 0; v < n; ++v) {
            if (!front[v]) continue;
            uint64_t deg = rp[v + 1] - rp[v];
            pr[v] = pr[v] / 2.0;
            nfront[v] = deg > 0 && pr[v] >= eps * (double)deg;
        }
        /* gather, then filter over the kept and the activated vertices */
        nf = 0;
        for (uint32_t v = 0; v < n; ++v) {
            if (recv[v]) pr[v] += msg[v];
            if (nfront[v] || recv[v]) {
                uint64_t deg = rp[v + 1] - rp[v];
                nfront[v] = deg > 0 && pr[v] >= eps * (double)deg;
            }
            nf += nfront[v];
        }
        uint8_t *tmp = front; front = nfront; nfront = tmp;
        ++t;
    }
    free(msg); free(front); free(nfront); free(recv);
    if (iters_out) *iters_out = t;
    return 0;
}

/* Breadth-first search over out-edges from root with a FIFO queue.
 * level[v] = hop distance (U32_INF if unreached).  parent[root] = root and,
 * for every other reached v, parent[v] = the smallest u with an edge u->v and
 * level[u] = level[v]-1 (U32_INF if unreached). */
int orc_bfs(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t root,
            uint32_t *level, uint32_t *parent) {
    if (root >= n) return -1;
    uint32_t *queue = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!queue) return -1;
    for (uint32_t v = 0; v < n; ++v) { level[v] = U32_INF; parent[v] = U32_INF; }
    uint64_t head = 0, tail = 0;
    level[root] = 0;
    queue[tail++] = root;
    while (head < tail) {
        uint32_t u = queue[head++];
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
            uint32_t v = col[e];
            if (level[v] == U32_INF) { level[v] = level[u] + 1; queue[tail++] = v; }
        }
    }
    for (uint32_t u = 0; u < n; ++u) {
        if (level[u] == U32_INF) continue;
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
            uint32_t v = col[e];
            if (v != root && level[v] == level[u] + 1 && u < parent[v]) parent[v] = u;
        }
    }
    parent[root] = root;
    free(queue);
    return 0;
}

static uint32_t uf_find(uint32_t *up, uint32_t v) {
    while (up[v] != v) { up[v] = up[up[v]]; v = up[v]; }
    return v;
}

/* Connected components of the graph with edge directions ignored, by
 * union-find.  Roots are always the smaller ID, so label[v] = min ID in v's
 * component. */
int orc_cc(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t *label) {
    uint32_t *up = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!up) return -1;
    for (uint32_t v = 0; v < n; ++v) up[v] = v;
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
            uint32_t a = uf_find(up, u), b = uf_find(up, col[e]);
            if (a < b) up[b] = a;
            else if (b < a) up[a] = b;
        }
    }
    for (uint32_t v = 0; v < n; ++v) label[v] = uf_find(up, v);
    free(up);
    return 0;
}

/* Single-source shortest paths over out-edges with non-negative integer
 * weights: Dijkstra with a binary heap and lazy deletion.  dist in uint64;
 * unreachable = U64_INF. */
typedef struct { uint64_t d; uint32_t v; } heap_item;

static void heap_push(heap_item *h, uint64_t *sz, heap_item it) {
    uint64_t i = (*sz)++;
    h[i] = it;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h[p].d <= h[i].d) break;
        heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, uint64_t *sz) {
    heap_item top = h[0];
    h[0] = h[--(*sz)];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *sz && h[l].d < h[m].d) m = l;
        if (r < *sz && h[r].d < h[m].d) m = r;
        if (m == i) break;
        heap_item t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

int orc_sssp(uint32_t n, const uint64_t *rp, const uint32_t *col, const int32_t *w,
             uint32_t root, uint64_t *dist) {
    if (root >= n) return -1;
    uint64_t m = rp[n];
    heap_item *h = (heap_item *)malloc(sizeof(heap_item) * (m + 1));
    if (!h) return -1;
    for (uint32_t v = 0; v < n; ++v) dist[v] = U64_INF;
    uint64_t sz = 0;
    dist[root] = 0;
    heap_push(h, &sz, (heap_item){0, root});
    while (sz) {
        heap_item it = heap_pop(h, &sz);
        if (it.d != dist[it.v]) continue;
        for (uint64_t e = rp[it.v]; e < rp[it.v + 1]; ++e) {
            if (w[e] < 0) { free(h); return -2; }
            uint64_t nd = it.d + (uint64_t)w[e];
            if (nd < dist[col[e]]) { dist[col[e]] = nd; heap_push(h, &sz, (heap_item){nd, col[e]}); }
        }
    }
    free(h);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. (mode) -- Sec. 3.2                                                     */
/* ------------------------------------------------------------------------ */

/* Returns 2 (PC), 1 (SC) or 0 (not scattered) for one partition.
 * Sec. 3.2 with s_i = s_v = 4 bytes:
 *   SC traffic = (V_a + E_a) s_i + 2 (r^p E_a s_v + E_a s_i)
 *   PC traffic = r^p E^p s_i + k s_i + 2 r^p E^p s_v + E^p s_i
 * and PC is chosen iff PC / BW_PC <= SC / BW_SC, with BW_PC / BW_SC = num/den.
 * r^p E^p is the number of PNG entries n_png of p, so multiplying both sides
 * by E^p (and dividing out the common factor 4) makes the test exact:
 *   den * E^p * (n_png + k + 2 n_png + E^p) <= num * (V_a E^p + 3 E_a E^p + 2 n_png E_a). */
int orc_mode_decide(uint64_t k, uint64_t Ep, uint64_t npng, uint64_t Va, uint64_t Ea,
                    uint32_t num, uint32_t den) {
    if (Va == 0 || Ep == 0) return 0;
    u128 pc = (u128)den * Ep * (u128)(npng + k + 2 * npng + Ep);
    u128 sc = (u128)num * ((u128)Va * Ep + (u128)3 * Ea * Ep + (u128)2 * npng * Ea);
    return pc <= sc ? 2 : 1;
}

/* Model bytes of a partition's chosen mode (Sec. 3.2, s_i = s_v = 4), as a
 * double because r^p E_a is fractional in the SC formula. */
double orc_mode_bytes(int mode, uint64_t k, uint64_t Ep, uint64_t npng, uint64_t Va, uint64_t Ea) {
    if (mode == 2) return 4.0 * (double)(npng + k + 2 * npng + Ep);
    if (mode == 1) {
        double r = Ep ? (double)npng / (double)Ep : 0.0;
        return 4.0 * ((double)Va + 3.0 * (double)Ea + 2.0 * r * (double)Ea);
    }
    return 0.0;
}

/* Per-partition static quantities of the index partitioning (Sec. 3.1.1-3.1.2):
 * partition p holds vertices [pP, (p+1)P); E^p = out-edges of p;
 * n_png^p = sum over v in p of its out-partition-degree (distinct destination
 * partitions), i.e. r^p E^p. */
int orc_partition_stats(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t P,
                        uint64_t *Ep, uint64_t *npng) {
    if (P == 0) return -1;
    uint64_t k = ((uint64_t)n + P - 1) / P;
    for (uint64_t p = 0; p < k; ++p) { Ep[p] = 0; npng[p] = 0; }
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t p = v / P;
        Ep[p] += rp[v + 1] - rp[v];
        /* count distinct destination partitions of v (rows need not be sorted) */
        for (uint64_t e = rp[v]; e < rp[v + 1]; ++e) {
            uint64_t q = col[e] / P;
            int seen = 0;
            for (uint64_t f = rp[v]; f < e; ++f) if (col[f] / P == q) { seen = 1; break; }
            if (!seen) npng[p]++;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tier 2 -- serial GPOP engine (Alg. 2, Alg. 3, Eq. (mode))                 */
/* ------------------------------------------------------------------------ */

enum { ALG_PAGERANK = 0, ALG_BFS = 1, ALG_CC = 2, ALG_SSSP = 3, ALG_PPR = 4 };
enum { POL_ANALYTIC = 0, POL_FORCE_SC = 2, POL_FORCE_PC = 3 };

/* One edge of the PNG ordering: sorted by (p, q, source, destination). */
typedef struct { uint32_t p, q, u, v; int32_t w; } png_edge;

static int cmp_png_edge(const void *a, const void *b) {
    const png_edge *x = (const png_edge *)a, *y = (const png_edge *)b;
    if (x->p != y->p) return x->p < y->p ? -1 : 1;
    if (x->q != y->q) return x->q < y->q ? -1 : 1;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

/* A message in a bin: one source value plus the destination ids (and, for
 * weighted graphs, their edge weights) it carries. */
typedef struct { double fval; uint64_t ival; int null_msg; uint64_t id_beg, id_end; } message;

typedef struct {
    uint32_t n, P, k, algo, src;
    double d;                 /* PageRank damping, or 1 - restart for PPR */
    const uint64_t *rp;
    /* static PNG layout: edges grouped into bins (p,q), messages per source */
    png_edge *pe;             /* E entries sorted by (p,q,u,v) */
    uint64_t nbins;
    uint32_t *bin_p, *bin_q;  /* per bin */
    uint64_t *bin_e0, *bin_e1;/* edge range of each bin in pe */
    uint64_t *row_bin0;       /* first bin of each partition (k+1) */
    uint64_t *col_bin_cnt;    /* bins of each column (k+1 prefix) */
    uint64_t *col_bins;       /* bin ids grouped by q, ascending p */
    uint64_t *Ep, *npng;      /* per partition */
} gpop_t;

/* Vertex state of the applications (Alg. 4-7 and the CC / PPR readings). */
typedef struct {
    double *x;                /* PageRank / PPR */
    uint64_t *val;            /* BFS parent, SSSP distance, CC label */
    uint32_t *level;          /* BFS level */
    uint8_t *active, *next;   /* frontier flags */
} state_t;

static int gpop_layout(gpop_t *g, uint32_t n, const uint64_t *rp, const uint32_t *col,
                       const int32_t *w, uint32_t P) {
    uint64_t m = rp[n];
    g->n = n; g->P = P; g->rp = rp;
    g->k = (uint32_t)(((uint64_t)n + P - 1) / P);
    g->pe = (png_edge *)malloc(sizeof(png_edge) * (m ? m : 1));
    if (!g->pe) return -1;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = rp[u]; e < rp[u + 1]; ++e) {
            png_edge x = { u / P, col[e] / P, u, col[e], w ? w[e] : 0 };
            g->pe[e] = x;
        }
    qsort(g->pe, (size_t)m, sizeof(png_edge), cmp_png_edge);
    /* bins = maximal runs of equal (p,q) */
    uint64_t nb = 0;
    for (uint64_t e = 0; e < m; ++e)
        if (e == 0 || g->pe[e].p != g->pe[e - 1].p || g->pe[e].q != g->pe[e - 1].q) ++nb;
    g->nbins = nb;
    g->bin_p = (uint32_t *)malloc(sizeof(uint32_t) * (nb + 1));
    g->bin_q = (uint32_t *)malloc(sizeof(uint32_t) * (nb + 1));
    g->bin_e0 = (uint64_t *)malloc(sizeof(uint64_t) * (nb + 1));
    g->bin_e1 = (uint64_t *)malloc(sizeof(uint64_t) * (nb + 1));
    g->row_bin0 = (uint64_t *)calloc(g->k + 1, sizeof(uint64_t));
    g->col_bin_cnt = (uint64_t *)calloc(g->k + 1, sizeof(uint64_t));
    g->col_bins = (uint64_t *)malloc(sizeof(uint64_t) * (nb + 1));
    g->Ep = (uint64_t *)calloc(g->k + 1, sizeof(uint64_t));
    g->npng = (uint64_t *)calloc(g->k + 1, sizeof(uint64_t));
    uint64_t b = 0;
    for (uint64_t e = 0; e < m; ++e) {
        if (e == 0 || g->pe[e].p != g->pe[e - 1].p || g->pe[e].q != g->pe[e - 1].q) {
            if (b) g->bin_e1[b - 1] = e;
            g->bin_p[b] = g->pe[e].p; g->bin_q[b] = g->pe[e].q; g->bin_e0[b] = e;
            ++b;
        }
        g->Ep[g->pe[e].p]++;
        if (e == 0 || g->pe[e].p != g->pe[e - 1].p || g->pe[e].q != g->pe[e - 1].q || g->pe[e].u != g->pe[e - 1].u)
            g->npng[g->pe[e].p]++;
    }
    if (b) g->bin_e1[b - 1] = m;
    /* row and column indices of the bins */
    for (uint64_t i = 0; i < nb; ++i) { g->row_bin0[g->bin_p[i] + 1]++; g->col_bin_cnt[g->bin_q[i] + 1]++; }
    for (uint32_t p = 0; p < g->k; ++p) { g->row_bin0[p + 1] += g->row_bin0[p]; g->col_bin_cnt[p + 1] += g->col_bin_cnt[p]; }
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * (g->k + 1));
    memcpy(fill, g->col_bin_cnt, sizeof(uint64_t) * (g->k + 1));
    for (uint64_t i = 0; i < nb; ++i) g->col_bins[fill[g->bin_q[i]]++] = i; /* ascending p within q */
    free(fill);
    return 0;
}

static void gpop_free(gpop_t *g) {
    free(g->pe); free(g->bin_p); free(g->bin_q); free(g->bin_e0); free(g->bin_e1);
    free(g->row_bin0); free(g->col_bin_cnt); free(g->col_bins); free(g->Ep); free(g->npng);
}

/* --- user functions (Sec. 4) for each application ------------------------ */

/* scatterFunc: the value an active vertex sends. */
static void uf_scatter(const gpop_t *g, const state_t *s, uint32_t v, double *fv, uint64_t *iv) {
    uint64_t deg = g->rp[v + 1] - g->rp[v];
    switch (g->algo) {
    case ALG_PAGERANK: case ALG_PPR: *fv = s->x[v] / (double)deg; break;   /* Alg. 6, Alg. 4 style */
    case ALG_BFS: *iv = v; break;                                          /* Alg. 5: node id */
    default: *iv = s->val[v]; break;                                       /* Alg. 7 distance, CC label */
    }
}

/* initFunc: update1 then cond1, applied to the vertices just scattered. */
static int uf_init(const gpop_t *g, state_t *s, uint32_t v) {
    switch (g->algo) {
    case ALG_PAGERANK: s->x[v] = 0.0; return 1;                  /* Alg. 6 */
    case ALG_PPR: s->x[v] = 0.0; return v == g->src;             /* seed stays active */
    default: return 0;                                           /* Alg. 5, Alg. 7, CC */
    }
}

/* gatherFunc with applyWeight folded in: returns 1 if v becomes active. */
static int uf_gather(const gpop_t *g, state_t *s, uint32_t v, double fv, uint64_t iv,
                     int32_t wt, uint32_t iter) {
    switch (g->algo) {
    case ALG_PAGERANK: case ALG_PPR: s->x[v] += fv; return 1;
    case ALG_BFS:
        if (s->level[v] == U32_INF) { s->level[v] = iter; s->val[v] = iv; return 1; }
        if (s->level[v] == iter && iv < s->val[v]) s->val[v] = iv;  /* min-ID reading */
        return 0;
    case ALG_SSSP: {
        uint64_t cand = iv + (uint64_t)wt;                       /* Alg. 7 applyWeight */
        if (cand < s->val[v]) { s->val[v] = cand; return 1; }
        return 0;
    }
    default:                                                     /* CC: keep the minimum label */
        if (iv < s->val[v]) { s->val[v] = iv; return 1; }
        return 0;
    }
}

/* filterFunc: update2 then cond2 on the preliminary frontier. */
static int uf_filter(const gpop_t *g, state_t *s, uint32_t v) {
    switch (g->algo) {
    case ALG_PAGERANK: s->x[v] = (1.0 - g->d) / g->n + g->d * s->x[v]; return 1;   /* Alg. 6 */
    case ALG_PPR: s->x[v] = (v == g->src ? 1.0 - g->d : 0.0) + g->d * s->x[v]; return s->x[v] > 0.0;
    default: return 1;
    }
}

/*
 * Runs the serial engine.  Outputs:
 *   x        (PageRank/PPR, n doubles) or
 *   val      (BFS parent / SSSP distance / CC label, n uint64; U64_INF = none),
 *   level    (BFS only, n uint32),
 *   trace_modes (optional, max_iters * k bytes: 0 none, 1 SC, 2 PC),
 *   trace_va / trace_ea (optional, max_iters entries: frontier size / active
 *            out-edges entering each iteration),
 *   trace_bytes (optional, max_iters doubles: Eq. (SC)/(PC) bytes of the
 *            chosen modes),
 *   iters_out, res_out.
 * damping: PageRank d, or for PPR the continuation probability 1 - alpha.
 */
int orc_gpop(uint32_t n, const uint64_t *rp, const uint32_t *col, const int32_t *w,
             uint32_t P, uint32_t algo, uint32_t src, double damping, uint32_t max_iters,
             double tol, uint32_t policy, uint32_t bw_num, uint32_t bw_den,
             double *x, uint64_t *val, uint32_t *level,
             uint8_t *trace_modes, uint64_t *trace_va, uint64_t *trace_ea, double *trace_bytes,
             uint32_t *iters_out, double *res_out) {
    gpop_t g;
    memset(&g, 0, sizeof g);
    if (n == 0 || P == 0 || (algo != ALG_PAGERANK && algo != ALG_CC && src >= n)) return -1;
    if (gpop_layout(&g, n, rp, col, w, P) != 0) return -1;
    g.algo = algo; g.src = src; g.d = damping;
    uint64_t m = rp[n];

    state_t s;
    memset(&s, 0, sizeof s);
    s.active = (uint8_t *)calloc(n, 1);
    s.next = (uint8_t *)calloc(n, 1);
    double *xold = NULL;
    if (algo == ALG_PAGERANK || algo == ALG_PPR) {
        s.x = x;
        xold = (double *)malloc(sizeof(double) * n);
    } else {
        s.val = val;
    }
    if (algo == ALG_BFS) s.level = level;

    /* program initialisation, as in the driver function of Alg. 4, per application */
    for (uint32_t v = 0; v < n; ++v) {
        switch (algo) {
        case ALG_PAGERANK: s.x[v] = 1.0 / n; s.active[v] = 1; break;
        case ALG_PPR: s.x[v] = (v == src); s.active[v] = (v == src); break;
        case ALG_BFS: s.val[v] = (v == src) ? v : U64_INF; s.level[v] = (v == src) ? 0 : U32_INF; s.active[v] = (v == src); break;
        case ALG_SSSP: s.val[v] = (v == src) ? 0 : U64_INF; s.active[v] = (v == src); break;
        default: s.val[v] = v; s.active[v] = 1; break;
        }
    }

    /* bins: per bin, a message array (PC: one slot per PNG source; SC: only active sources) */
    uint64_t nb = g.nbins;
    message *msgs = (message *)malloc(sizeof(message) * (m ? m : 1));
    uint64_t *bin_m0 = (uint64_t *)malloc(sizeof(uint64_t) * (nb + 1));
    uint64_t *bin_mn = (uint64_t *)calloc(nb + 1, sizeof(uint64_t));
    {   /* message capacity of a bin = its PNG sources (at most its edges) */
        uint64_t off = 0;
        for (uint64_t b = 0; b < nb; ++b) { bin_m0[b] = off; off += g.bin_e1[b] - g.bin_e0[b]; }
    }
    uint8_t *mode = (uint8_t *)calloc(g.k, 1);
    uint8_t *gflag = (uint8_t *)calloc(g.k, 1);
    uint64_t *Va = (uint64_t *)calloc(g.k, sizeof(uint64_t));
    uint64_t *Ea = (uint64_t *)calloc(g.k, sizeof(uint64_t));

    uint32_t iter = 0;
    double res = 0.0;
    for (;;) {
        /* frontier sizes per partition entering this iteration */
        uint64_t tot_v = 0, tot_e = 0;
        for (uint32_t p = 0; p < g.k; ++p) { Va[p] = 0; Ea[p] = 0; }
        for (uint32_t v = 0; v < n; ++v)
            if (s.active[v]) { Va[v / P]++; Ea[v / P] += rp[v + 1] - rp[v]; tot_v++; tot_e += rp[v + 1] - rp[v]; }
        if (tot_v == 0 || iter >= max_iters) break;
        if ((algo == ALG_PAGERANK || algo == ALG_PPR) && iter > 0 && res < tol) break;
        ++iter;

        /* ---- Scatter (Alg. 2; Alg. 3 for PC mode) ---- */
        double bytes = 0.0;
        for (uint32_t p = 0; p < g.k; ++p) {
            int md;
            if (Va[p] == 0 || g.Ep[p] == 0) md = 0;
            else if (policy == POL_FORCE_SC) md = 1;
            else if (policy == POL_FORCE_PC) md = 2;
            else md = orc_mode_decide(g.k, g.Ep[p], g.npng[p], Va[p], Ea[p], bw_num, bw_den);
            mode[p] = (uint8_t)md;
            bytes += orc_mode_bytes(md, g.k, g.Ep[p], g.npng[p], Va[p], Ea[p]);
            if (trace_modes) trace_modes[(uint64_t)(iter - 1) * g.k + p] = (uint8_t)md;
        }
        if (trace_va) trace_va[iter - 1] = tot_v;
        if (trace_ea) trace_ea[iter - 1] = tot_e;
        if (trace_bytes) trace_bytes[iter - 1] = bytes;

        if (xold) memcpy(xold, s.x, sizeof(double) * n);   /* x_t, for the L1 change */
        for (uint32_t p = 0; p < g.k; ++p) gflag[p] = 0;
        for (uint32_t p = 0; p < g.k; ++p) {
            if (mode[p] == 0) continue;
            for (uint64_t b = g.row_bin0[p]; b < g.row_bin0[p + 1]; ++b) {
                /* walk the bin's edges message by message (runs of equal source) */
                uint64_t cnt = 0;
                for (uint64_t e = g.bin_e0[b]; e < g.bin_e1[b];) {
                    uint32_t u = g.pe[e].u;
                    uint64_t e1 = e;
                    while (e1 < g.bin_e1[b] && g.pe[e1].u == u) ++e1;
                    if (mode[p] == 2 || s.active[u]) {
                        /* PC inserts every source of N_i^p(q) (Alg. 3); SC only active ones (Alg. 2) */
                        message *mm = &msgs[bin_m0[b] + cnt++];
                        mm->null_msg = !s.active[u];
                        mm->fval = 0.0; mm->ival = 0;
                        if (s.active[u]) uf_scatter(&g, &s, u, &mm->fval, &mm->ival);
                        mm->id_beg = e; mm->id_end = e1;
                    }
                    e = e1;
                }
                bin_mn[b] = cnt;
                if (cnt) gflag[g.bin_q[b]] = 1;
            }
        }
        /* reInit Frontier step of Alg. 2: initFunc on every active vertex of sPartList */
        for (uint32_t v = 0; v < n; ++v) s.next[v] = s.active[v] ? (uint8_t)uf_init(&g, &s, v) : 0;

        /* ---- Gather step of Alg. 2 ---- */
        for (uint32_t q = 0; q < g.k; ++q) {
            if (!gflag[q]) continue;
            for (uint64_t i = g.col_bin_cnt[q]; i < g.col_bin_cnt[q + 1]; ++i) {
                uint64_t b = g.col_bins[i];
                if (mode[g.bin_p[b]] == 0) continue;
                for (uint64_t j = 0; j < bin_mn[b]; ++j) {
                    const message *mm = &msgs[bin_m0[b] + j];
                    if (mm->null_msg) continue;            /* reading: NULL messages are ignored */
                    for (uint64_t e = mm->id_beg; e < mm->id_end; ++e) {
                        uint32_t v = g.pe[e].v;
                        if (uf_gather(&g, &s, v, mm->fval, mm->ival, g.pe[e].w, iter)) s.next[v] = 1;
                    }
                }
            }
        }
        /* ---- filter Frontier step of Alg. 2 ---- */
        for (uint32_t v = 0; v < n; ++v)
            if (s.next[v]) s.next[v] = (uint8_t)uf_filter(&g, &s, v);

        if (xold) {
            res = 0.0;
            for (uint32_t v = 0; v < n; ++v) res += fabs(s.x[v] - xold[v]);
        }
        uint8_t *tmp = s.active; s.active = s.next; s.next = tmp;
        if (res_out) *res_out = res;
    }
    if (iters_out) *iters_out = iter;
    free(msgs); free(bin_m0); free(bin_mn); free(mode); free(gflag); free(Va); free(Ea);
    free(s.active); free(s.next); free(xold);
    gpop_free(&g);
    return 0;
}
