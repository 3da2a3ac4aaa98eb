/*
 * ttc_oracle.c -- plain, slow CPU oracle for exact (d13, d12, d23)-temporal
 * triangle counts (Pashanasangi & Seshadhri, KDD'21).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes is the plain definition:
 *   - Sec. 3: a temporal graph is a list of directed edges (u, v, t); an edge
 *     is identified by its position idx in the input arrays.
 *   - Def. 1 (Sec. 1.1): three edges whose induced static graph is a triangle
 *     form a (d13, d12, d23)-temporal triangle when t1 < t2 < t3,
 *     t2 - t1 <= d12, t3 - t2 <= d23 and t3 - t1 <= d13.
 *   - Fig. 2: the eight triangle types T1..T8, read off the first edge
 *     e1 = a->b (its tail a is the figure's red vertex, its head b the green
 *     one, the third vertex c the blue one) and the pairs/directions of e2
 *     and e3.  Output slot k-1 holds the count of type T_k.
 *
 * Readings taken where the paper is silent:
 *   - Ties: the paper assumes unique timestamps (Sec. 3).  Edges are ordered
 *     by the key (t, idx); "t1 < t2 < t3" is read as key order and the three
 *     windows are applied to timestamp differences, inclusive.  The strict
 *     variant (the *_ex entry points with strict = 1) reads Def. 1's
 *     t1 < t2 < t3 literally instead: a triple whose edges share a timestamp
 *     is not counted.
 *   - Self-loops never lie on three distinct vertices; they are dropped.
 *   - Duplicate (u, v, t) edges are distinct edges, ordered by idx.
 *   - delta components are taken as given (no normalisation); each is >= 0.
 *   - Counts are exact: accumulated in 128 bits; a total that does not fit
 *     in 64 bits is reported as an overflow instead of wrapping.
 *
 * Two evaluators:
 *   O0 (ttc_oracle_bruteforce): every triple of edges, Def. 1 checked
 *      literally.  O(m^3); tiny graphs only.
 *   O1 (ttc_oracle_count): static triangles found by plain adjacency (vertex
 *      ids a < b < c, no degeneracy ordering, no orientation); for each
 *      triangle and each assignment of its three vertex pairs to the roles
 *      (first, second, third) the sum of Lemma 1 is evaluated directly:
 *      for each e1 on the first pair, each e2 on the second pair with
 *      key(e2) > key(e1) and t2 - t1 <= d12, the number of e3 on the third
 *      pair with key(e3) > key(e2) and t3 <= min(t2 + d23, t1 + d13),
 *      counted separately for each direction of the third pair.
 *   O1f (ttc_oracle_count_fwd, ttc_oracle_stats_fwd): the same per-triangle
 *      sums, with the static triangles found by the textbook "forward" rule
 *      instead of the plain one (every pair oriented from the endpoint of
 *      smaller (degree, id) to the larger; each triangle found once, at its
 *      first vertex, by merging two sorted out-lists).  On power-law graphs
 *      the plain rule visits about deg^2 vertex pairs at every hub, which
 *      takes hours at a million vertices; the forward rule visits the same
 *      triangles in O(m_s^1.5).  The tests check that both rules give the
 *      same triangles and counts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

enum { ORACLE_OK = 0, ORACLE_ERR_INVALID = -1, ORACLE_ERR_NOMEM = -3, ORACLE_ERR_OVERFLOW = -6 };

typedef struct {
    uint32_t u, v;   /* tail, head */
    int64_t t;
    uint64_t idx;    /* position in the input arrays */
} edge_t;

/* key(e) = (t(e), idx(e)); strict key order is the reading of t1 < t2 < t3 */
static int key_less(const edge_t *a, const edge_t *b) {
    return a->t < b->t || (a->t == b->t && a->idx < b->idx);
}

static int edge_on(const edge_t *e, uint32_t x, uint32_t y) {
    return (e->u == x && e->v == y) || (e->u == y && e->v == x);
}

/*
 * Fig. 2, read one picture at a time.  e1 = a->b; c is the third vertex.
 *   T1: e2 = c->b, e3 = a->c      T5: e2 = a->c, e3 = c->b
 *   T2: e2 = c->b, e3 = c->a      T6: e2 = c->a, e3 = c->b
 *   T3: e2 = b->c, e3 = a->c      T7: e2 = a->c, e3 = b->c
 *   T4: e2 = b->c, e3 = c->a      T8: e2 = c->a, e3 = b->c
 * Returns 0..7 for T1..T8.  The caller guarantees the three edges lie on the
 * three pairs of one triangle, one edge per pair.
 */
static int classify(const edge_t *e1, const edge_t *e2, const edge_t *e3) {
    const uint32_t a = e1->u, b = e1->v;
    const uint32_t c = (e2->u != a && e2->u != b) ? e2->u : e2->v;
    const int e2_cb = (e2->u == c && e2->v == b), e2_bc = (e2->u == b && e2->v == c);
    const int e2_ac = (e2->u == a && e2->v == c), e2_ca = (e2->u == c && e2->v == a);
    const int e3_ac = (e3->u == a && e3->v == c), e3_ca = (e3->u == c && e3->v == a);
    const int e3_cb = (e3->u == c && e3->v == b), e3_bc = (e3->u == b && e3->v == c);
    if (e2_cb && e3_ac) return 0;
    if (e2_cb && e3_ca) return 1;
    if (e2_bc && e3_ac) return 2;
    if (e2_bc && e3_ca) return 3;
    if (e2_ac && e3_cb) return 4;
    if (e2_ca && e3_cb) return 5;
    if (e2_ac && e3_bc) return 6;
    if (e2_ca && e3_bc) return 7;
    return -1; /* not reachable for a valid triangle */
}

/* Def. 1 windows on (key-sorted) e1, e2, e3, in 128-bit arithmetic. */
static int in_windows(const edge_t *e1, const edge_t *e2, const edge_t *e3,
                      int64_t d13, int64_t d12, int64_t d23) {
    return (i128)e2->t - e1->t <= d12 && (i128)e3->t - e2->t <= d23 && (i128)e3->t - e1->t <= d13;
}

static int64_t drop_self_loops(const uint32_t *src, const uint32_t *dst, const int64_t *t,
                               uint64_t m, edge_t *out) {
    int64_t k = 0;
    for (uint64_t i = 0; i < m; i++) {
        if (src[i] == dst[i]) continue;
        out[k].u = src[i]; out[k].v = dst[i]; out[k].t = t[i]; out[k].idx = i; k++;
    }
    return k;
}

static int check_deltas(const int64_t *deltas, uint32_t nd) {
    for (uint32_t q = 0; q < 3 * nd; q++) if (deltas[q] < 0) return 0;
    return 1;
}

static int finish(const u128 *acc, uint32_t nd, uint64_t *out) {
    int rc = ORACLE_OK;
    for (uint32_t q = 0; q < 8 * nd; q++) {
        if (acc[q] > (u128)UINT64_MAX) { rc = ORACLE_ERR_OVERFLOW; out[q] = UINT64_MAX; }
        else out[q] = (uint64_t)acc[q];
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* O0: brute force over all edge triples                                     */
/* ------------------------------------------------------------------------ */
int ttc_oracle_bruteforce_ex(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                             const int64_t *deltas, uint32_t nd, int strict, uint64_t *out);

int ttc_oracle_bruteforce(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                          const int64_t *deltas, uint32_t nd, uint64_t *out) {
    return ttc_oracle_bruteforce_ex(src, dst, t, m, deltas, nd, 0, out);
}

int ttc_oracle_bruteforce_ex(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                             const int64_t *deltas, uint32_t nd, int strict, uint64_t *out) {
    if ((m && (!src || !dst || !t)) || !out || (nd && !deltas) || !check_deltas(deltas, nd))
        return ORACLE_ERR_INVALID;
    edge_t *e = (edge_t *)malloc(sizeof(edge_t) * (m ? m : 1));
    u128 *acc = (u128 *)calloc(8 * (size_t)(nd ? nd : 1), sizeof(u128));
    if (!e || !acc) { free(e); free(acc); return ORACLE_ERR_NOMEM; }
    const int64_t k = drop_self_loops(src, dst, t, m, e);
    for (int64_t i = 0; i < k; i++)
        for (int64_t j = i + 1; j < k; j++)
            for (int64_t l = j + 1; l < k; l++) {
                const edge_t *x[3] = {&e[i], &e[j], &e[l]};
                /* sort the three edges by key */
                for (int p = 0; p < 2; p++)
                    for (int q = 0; q < 2 - p; q++)
                        if (key_less(x[q + 1], x[q])) { const edge_t *s = x[q]; x[q] = x[q + 1]; x[q + 1] = s; }
                /* induced static graph is a triangle: exactly three distinct
                   vertices and three distinct vertex pairs */
                const uint32_t vs[6] = {x[0]->u, x[0]->v, x[1]->u, x[1]->v, x[2]->u, x[2]->v};
                int distinct = 0;
                for (int p = 0; p < 6; p++) {
                    int seen = 0;
                    for (int q = 0; q < p; q++) seen |= (vs[q] == vs[p]);
                    distinct += !seen;
                }
                if (distinct != 3) continue;
                if (edge_on(x[1], x[0]->u, x[0]->v) || edge_on(x[2], x[0]->u, x[0]->v) ||
                    edge_on(x[2], x[1]->u, x[1]->v))
                    continue;
                const int ty = classify(x[0], x[1], x[2]);
                if (ty < 0) continue;
                if (strict && !(x[0]->t < x[1]->t && x[1]->t < x[2]->t)) continue;
                for (uint32_t q = 0; q < nd; q++)
                    if (in_windows(x[0], x[1], x[2], deltas[3 * q], deltas[3 * q + 1], deltas[3 * q + 2]))
                        acc[8 * q + ty] += 1;
            }
    const int rc = finish(acc, nd, out);
    free(e); free(acc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* O1: plain adjacency + Lemma 1 evaluated directly                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t lo, hi;     /* lo < hi by vertex id */
    uint64_t first, len; /* edges of this pair in `pe`, sorted by key */
} pair_t;

typedef struct {
    int64_t k;          /* edges after self-loop removal */
    edge_t *pe;         /* edges grouped by pair, key-sorted inside a pair */
    int64_t ms;         /* number of pairs (static edges) */
    pair_t *pairs;      /* sorted by (lo, hi) */
    uint32_t n;         /* max vertex id + 1 */
    uint64_t *adj_off;  /* n + 1 */
    uint32_t *adj_nbr;  /* 2 ms, sorted by neighbour id inside a vertex */
    int64_t *adj_pair;  /* pair index of each adjacency entry */
} graph_t;

static int cmp_pair_then_key(const void *pa, const void *pb) {
    const edge_t *a = (const edge_t *)pa, *b = (const edge_t *)pb;
    const uint32_t alo = a->u < a->v ? a->u : a->v, ahi = a->u < a->v ? a->v : a->u;
    const uint32_t blo = b->u < b->v ? b->u : b->v, bhi = b->u < b->v ? b->v : b->u;
    if (alo != blo) return alo < blo ? -1 : 1;
    if (ahi != bhi) return ahi < bhi ? -1 : 1;
    if (key_less(a, b)) return -1;
    if (key_less(b, a)) return 1;
    return 0;
}

typedef struct { uint32_t v, nbr; int64_t pair; } adj_entry;
static int cmp_adj(const void *pa, const void *pb) {
    const adj_entry *a = (const adj_entry *)pa, *b = (const adj_entry *)pb;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    if (a->nbr != b->nbr) return a->nbr < b->nbr ? -1 : 1;
    return 0;
}

static void graph_free(graph_t *g) {
    free(g->pe); free(g->pairs); free(g->adj_off); free(g->adj_nbr); free(g->adj_pair);
    memset(g, 0, sizeof(*g));
}

static int graph_build(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                       int want_adjacency, graph_t *g) {
    memset(g, 0, sizeof(*g));
    g->pe = (edge_t *)malloc(sizeof(edge_t) * (m ? m : 1));
    if (!g->pe) return ORACLE_ERR_NOMEM;
    g->k = drop_self_loops(src, dst, t, m, g->pe);
    qsort(g->pe, (size_t)g->k, sizeof(edge_t), cmp_pair_then_key);
    g->pairs = (pair_t *)malloc(sizeof(pair_t) * (g->k ? g->k : 1));
    if (!g->pairs) { graph_free(g); return ORACLE_ERR_NOMEM; }
    uint32_t maxid = 0;
    for (int64_t i = 0; i < g->k; i++) {
        const edge_t *e = &g->pe[i];
        const uint32_t lo = e->u < e->v ? e->u : e->v, hi = e->u < e->v ? e->v : e->u;
        if (e->v > maxid) maxid = e->v;
        if (e->u > maxid) maxid = e->u;
        if (g->ms == 0 || g->pairs[g->ms - 1].lo != lo || g->pairs[g->ms - 1].hi != hi) {
            g->pairs[g->ms].lo = lo; g->pairs[g->ms].hi = hi;
            g->pairs[g->ms].first = (uint64_t)i; g->pairs[g->ms].len = 0;
            g->ms++;
        }
        g->pairs[g->ms - 1].len++;
    }
    g->n = g->k ? maxid + 1 : 0;
    if (!want_adjacency) return ORACLE_OK;
    adj_entry *ae = (adj_entry *)malloc(sizeof(adj_entry) * (2 * g->ms + 1));
    g->adj_off = (uint64_t *)calloc((size_t)g->n + 1, sizeof(uint64_t));
    g->adj_nbr = (uint32_t *)malloc(sizeof(uint32_t) * (2 * g->ms + 1));
    g->adj_pair = (int64_t *)malloc(sizeof(int64_t) * (2 * g->ms + 1));
    if (!ae || !g->adj_off || !g->adj_nbr || !g->adj_pair) { free(ae); graph_free(g); return ORACLE_ERR_NOMEM; }
    for (int64_t p = 0; p < g->ms; p++) {
        ae[2 * p].v = g->pairs[p].lo; ae[2 * p].nbr = g->pairs[p].hi; ae[2 * p].pair = p;
        ae[2 * p + 1].v = g->pairs[p].hi; ae[2 * p + 1].nbr = g->pairs[p].lo; ae[2 * p + 1].pair = p;
    }
    qsort(ae, (size_t)(2 * g->ms), sizeof(adj_entry), cmp_adj);
    for (int64_t i = 0; i < 2 * g->ms; i++) {
        g->adj_off[ae[i].v + 1]++;
        g->adj_nbr[i] = ae[i].nbr; g->adj_pair[i] = ae[i].pair;
    }
    for (uint32_t v = 0; v < g->n; v++) g->adj_off[v + 1] += g->adj_off[v];
    free(ae);
    return ORACLE_OK;
}

/* index of the pair {x, y} in g->pairs, or -1 */
static int64_t find_pair(const graph_t *g, uint32_t x, uint32_t y) {
    const uint32_t lo = x < y ? x : y, hi = x < y ? y : x;
    int64_t l = 0, r = g->ms;
    while (l < r) {
        const int64_t mid = l + (r - l) / 2;
        const pair_t *p = &g->pairs[mid];
        if (p->lo < lo || (p->lo == lo && p->hi < hi)) l = mid + 1; else r = mid;
    }
    return (l < g->ms && g->pairs[l].lo == lo && g->pairs[l].hi == hi) ? l : -1;
}

/* one direction of one pair: edges with tail `tail`, key-sorted */
typedef struct { const edge_t **e; int64_t len; } sublist_t;

static int split_by_tail(const graph_t *g, int64_t p, uint32_t tail, const edge_t **buf, sublist_t *out) {
    int64_t k = 0;
    const pair_t *pp = &g->pairs[p];
    for (uint64_t i = 0; i < pp->len; i++) {
        const edge_t *e = &g->pe[pp->first + i];
        if (e->u == tail) buf[k++] = e;
    }
    out->e = buf; out->len = k;
    return 0;
}

/* number of edges of `s` with key strictly greater than key(x) -> first index */
static int64_t first_key_after(const sublist_t *s, const edge_t *x) {
    int64_t l = 0, r = s->len;
    while (l < r) { const int64_t mid = l + (r - l) / 2; if (key_less(x, s->e[mid])) r = mid; else l = mid + 1; }
    return l;
}
/* number of edges of `s` with t <= bound (s is key-sorted, so t-sorted) */
static int64_t count_t_le(const sublist_t *s, i128 bound) {
    int64_t l = 0, r = s->len;
    while (l < r) { const int64_t mid = l + (r - l) / 2; if ((i128)s->e[mid]->t <= bound) l = mid + 1; else r = mid; }
    return l;
}

/* first index of `s` after x: by key, or (strict) by time, t > t(x) */
static int64_t first_after(const sublist_t *s, const edge_t *x, int strict) {
    return strict ? count_t_le(s, (i128)x->t) : first_key_after(s, x);
}

/*
 * Lemma 1 for one static triangle with the role assignment (P1, P2, P3) and
 * every direction: sum over e1 in P1, e2 in P2 (key after e1, t2 - t1 <= d12)
 * of #{e3 in P3 (each direction separately): key(e3) > key(e2),
 * t3 <= min(t2 + d23, t1 + d13)}.  Each hit set is classified by Fig. 2.
 * strict: "after" is t2 > t1 and t3 > t2 instead of key order.
 */
static void lemma1_roles(const int64_t pr[3], const sublist_t sub[3][2],
                         const int64_t *deltas, uint32_t nd, int strict, u128 *acc) {
    int64_t maxd12 = 0;
    for (uint32_t q = 0; q < nd; q++) if (deltas[3 * q + 1] > maxd12) maxd12 = deltas[3 * q + 1];
    for (int d1 = 0; d1 < 2; d1++) {
        const sublist_t *S1 = &sub[pr[0]][d1];
        for (int d2 = 0; d2 < 2; d2++) {
            const sublist_t *S2 = &sub[pr[1]][d2];
            for (int d3 = 0; d3 < 2; d3++) {
                const sublist_t *S3 = &sub[pr[2]][d3];
                if (!S1->len || !S2->len || !S3->len) continue;
                for (int64_t i = 0; i < S1->len; i++) {
                    const edge_t *e1 = S1->e[i];
                    for (int64_t j = first_after(S2, e1, strict); j < S2->len; j++) {
                        const edge_t *e2 = S2->e[j];
                        const i128 gap12 = (i128)e2->t - e1->t;
                        if (gap12 > maxd12) break; /* later e2 are later still */
                        const int64_t lo3 = first_after(S3, e2, strict);
                        if (lo3 >= S3->len) continue;
                        const int ty = classify(e1, e2, S3->e[lo3]);
                        for (uint32_t q = 0; q < nd; q++) {
                            const int64_t d13 = deltas[3 * q], d12 = deltas[3 * q + 1], d23 = deltas[3 * q + 2];
                            if (gap12 > d12) continue;
                            i128 bound = (i128)e2->t + d23;
                            if ((i128)e1->t + d13 < bound) bound = (i128)e1->t + d13;
                            const int64_t hi3 = count_t_le(S3, bound);
                            if (hi3 > lo3) acc[8 * q + ty] += (u128)(hi3 - lo3);
                        }
                    }
                }
            }
        }
    }
}

/* all six role assignments of one static triangle {a, b, c} */
static int count_one_triangle(const graph_t *g, const int64_t p[3], const uint32_t lo_hi[3][2],
                              const int64_t *deltas, uint32_t nd, int strict, u128 *acc) {
    /* split each pair into its two directions */
    size_t tot = 0;
    for (int i = 0; i < 3; i++) tot += g->pairs[p[i]].len;
    const edge_t **buf = (const edge_t **)malloc(sizeof(edge_t *) * (tot + 1));
    if (!buf) return ORACLE_ERR_NOMEM;
    sublist_t sub[3][2];
    size_t off = 0;
    for (int i = 0; i < 3; i++) {
        for (int d = 0; d < 2; d++) {
            split_by_tail(g, p[i], lo_hi[i][d], buf + off, &sub[i][d]);
            off += (size_t)sub[i][d].len;
        }
    }
    static const int64_t roles[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int r = 0; r < 6; r++) lemma1_roles(roles[r], (const sublist_t(*)[2])sub, deltas, nd, strict, acc);
    free(buf);
    return ORACLE_OK;
}

static int threads_or_default(int threads) {
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/*
 * O1 restricted to the static triangles whose smallest vertex id a satisfies
 * a % nparts == part (a sampling aid for timing: the parts partition the
 * triangles, so their counts sum to the full count).
 */
static int count_part(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                      const int64_t *deltas, uint32_t nd, int threads, uint32_t part, uint32_t nparts, int strict,
                      uint64_t *out);

int ttc_oracle_count(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                     const int64_t *deltas, uint32_t nd, int threads, uint64_t *out) {
    return count_part(src, dst, t, m, deltas, nd, threads, 0, 1, 0, out);
}

int ttc_oracle_count_ex(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                        const int64_t *deltas, uint32_t nd, int threads, int strict, uint64_t *out) {
    return count_part(src, dst, t, m, deltas, nd, threads, 0, 1, strict, out);
}

int ttc_oracle_count_part(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                          const int64_t *deltas, uint32_t nd, int threads, uint32_t part, uint32_t nparts,
                          uint64_t *out) {
    return count_part(src, dst, t, m, deltas, nd, threads, part, nparts, 0, out);
}

static int count_part(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                      const int64_t *deltas, uint32_t nd, int threads, uint32_t part, uint32_t nparts, int strict,
                      uint64_t *out) {
    if (nparts == 0 || part >= nparts) return ORACLE_ERR_INVALID;
    if ((m && (!src || !dst || !t)) || !out || (nd && !deltas) || !check_deltas(deltas, nd))
        return ORACLE_ERR_INVALID;
    graph_t g;
    int rc = graph_build(src, dst, t, m, 1, &g);
    if (rc) return rc;
    const int nt = threads_or_default(threads);
    u128 *acc = (u128 *)calloc((size_t)nt * 8 * (nd ? nd : 1), sizeof(u128));
    if (!acc) { graph_free(&g); return ORACLE_ERR_NOMEM; }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
    for (int64_t a = part; a < (int64_t)g.n; a += nparts) {
#ifdef _OPENMP
        u128 *my = acc + (size_t)omp_get_thread_num() * 8 * nd;
#else
        u128 *my = acc;
#endif
        /* triangles a < b < c by vertex id, found by adjacency lookup */
        for (uint64_t i = g.adj_off[a]; i < g.adj_off[a + 1]; i++) {
            const uint32_t b = g.adj_nbr[i];
            if (b <= (uint32_t)a) continue;
            for (uint64_t j = i + 1; j < g.adj_off[a + 1]; j++) {
                const uint32_t c = g.adj_nbr[j];
                const int64_t pbc = find_pair(&g, b, c);
                if (pbc < 0) continue;
                const int64_t pp[3] = {g.adj_pair[i], g.adj_pair[j], pbc};
                const uint32_t lh[3][2] = {{(uint32_t)a, b}, {(uint32_t)a, c}, {b, c}};
                if (count_one_triangle(&g, pp, lh, deltas, nd, strict, my)) err = 1;
            }
        }
    }
    u128 *tot = acc;
    for (int th = 1; th < nt; th++)
        for (uint32_t q = 0; q < 8 * nd; q++) tot[q] += acc[(size_t)th * 8 * nd + q];
    rc = err ? ORACLE_ERR_NOMEM : finish(tot, nd, out);
    free(acc);
    graph_free(&g);
    return rc;
}

/*
 * Per-triangle counts for given vertex triples {x, y, z} (any order).  A
 * triple that is not a static triangle yields zeros.  out is [k][nd][8].
 */
int ttc_oracle_count_triangles(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                               const uint32_t *tri, uint64_t k, const int64_t *deltas, uint32_t nd,
                               int threads, uint64_t *out) {
    if ((m && (!src || !dst || !t)) || (k && (!tri || !out)) || (nd && !deltas) || !check_deltas(deltas, nd))
        return ORACLE_ERR_INVALID;
    graph_t g;
    int rc = graph_build(src, dst, t, m, 0, &g);
    if (rc) return rc;
    int err = 0, ovf = 0;
    const int nt = threads_or_default(threads);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t i = 0; i < (int64_t)k; i++) {
        u128 acc[8 * 64];
        u128 *a = nd <= 64 ? acc : (u128 *)calloc(8 * (size_t)nd, sizeof(u128));
        if (!a) { err = 1; continue; }
        memset(a, 0, sizeof(u128) * 8 * nd);
        uint32_t x = tri[3 * i], y = tri[3 * i + 1], z = tri[3 * i + 2];
        /* sort the ids so the pairs are named as in O1 */
        if (x > y) { uint32_t s = x; x = y; y = s; }
        if (y > z) { uint32_t s = y; y = z; z = s; }
        if (x > y) { uint32_t s = x; x = y; y = s; }
        const int64_t pp[3] = {find_pair(&g, x, y), find_pair(&g, x, z), find_pair(&g, y, z)};
        if (x != y && y != z && pp[0] >= 0 && pp[1] >= 0 && pp[2] >= 0) {
            const uint32_t lh[3][2] = {{x, y}, {x, z}, {y, z}};
            if (count_one_triangle(&g, pp, lh, deltas, nd, 0, a)) err = 1;
        }
        for (uint32_t q = 0; q < 8 * nd; q++) {
            if (a[q] > (u128)UINT64_MAX) { ovf = 1; out[8 * nd * i + q] = UINT64_MAX; }
            else out[8 * nd * i + q] = (uint64_t)a[q];
        }
        if (a != acc) free(a);
    }
    graph_free(&g);
    return err ? ORACLE_ERR_NOMEM : ovf ? ORACLE_ERR_OVERFLOW : ORACLE_OK;
}

/*
 * The forward rule.  Pairs are oriented from the endpoint that comes first in
 * (degree, id) order; out(v) keeps v's adjacency order (by neighbour id).  A
 * triangle whose vertices come in the order a, b, c is visited once: at a,
 * for the out-neighbour b, as the common element c of out(a) and out(b).
 * The visitor gets the vertex ids sorted (x < y < z) and the pair indices
 * of {x, y}, {x, z}, {y, z}.
 */
typedef struct {
    uint64_t *off;   /* n + 1 */
    uint32_t *nbr;   /* out-neighbours, by id */
    int64_t *pair;   /* pair index of each out-entry */
} fwd_adj_t;

static void fwd_free(fwd_adj_t *f) {
    free(f->off); free(f->nbr); free(f->pair);
    memset(f, 0, sizeof(*f));
}

static int fwd_first(const graph_t *g, uint32_t v, uint32_t w) {
    const uint64_t dv = g->adj_off[v + 1] - g->adj_off[v], dw = g->adj_off[w + 1] - g->adj_off[w];
    return dv < dw || (dv == dw && v < w);
}

static int fwd_build(const graph_t *g, fwd_adj_t *f) {
    memset(f, 0, sizeof(*f));
    f->off = (uint64_t *)calloc((size_t)g->n + 1, sizeof(uint64_t));
    f->nbr = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)g->ms + 1));
    f->pair = (int64_t *)malloc(sizeof(int64_t) * ((size_t)g->ms + 1));
    if (!f->off || !f->nbr || !f->pair) { fwd_free(f); return ORACLE_ERR_NOMEM; }
    uint64_t k = 0;
    for (uint32_t v = 0; v < g->n; v++) {
        f->off[v] = k;
        for (uint64_t i = g->adj_off[v]; i < g->adj_off[v + 1]; i++) {
            if (!fwd_first(g, v, g->adj_nbr[i])) continue;
            f->nbr[k] = g->adj_nbr[i];
            f->pair[k] = g->adj_pair[i];
            k++;
        }
    }
    f->off[g->n] = k;
    return ORACLE_OK;
}

typedef void (*tri_visit_t)(const graph_t *g, const uint32_t xyz[3], const int64_t p[3], void *ctx, int thread);

static void fwd_enumerate(const graph_t *g, const fwd_adj_t *f, int nt, tri_visit_t visit, void *ctx) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t a = 0; a < (int64_t)g->n; a++) {
#ifdef _OPENMP
        const int th = omp_get_thread_num();
#else
        const int th = 0;
#endif
        for (uint64_t i = f->off[a]; i < f->off[a + 1]; i++) {
            const uint32_t b = f->nbr[i];
            uint64_t p = f->off[a], q = f->off[b];
            while (p < f->off[a + 1] && q < f->off[b + 1]) {
                if (f->nbr[p] < f->nbr[q]) { p++; continue; }
                if (f->nbr[p] > f->nbr[q]) { q++; continue; }
                /* c = f->nbr[p]: pairs {a, b} = f->pair[i], {a, c} = f->pair[p], {b, c} = f->pair[q] */
                const uint32_t v[3] = {(uint32_t)a, b, f->nbr[p]};
                const int64_t pv[3] = {f->pair[i], f->pair[p], f->pair[q]};  /* {v0,v1}, {v0,v2}, {v1,v2} */
                /* sort the ids; the pair of two ids is the one not naming the third */
                int o[3] = {0, 1, 2};
                if (v[o[0]] > v[o[1]]) { int x = o[0]; o[0] = o[1]; o[1] = x; }
                if (v[o[1]] > v[o[2]]) { int x = o[1]; o[1] = o[2]; o[2] = x; }
                if (v[o[0]] > v[o[1]]) { int x = o[0]; o[0] = o[1]; o[1] = x; }
                /* pair index of {v_i, v_j}: vertex k = 3 - i - j is the one left out */
                static const int pair_without[3] = {2, 1, 0};
                const uint32_t xyz[3] = {v[o[0]], v[o[1]], v[o[2]]};
                const int64_t pp[3] = {pv[pair_without[o[2]]], pv[pair_without[o[1]]], pv[pair_without[o[0]]]};
                visit(g, xyz, pp, ctx, th);
                p++;
                q++;
            }
        }
    }
}

typedef struct {
    const int64_t *deltas;
    uint32_t nd;
    int strict;
    u128 *acc;   /* per thread: 8 * nd */
    int err;
} fwd_count_ctx;

static void fwd_count_visit(const graph_t *g, const uint32_t xyz[3], const int64_t p[3], void *vctx, int th) {
    fwd_count_ctx *c = (fwd_count_ctx *)vctx;
    const uint32_t lh[3][2] = {{xyz[0], xyz[1]}, {xyz[0], xyz[2]}, {xyz[1], xyz[2]}};
    if (count_one_triangle(g, p, lh, c->deltas, c->nd, c->strict, c->acc + (size_t)th * 8 * c->nd)) c->err = 1;
}

/* O1 with the forward rule: the same result as ttc_oracle_count_ex. */
int ttc_oracle_count_fwd(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                         const int64_t *deltas, uint32_t nd, int threads, int strict, uint64_t *out) {
    if ((m && (!src || !dst || !t)) || !out || (nd && !deltas) || !check_deltas(deltas, nd))
        return ORACLE_ERR_INVALID;
    graph_t g;
    int rc = graph_build(src, dst, t, m, 1, &g);
    if (rc) return rc;
    fwd_adj_t f;
    rc = fwd_build(&g, &f);
    if (rc) { graph_free(&g); return rc; }
    const int nt = threads_or_default(threads);
    fwd_count_ctx c = {deltas, nd, strict, (u128 *)calloc((size_t)nt * 8 * (nd ? nd : 1), sizeof(u128)), 0};
    if (!c.acc) { fwd_free(&f); graph_free(&g); return ORACLE_ERR_NOMEM; }
    fwd_enumerate(&g, &f, nt, fwd_count_visit, &c);
    for (int th = 1; th < nt; th++)
        for (uint32_t q = 0; q < 8 * nd; q++) c.acc[q] += c.acc[(size_t)th * 8 * nd + q];
    rc = c.err ? ORACLE_ERR_NOMEM : finish(c.acc, nd, out);
    free(c.acc);
    fwd_free(&f);
    graph_free(&g);
    return rc;
}

typedef struct {
    uint64_t *tau, *work;  /* per thread */
    u128 *prod;
} fwd_stats_ctx;

static void fwd_stats_visit(const graph_t *g, const uint32_t xyz[3], const int64_t p[3], void *vctx, int th) {
    (void)xyz;
    fwd_stats_ctx *c = (fwd_stats_ctx *)vctx;
    const uint64_t s1 = g->pairs[p[0]].len, s2 = g->pairs[p[1]].len, s3 = g->pairs[p[2]].len;
    c->tau[th]++;
    c->work[th] += 8 * (s1 + s2 + s3) + 12;
    c->prod[th] += (u128)s1 * s2 * s3;
}

/*
 * Static statistics (Sec. 3, Table 2 columns): n, m (self-loops dropped),
 * m_s, tau (static triangles), sigma_max (largest undirected multiplicity),
 * and two sums over static triangles {a, b, c} with undirected
 * multiplicities s_ab, s_ac, s_bc:
 *   work_bytes = sum of 8 (s_ab + s_ac + s_bc) + 12
 *   prod       = sum of s_ab s_ac s_bc  (the total count when every window
 *                is unbounded; returned as two 64-bit halves)
 * stats = {n, m, m_s, tau, sigma_max, work_bytes, prod_lo, prod_hi}.
 */
int ttc_oracle_stats(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                     int threads, uint64_t *stats) {
    if ((m && (!src || !dst || !t)) || !stats) return ORACLE_ERR_INVALID;
    graph_t g;
    int rc = graph_build(src, dst, t, m, 1, &g);
    if (rc) return rc;
    const int nt = threads_or_default(threads);
    uint64_t tau = 0, work = 0, smax = 0;
    u128 prod = 0;
    for (int64_t p = 0; p < g.ms; p++) if (g.pairs[p].len > smax) smax = g.pairs[p].len;
#pragma omp parallel num_threads(nt)
    {
        uint64_t my_tau = 0, my_work = 0;
        u128 my_prod = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t a = 0; a < (int64_t)g.n; a++) {
            for (uint64_t i = g.adj_off[a]; i < g.adj_off[a + 1]; i++) {
                const uint32_t b = g.adj_nbr[i];
                if (b <= (uint32_t)a) continue;
                for (uint64_t j = i + 1; j < g.adj_off[a + 1]; j++) {
                    const int64_t pbc = find_pair(&g, b, g.adj_nbr[j]);
                    if (pbc < 0) continue;
                    const uint64_t s1 = g.pairs[g.adj_pair[i]].len, s2 = g.pairs[g.adj_pair[j]].len,
                                   s3 = g.pairs[pbc].len;
                    my_tau++;
                    my_work += 8 * (s1 + s2 + s3) + 12;
                    my_prod += (u128)s1 * s2 * s3;
                }
            }
        }
#pragma omp critical
        { tau += my_tau; work += my_work; prod += my_prod; }
    }
    stats[0] = g.n; stats[1] = (uint64_t)g.k; stats[2] = (uint64_t)g.ms; stats[3] = tau;
    stats[4] = smax; stats[5] = work; stats[6] = (uint64_t)prod; stats[7] = (uint64_t)(prod >> 64);
    graph_free(&g);
    return ORACLE_OK;
}

/* ttc_oracle_stats with the forward rule: the same statistics. */
int ttc_oracle_stats_fwd(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                         int threads, uint64_t *stats) {
    if ((m && (!src || !dst || !t)) || !stats) return ORACLE_ERR_INVALID;
    graph_t g;
    int rc = graph_build(src, dst, t, m, 1, &g);
    if (rc) return rc;
    fwd_adj_t f;
    rc = fwd_build(&g, &f);
    if (rc) { graph_free(&g); return rc; }
    const int nt = threads_or_default(threads);
    fwd_stats_ctx c = {(uint64_t *)calloc((size_t)nt, 8), (uint64_t *)calloc((size_t)nt, 8),
                       (u128 *)calloc((size_t)nt, sizeof(u128))};
    if (!c.tau || !c.work || !c.prod) {
        free(c.tau); free(c.work); free(c.prod); fwd_free(&f); graph_free(&g);
        return ORACLE_ERR_NOMEM;
    }
    fwd_enumerate(&g, &f, nt, fwd_stats_visit, &c);
    uint64_t tau = 0, work = 0, smax = 0;
    u128 prod = 0;
    for (int th = 0; th < nt; th++) { tau += c.tau[th]; work += c.work[th]; prod += c.prod[th]; }
    for (int64_t p = 0; p < g.ms; p++) if (g.pairs[p].len > smax) smax = g.pairs[p].len;
    stats[0] = g.n; stats[1] = (uint64_t)g.k; stats[2] = (uint64_t)g.ms; stats[3] = tau;
    stats[4] = smax; stats[5] = work; stats[6] = (uint64_t)prod; stats[7] = (uint64_t)(prod >> 64);
    free(c.tau); free(c.work); free(c.prod);
    fwd_free(&f);
    graph_free(&g);
    return ORACLE_OK;
}
