/*
 * ffg_oracle.c -- plain, slow, single-threaded CPU oracle of the fitness flow
 * graph metric.  TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU
 * baseline).  Compile with -ffp-contract=off so every FP64 expression rounds
 * exactly as written.
 *
 * Parity status per function (what pins each one is in tests/):
 *   or_raw_count       pinned: the paper's space sizes equal the product of
 *                      its list lengths (Sec. V table vs appendix table).
 *   or_valid_mask      pinned: brute force over itertools.product.
 *   or_build           pinned: brute-force all-pairs Hamming-distance-1 scan,
 *                      the adjacent-value worked example of Sec. III-B,
 *                      degree identities, networkx-free brute checks.
 *   or_pagerank_power  pinned: dense linear solve of the Google system,
 *                      chain / star / tournament closed forms, contraction
 *                      bound against or_pagerank_exact.
 *   or_pagerank_exact  pinned: the same dense solve and closed forms.
 *   or_dag_values      pinned: dense solve of (I - d A) y = 1, chain and star
 *                      closed forms, and y / sum y = or_pagerank_exact.
 *   or_absorption      pinned: dense solve of (I - A) a = 1/n, chain and star
 *                      closed forms, the mass of the sinks sums to 1.
 *   or_walks           pinned: the SplitMix64 reference outputs, a chain (every
 *                      walk ends at its end), arrival frequencies within
 *                      binomial bounds of or_absorption.
 *   or_centrality      pinned: hand examples, monotonicity, limits.
 *   or_minima_fraction pinned: a hand example, the global minimum gives 1,
 *                      every fraction lies in (0, 1].
 */
#include "ffg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* search space (Sec. III-B): X = S_1 x ... x S_n, raw index row-major       */
/* ------------------------------------------------------------------------ */

int or_raw_count(const or_space *s, int64_t *n_raw)
{
    if (!s || s->n_params < 1 || s->n_params > 16 || !s->radix || !s->values) return OR_BAD_ARG;
    int64_t r = 1;
    for (int i = 0; i < s->n_params; ++i) {
        if (s->radix[i] < 1) return OR_BAD_ARG;
        if (r > ((int64_t)1 << 62) / s->radix[i]) return OR_OVERFLOW;
        r *= s->radix[i];
    }
    *n_raw = r;
    return OR_OK;
}

/* digits of raw point r: the last parameter varies fastest */
static void decode(const or_space *s, int64_t r, int32_t *digit)
{
    for (int i = s->n_params - 1; i >= 0; --i) {
        digit[i] = (int32_t)(r % s->radix[i]);
        r /= s->radix[i];
    }
}

static int64_t encode(const or_space *s, const int32_t *digit)
{
    int64_t r = 0;
    for (int i = 0; i < s->n_params; ++i) r = r * s->radix[i] + digit[i];
    return r;
}

static int64_t value_of(const or_space *s, int param, int32_t digit)
{
    int64_t off = 0;
    for (int i = 0; i < param; ++i) off += s->radix[i];
    return s->values[off + digit];
}

/* product of the values of the listed parameters; 0 on success */
static int product(const or_space *s, const int32_t *digit, const int32_t *idx, int n,
                   int64_t *out)
{
    int64_t p = 1;
    for (int k = 0; k < n; ++k) {
        int64_t v = value_of(s, idx[k], digit[idx[k]]);
        if (__builtin_mul_overflow(p, v, &p)) return OR_OVERFLOW;
    }
    *out = p;
    return OR_OK;
}

/* 1 if the configuration satisfies every clause, 0 if not, <0 on error.
 * Every clause is evaluated (no early exit), so a product that does not fit
 * int64 is reported for any space in which it can occur. */
static int satisfies(const or_space *s, const int32_t *digit)
{
    int all = 1;
    for (int c = 0; c < s->n_clauses; ++c) {
        const or_clause *cl = &s->clauses[c];
        int64_t pa, pb;
        if (product(s, digit, cl->a, cl->n_a, &pa) || product(s, digit, cl->b, cl->n_b, &pb))
            return -OR_OVERFLOW;
        int ok;
        switch (cl->kind) {
        case OR_PROD_LE: ok = pa <= cl->bound; break;
        case OR_PROD_GE: ok = pa >= cl->bound; break;
        case OR_DIVIDES: ok = (pb != 0) && (pa % pb == 0); break;
        case OR_PROD_LE_PROD: ok = pa <= pb; break;
        default: return -OR_BAD_ARG;
        }
        all = all && ok;
    }
    return all;
}

static int check_clauses(const or_space *s)
{
    if (s->n_clauses < 0 || (s->n_clauses > 0 && !s->clauses)) return OR_BAD_ARG;
    for (int c = 0; c < s->n_clauses; ++c) {
        const or_clause *cl = &s->clauses[c];
        if (cl->n_a < 0 || cl->n_a > 16 || cl->n_b < 0 || cl->n_b > 16) return OR_BAD_ARG;
        for (int k = 0; k < cl->n_a; ++k)
            if (cl->a[k] < 0 || cl->a[k] >= s->n_params) return OR_BAD_ARG;
        for (int k = 0; k < cl->n_b; ++k)
            if (cl->b[k] < 0 || cl->b[k] >= s->n_params) return OR_BAD_ARG;
    }
    return OR_OK;
}

int or_valid_mask(const or_space *s, uint8_t *valid)
{
    int64_t R;
    int st = or_raw_count(s, &R);
    if (st) return st;
    if ((st = check_clauses(s))) return st;
    int32_t digit[16];
    for (int64_t r = 0; r < R; ++r) {
        decode(s, r, digit);
        int ok = satisfies(s, digit);
        if (ok < 0) return -ok;
        valid[r] = (uint8_t)ok;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* fitness flow graph (Sec. VII-B)                                           */
/* ------------------------------------------------------------------------ */

/* the neighbour set N(x) of Sec. III-B: every point that differs from x in
 * exactly one parameter (Hamming), or in one parameter whose new value is
 * next to the old one in that parameter's list (adjacent).  Only valid
 * configurations are points of the space.  Writes node ids, returns count. */
static int neighbours(const or_space *s, const int64_t *node_of_raw, int nbh,
                      const int32_t *digit, int32_t *out)
{
    int32_t y[16];
    int cnt = 0;
    for (int i = 0; i < s->n_params; ++i) {
        for (int j = 0; j < s->radix[i]; ++j) {
            if (j == digit[i]) continue;
            if (nbh == OR_ADJACENT && j != digit[i] - 1 && j != digit[i] + 1) continue;
            memcpy(y, digit, sizeof(int32_t) * (size_t)s->n_params);
            y[i] = j;
            int64_t node = node_of_raw[encode(s, y)];
            if (node >= 0) out[cnt++] = (int32_t)node;
        }
    }
    return cnt;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void or_graph_free(or_graph *g)
{
    if (!g) return;
    free(g->node_raw); free(g->out_ptr); free(g->out_idx); free(g->in_ptr); free(g->in_idx);
    free(g->outdeg); free(g->is_min); free(g->failed); free(g->node_fit);
    memset(g, 0, sizeof(*g));
}

int or_build(const or_space *s, const double *fitness_raw, int nbh, double fail_thr, or_graph *g)
{
    memset(g, 0, sizeof(*g));
    if (nbh != OR_HAMMING && nbh != OR_ADJACENT) return OR_BAD_ARG;
    int64_t R;
    int st = or_raw_count(s, &R);
    if (st) return st;
    uint8_t *valid = (uint8_t *)malloc((size_t)R);
    int64_t *node_of_raw = (int64_t *)malloc(sizeof(int64_t) * (size_t)R);
    if (!valid || !node_of_raw) { free(valid); free(node_of_raw); return OR_NO_MEMORY; }
    if ((st = or_valid_mask(s, valid))) { free(valid); free(node_of_raw); return st; }

    /* node id = rank of the raw index among valid configurations */
    int64_t N = 0;
    for (int64_t r = 0; r < R; ++r) node_of_raw[r] = valid[r] ? N++ : -1;
    free(valid);
    g->n_raw = R;
    g->n_nodes = N;
    if (N >= ((int64_t)1 << 31)) { free(node_of_raw); return OR_OVERFLOW; }

    g->node_raw = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    g->out_ptr = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    g->in_ptr = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    g->outdeg = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t));
    g->is_min = (uint8_t *)calloc((size_t)N + 1, 1);
    g->failed = (uint8_t *)calloc((size_t)N + 1, 1);
    g->node_fit = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *key = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    int64_t max_cand = 0;
    for (int i = 0; i < s->n_params; ++i) max_cand += s->radix[i];
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(max_cand + 1));
    if (!g->node_raw || !g->out_ptr || !g->in_ptr || !g->outdeg || !g->is_min || !g->failed ||
        !g->node_fit || !key || !nb) {
        free(node_of_raw); free(key); free(nb); or_graph_free(g); return OR_NO_MEMORY;
    }

    /* failed configurations (Sec. V): fitness not below the failure
     * threshold, NaN included; they compare as +infinity */
    for (int64_t r = 0, v = 0; r < R; ++r) {
        if (node_of_raw[r] < 0) continue;
        double f = fitness_raw[r];
        g->node_raw[v] = r;
        g->node_fit[v] = f;
        g->failed[v] = !(f < fail_thr);
        key[v] = g->failed[v] ? INFINITY : f;
        ++v;
    }

    /* pass 1: out-degrees.  Edge u -> v iff v in N(u) and key(v) < key(u). */
    int32_t digit[16];
    for (int64_t u = 0; u < N; ++u) {
        decode(s, g->node_raw[u], digit);
        int c = neighbours(s, node_of_raw, nbh, digit, nb);
        int32_t d = 0;
        for (int k = 0; k < c; ++k) d += key[nb[k]] < key[u];
        g->outdeg[u] = d;
        g->out_ptr[u + 1] = g->out_ptr[u] + d;
    }
    int64_t E = g->out_ptr[N];
    g->n_edges = E;
    g->out_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E + 1));
    g->in_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (!g->out_idx || !g->in_idx || !fill) {
        free(node_of_raw); free(key); free(nb); free(fill); or_graph_free(g); return OR_NO_MEMORY;
    }

    /* pass 2: out lists, each sorted ascending by node id */
    for (int64_t u = 0; u < N; ++u) {
        decode(s, g->node_raw[u], digit);
        int c = neighbours(s, node_of_raw, nbh, digit, nb);
        qsort(nb, (size_t)c, sizeof(int32_t), cmp_i32);
        int64_t o = g->out_ptr[u];
        for (int k = 0; k < c; ++k)
            if (key[nb[k]] < key[u]) g->out_idx[o++] = nb[k];
    }

    /* in lists: the transpose, filled by ascending source id */
    for (int64_t e = 0; e < E; ++e) g->in_ptr[g->out_idx[e] + 1] += 1;
    for (int64_t v = 0; v < N; ++v) g->in_ptr[v + 1] += g->in_ptr[v];
    for (int64_t v = 0; v < N; ++v) fill[v] = g->in_ptr[v];
    for (int64_t u = 0; u < N; ++u)
        for (int64_t e = g->out_ptr[u]; e < g->out_ptr[u + 1]; ++e)
            g->in_idx[fill[g->out_idx[e]]++] = (int32_t)u;

    /* local minima (Sec. III-B): no neighbour with better fitness; failed
     * points are not minima.  f_opt = best non-failed fitness. */
    g->f_opt = INFINITY;
    for (int64_t v = 0; v < N; ++v) {
        g->is_min[v] = !g->failed[v] && g->outdeg[v] == 0;
        if (!g->failed[v] && g->node_fit[v] < g->f_opt) g->f_opt = g->node_fit[v];
    }
    free(fill); free(node_of_raw); free(key); free(nb);
    return N > 0 ? OR_OK : OR_EMPTY;
}

/* ------------------------------------------------------------------------ */
/* PageRank (Sec. VII-B): column-stochastic A[v,u] = 1/outdeg(u) for u->v,   */
/* damping alpha, uniform teleport, dangling mass spread uniformly          */
/* ------------------------------------------------------------------------ */

int or_pagerank_power(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                      const int32_t *outdeg, double alpha, double tol, int32_t max_iter,
                      double *x, int32_t *iters, double *residual)
{
    if (n <= 0 || !(alpha > 0.0 && alpha < 1.0) || max_iter < 1) return OR_BAD_ARG;
    double *xn = (double *)malloc(sizeof(double) * (size_t)n);
    if (!xn) return OR_NO_MEMORY;
    for (int64_t v = 0; v < n; ++v) x[v] = 1.0 / (double)n;
    int32_t k = 0;
    double res = INFINITY;
    while (k < max_iter) {
        double D = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (outdeg[u] == 0) D += x[u];
        double c = (alpha * D + 1.0 - alpha) / (double)n;
        for (int64_t v = 0; v < n; ++v) {
            double s = 0.0;
            for (int64_t e = in_ptr[v]; e < in_ptr[v + 1]; ++e)
                s += x[in_idx[e]] / (double)outdeg[in_idx[e]];
            xn[v] = alpha * s + c;
        }
        res = 0.0;
        for (int64_t v = 0; v < n; ++v) res += fabs(xn[v] - x[v]);
        memcpy(x, xn, sizeof(double) * (size_t)n);
        ++k;
        if (res < tol) break;
    }
    free(xn);
    *iters = k;
    *residual = res;
    return res < tol ? OR_OK : OR_NOT_CONVERGED;
}

typedef struct { double key; int64_t id; } keyed;

static int cmp_desc(const void *a, const void *b)
{
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key > y->key) return -1;
    if (x->key < y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* Neumaier's compensated sum (Neumaier 1974) */
static double neumaier_add(double sum, double v, double *comp)
{
    double t = sum + v;
    if (fabs(sum) >= fabs(v)) *comp += (sum - t) + v;
    else *comp += (v - t) + sum;
    return t;
}

/* With uniform teleport and uniform dangling redistribution the PageRank
 * vector satisfies (I - alpha P) x = c 1 for a scalar c, so x is y / sum(y)
 * with y = 1 + alpha P y.  Every FFG edge goes from higher to strictly lower
 * fitness, so the graph is acyclic and y is solved exactly by visiting nodes
 * in descending fitness (failed = +inf first). */
int or_pagerank_exact(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                      const int32_t *outdeg, const uint8_t *failed, const double *node_fit,
                      double alpha, double *x)
{
    if (n <= 0 || !(alpha >= 0.0 && alpha < 1.0)) return OR_BAD_ARG;
    keyed *order = (keyed *)malloc(sizeof(keyed) * (size_t)n);
    if (!order) return OR_NO_MEMORY;
    for (int64_t v = 0; v < n; ++v) {
        order[v].key = failed[v] ? INFINITY : node_fit[v];
        order[v].id = v;
    }
    qsort(order, (size_t)n, sizeof(keyed), cmp_desc);
    for (int64_t k = 0; k < n; ++k) {
        int64_t v = order[k].id;
        double s = 0.0;
        for (int64_t e = in_ptr[v]; e < in_ptr[v + 1]; ++e)
            s += x[in_idx[e]] / (double)outdeg[in_idx[e]];
        x[v] = 1.0 + alpha * s;
    }
    free(order);
    double sum = 0.0, comp = 0.0;
    for (int64_t v = 0; v < n; ++v) sum = neumaier_add(sum, x[v], &comp);
    sum += comp;
    for (int64_t v = 0; v < n; ++v) x[v] = x[v] / sum;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* the same recurrence, unnormalised and for any damping in [0, 1]:          */
/* y[v] = 1 + d * sum_{u -> v} y[u] / outdeg[u], nodes in descending key      */
/* (every edge runs to a strictly smaller key, so that order is topological) */
/* ------------------------------------------------------------------------ */

int or_dag_values(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                  const int32_t *outdeg, const uint8_t *failed, const double *node_fit,
                  double d, double *y)
{
    if (n <= 0 || !(d >= 0.0 && d <= 1.0)) return OR_BAD_ARG;
    keyed *order = (keyed *)malloc(sizeof(keyed) * (size_t)n);
    if (!order) return OR_NO_MEMORY;
    for (int64_t v = 0; v < n; ++v) {
        order[v].key = failed[v] ? INFINITY : node_fit[v];
        order[v].id = v;
    }
    qsort(order, (size_t)n, sizeof(keyed), cmp_desc);
    for (int64_t k = 0; k < n; ++k) {
        int64_t v = order[k].id;
        double s = 0.0;
        for (int64_t e = in_ptr[v]; e < in_ptr[v + 1]; ++e)
            s += y[in_idx[e]] / (double)outdeg[in_idx[e]];
        y[v] = 1.0 + d * s;
    }
    free(order);
    return OR_OK;
}

/* A walk starts at a uniformly random node and moves to a uniformly random   */
/* strictly better neighbour (an out-edge) until it reaches a node without    */
/* one.  a[v] = probability that it passes v; at a node without out-edges     */
/* the probability that it ends there (Sec. VII-B: the chance of arriving in  */
/* a minimum).  a = y / n for d = 1.                                          */
int or_absorption(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                  const int32_t *outdeg, const uint8_t *failed, const double *node_fit,
                  double *a)
{
    int st = or_dag_values(n, in_ptr, in_idx, outdeg, failed, node_fit, 1.0, a);
    if (st) return st;
    for (int64_t v = 0; v < n; ++v) a[v] = a[v] / (double)n;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* simulated improving walks (Sec. VII-B: a random walk on the FFG mimics a  */
/* randomised first-improvement local search)                                */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): output for state x, the
 * state having been advanced by the golden gamma first. */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

/* index in [0, m) from a draw: the high 32 bits scaled by m */
static uint64_t pick(uint64_t draw, uint64_t m) { return ((draw >> 32) * m) >> 32; }

int or_walks(int64_t n, const int64_t *out_ptr, const int32_t *out_idx, const int32_t *outdeg,
             uint64_t seed, int64_t n_walks, uint64_t *counts, int64_t *steps)
{
    if (n <= 0 || n_walks < 0) return OR_BAD_ARG;
    for (int64_t v = 0; v < n; ++v) counts[v] = 0;
    int64_t total = 0;
    for (int64_t j = 0; j < n_walks; ++j) {
        /* walk j: the k-th draw is the k-th output of the SplitMix64 stream
         * whose state starts at splitmix64(seed ^ j) */
        const uint64_t s0 = splitmix64(seed ^ (uint64_t)j);
        uint64_t k = 0;
        int64_t v = (int64_t)pick(splitmix64(s0 + k * 0x9e3779b97f4a7c15ULL), (uint64_t)n);
        while (outdeg[v] > 0) {
            ++k;
            const uint64_t i = pick(splitmix64(s0 + k * 0x9e3779b97f4a7c15ULL),
                                    (uint64_t)outdeg[v]);
            v = out_idx[out_ptr[v] + (int64_t)i];
            ++total;
        }
        counts[v] += 1;
    }
    if (steps) *steps = total;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* p-proportion of centrality (Sec. VII-B, Eq. 3)                            */
/* C_p = sum_{x in L_p} c(x) / sum_{x in L} c(x), L_p = minima with          */
/* f <= (1+p) f_opt (the non-strict reading, so that p = 0 keeps the optimum) */
/* ------------------------------------------------------------------------ */

int or_centrality(int64_t n, const uint8_t *is_min, const double *node_fit, const double *x,
                  double f_opt, const double *p, int32_t n_p, double *cp)
{
    if (n <= 0 || n_p < 0) return OR_BAD_ARG;
    for (int k = 0; k < n_p; ++k) {
        if (!(p[k] >= 0.0)) return OR_BAD_ARG;
        double thr = f_opt * (1.0 + p[k]);
        double sl = 0.0, cl = 0.0, sp = 0.0, cpk = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            if (!is_min[v]) continue;
            sl = neumaier_add(sl, x[v], &cl);
            if (node_fit[v] <= thr) sp = neumaier_add(sp, x[v], &cpk);
        }
        sl += cl;
        sp += cpk;
        if (!(sl > 0.0)) return OR_EMPTY;
        cp[k] = sp / sl;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* the naive metric (Sec. VII-A): f_opt / f(x) for every local minimum x,     */
/* in ascending node order                                                    */
/* ------------------------------------------------------------------------ */

int or_minima_fraction(int64_t n, const uint8_t *is_min, const double *node_fit, double f_opt,
                       double *frac, int64_t *n_out)
{
    if (n <= 0) return OR_BAD_ARG;
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v)
        if (is_min[v]) frac[k++] = f_opt / node_fit[v];
    *n_out = k;
    return k ? OR_OK : OR_EMPTY;
}
