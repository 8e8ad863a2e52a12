/*
 * ffg_oracle.h -- plain single-threaded CPU oracle for the fitness flow graph
 * (FFG) metric.  TEST INFRASTRUCTURE ONLY: used by the test suite, the
 * smoke check and the benchmark's CPU baseline, never by the library.
 *
 * It shares nothing with the CUDA library (no header, no helper, no table).
 * Every routine is the paper's definition written out in the most direct way:
 *   - search space: Cartesian product of integer value lists (Sec. III-B),
 *   - Hamming and adjacent neighbourhoods (Sec. III-B, Eq. 2 and the
 *     adjacent-value restriction that follows it),
 *   - local minimum: no neighbour with better fitness (Sec. III-B),
 *   - failed configurations carry fitness 1e10 (Sec. V),
 *   - FFG: an edge to every neighbour with lower fitness (Sec. VII-B),
 *   - PageRank on the column-normalised adjacency matrix (Sec. VII-B),
 *   - p-proportion of centrality C_p (Sec. VII-B, Eq. 3).
 */
#ifndef FFG_ORACLE_H
#define FFG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_BAD_ARG = 1, OR_OVERFLOW = 2, OR_NO_MEMORY = 3, OR_NOT_CONVERGED = 4,
       OR_EMPTY = 5 };
enum { OR_HAMMING = 0, OR_ADJACENT = 1 };
enum { OR_PROD_LE = 0, OR_PROD_GE = 1, OR_DIVIDES = 2, OR_PROD_LE_PROD = 3 };

typedef struct {
    int32_t kind;        /* OR_PROD_LE ... */
    int32_t n_a, n_b;    /* number of factor indices in a[] and b[] */
    int32_t a[16], b[16];/* parameter indices of the two products */
    int64_t bound;
} or_clause;

typedef struct {
    int32_t n_params;
    const int32_t *radix;      /* n_params list lengths */
    const int64_t *values;     /* concatenated value lists */
    int32_t n_clauses;
    const or_clause *clauses;
} or_space;

typedef struct {
    int64_t n_raw, n_nodes, n_edges;
    int64_t *node_raw;   /* raw index of every node, ascending */
    int64_t *out_ptr;    /* n_nodes + 1 */
    int32_t *out_idx;    /* n_edges, per row ascending */
    int64_t *in_ptr;     /* n_nodes + 1 */
    int32_t *in_idx;     /* n_edges, per row ascending */
    int32_t *outdeg;     /* n_nodes */
    uint8_t *is_min;     /* n_nodes */
    uint8_t *failed;     /* n_nodes */
    double  *node_fit;   /* n_nodes, fitness as given */
    double   f_opt;      /* minimum non-failed fitness, +inf if none */
} or_graph;

/* Raw size = product of list lengths; OR_OVERFLOW above 2^62. */
int or_raw_count(const or_space *s, int64_t *n_raw);

/* valid[r] = 1 iff every clause holds for raw point r (row-major digits). */
int or_valid_mask(const or_space *s, uint8_t *valid);

/* Build the FFG.  Arrays are malloc'ed; release with or_graph_free. */
int or_build(const or_space *s, const double *fitness_raw, int nbh, double fail_thr, or_graph *g);
void or_graph_free(or_graph *g);

/* Damped power iteration (uniform teleport, uniform dangling), FP64. */
int or_pagerank_power(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                      const int32_t *outdeg, double alpha, double tol, int32_t max_iter,
                      double *x, int32_t *iters, double *residual);

/* Fixed point of the same iteration solved directly on the DAG. */
int or_pagerank_exact(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                      const int32_t *outdeg, const uint8_t *failed, const double *node_fit,
                      double alpha, double *x);

/* y[v] = 1 + d * sum_{u -> v} y[u] / outdeg[u] in topological order, d in
 * [0, 1]; y / sum y is or_pagerank_exact's result for d < 1. */
int or_dag_values(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                  const int32_t *outdeg, const uint8_t *failed, const double *node_fit,
                  double d, double *y);

/* Probability that a walk from a uniformly random node, moving to uniformly
 * random better neighbours, passes each node (ends there, at sinks). */
int or_absorption(int64_t n, const int64_t *in_ptr, const int32_t *in_idx,
                  const int32_t *outdeg, const uint8_t *failed, const double *node_fit,
                  double *a);

/* SplitMix64 output for state x (the state advanced by the golden gamma). */
uint64_t or_splitmix64(uint64_t x);

/* n_walks improving walks: walk j starts at a uniformly random node and moves
 * to a uniformly random out-neighbour until a node without out-edges;
 * counts[v] = walks that ended at v; *steps = moves made. */
int or_walks(int64_t n, const int64_t *out_ptr, const int32_t *out_idx, const int32_t *outdeg,
             uint64_t seed, int64_t n_walks, uint64_t *counts, int64_t *steps);

/* f_opt / f(x) for every local minimum, ascending node order; *n_out = count. */
int or_minima_fraction(int64_t n, const uint8_t *is_min, const double *node_fit, double f_opt,
                       double *frac, int64_t *n_out);

/* C_p for every threshold p[k] (fractions, e.g. 0.05). */
int or_centrality(int64_t n, const uint8_t *is_min, const double *node_fit, const double *x,
                  double f_opt, const double *p, int32_t n_p, double *cp);

#ifdef __cplusplus
}
#endif
#endif
