/*
 * test_oracle.c -- self-test of the CPU oracle in plain C (TEST
 * INFRASTRUCTURE: built and run by the test suite, never by the library).
 *
 * Each check compares the oracle with a value fixed by the paper or by the
 * mathematics, not by the oracle itself:
 *   - raw sizes of the paper's four kernel spaces (products of the list
 *     lengths of its appendix table of tunable parameters; Sec. V table);
 *   - the adjacent-neighbour example of Sec. III-B ([16, 32, 64, 128]: the
 *     neighbours of 64 are 32 and 128, the only neighbour of 128 is 64);
 *   - a chain (one parameter, adjacent, fitness falling along the list):
 *     y_k = (1 - a^(k+1)) / (1 - a);
 *   - a tournament (one parameter with three values, Hamming, distinct
 *     fitness): y = 1, 1 + a/2, 1 + 3a/2 + a^2/2 from worst to best;
 *   - C_p of a hand example (Sec. VII-B, Eq. 3, non-strict threshold);
 *   - the first SplitMix64 outputs from state 0 (the published sequence).
 * Prints one line per failed check and exits non-zero if any failed.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "ffg_oracle.h"

static int failures = 0;

static void check(int ok, const char *what) {
    if (!ok) {
        printf("FAIL: %s\n", what);
        ++failures;
    }
}

static int close_rel(double a, double b, double tol) {
    return fabs(a - b) <= tol * fmax(1.0, fabs(b));
}

/* a space of one parameter whose values are vals[0..n) */
static or_space one_param(int32_t *radix, const int64_t *vals, int32_t n) {
    or_space s;
    radix[0] = n;
    s.n_params = 1;
    s.radix = radix;
    s.values = vals;
    s.n_clauses = 0;
    s.clauses = NULL;
    return s;
}

static void raw_sizes(void) {
    static const int32_t conv[] = {12, 6, 8, 8, 2, 2};
    static const int32_t gemm[] = {4, 4, 3, 3, 3, 3, 4, 4, 2, 2};
    static const int32_t pnpoly[] = {31, 11, 4, 2, 3};
    static const int32_t mi50[] = {8, 6, 3, 3, 2};
    static int64_t vals[64];
    struct { const int32_t *r; int32_t n; int64_t want; const char *name; } cases[] = {
        {conv, 6, 18432, "raw size of the convolution space"},
        {gemm, 10, 82944, "raw size of the GEMM space"},
        {pnpoly, 5, 8184, "raw size of the PnPoly space"},
        {mi50, 5, 864, "raw size of the convolution (MI50) space"},
    };
    for (int k = 0; k < 64; ++k) vals[k] = k + 1;
    for (int c = 0; c < 4; ++c) {
        or_space s = {cases[c].n, cases[c].r, vals, 0, NULL};
        int64_t n = -1;
        check(or_raw_count(&s, &n) == OR_OK && n == cases[c].want, cases[c].name);
    }
}

static void adjacent_example(void) {
    static const int64_t vals[] = {16, 32, 64, 128};
    int32_t radix[1];
    or_space s = one_param(radix, vals, 4);
    /* distinct fitness, so every neighbour pair carries exactly one edge */
    const double fit[] = {3.0, 1.0, 4.0, 2.0};
    or_graph g;
    check(or_build(&s, fit, OR_ADJACENT, 1e10, &g) == OR_OK, "adjacent example: build");
    if (failures) return;
    /* neighbours per node = out-degree + in-degree */
    const int64_t want[] = {1, 2, 2, 1};
    for (int v = 0; v < 4; ++v) {
        const int64_t deg = g.outdeg[v] + (g.in_ptr[v + 1] - g.in_ptr[v]);
        check(deg == want[v], "adjacent example: neighbour count");
    }
    /* 64 (node 2, f = 4) is worse than both 32 and 128: edges 2->1 and 2->3 */
    check(g.out_ptr[3] - g.out_ptr[2] == 2 && g.out_idx[g.out_ptr[2]] == 1 &&
              g.out_idx[g.out_ptr[2] + 1] == 3,
          "adjacent example: the neighbours of 64 are 32 and 128");
    /* 128 (node 3, f = 2) has the single neighbour 64, which is worse */
    check(g.outdeg[3] == 0 && g.in_ptr[4] - g.in_ptr[3] == 1 && g.in_idx[g.in_ptr[3]] == 2,
          "adjacent example: the only neighbour of 128 is 64");
    or_graph_free(&g);
}

static void chain(void) {
    enum { n = 9 };
    int64_t vals[n];
    double fit[n];
    for (int k = 0; k < n; ++k) {
        vals[k] = k;
        fit[k] = (double)(n - k);  /* falling along the list */
    }
    int32_t radix[1];
    or_space s = one_param(radix, vals, n);
    or_graph g;
    check(or_build(&s, fit, OR_ADJACENT, 1e10, &g) == OR_OK, "chain: build");
    if (failures) return;
    const double a = 0.85;
    double y[n];
    check(or_dag_values(g.n_nodes, g.in_ptr, g.in_idx, g.outdeg, g.failed, g.node_fit, a, y) ==
              OR_OK,
          "chain: dag values");
    for (int k = 0; k < n; ++k)
        check(close_rel(y[k], (1.0 - pow(a, k + 1)) / (1.0 - a), 1e-14),
              "chain: y_k = (1 - a^(k+1)) / (1 - a)");
    or_graph_free(&g);
}

static void tournament(void) {
    static const int64_t vals[] = {1, 2, 3};
    int32_t radix[1];
    or_space s = one_param(radix, vals, 3);
    const double fit[] = {2.0, 3.0, 1.0};  /* worst: node 1, then node 0, best: node 2 */
    or_graph g;
    check(or_build(&s, fit, OR_HAMMING, 1e10, &g) == OR_OK, "tournament: build");
    if (failures) return;
    const double a = 0.7;
    double y[3];
    check(or_dag_values(g.n_nodes, g.in_ptr, g.in_idx, g.outdeg, g.failed, g.node_fit, a, y) ==
              OR_OK,
          "tournament: dag values");
    check(close_rel(y[1], 1.0, 1e-15), "tournament: worst node y = 1");
    check(close_rel(y[0], 1.0 + a / 2, 1e-15), "tournament: middle node y = 1 + a/2");
    check(close_rel(y[2], 1.0 + 1.5 * a + 0.5 * a * a, 1e-15),
          "tournament: best node y = 1 + 3a/2 + a^2/2");
    /* the exact PageRank is y normalised */
    double x[3];
    check(or_pagerank_exact(g.n_nodes, g.in_ptr, g.in_idx, g.outdeg, g.failed, g.node_fit, a, x) ==
              OR_OK,
          "tournament: exact pagerank");
    const double sy = y[0] + y[1] + y[2];
    for (int v = 0; v < 3; ++v) check(close_rel(x[v], y[v] / sy, 1e-15), "tournament: x = y / sum y");
    or_graph_free(&g);
}

static void centrality(void) {
    /* minima at f = 1.00, 1.04 and 2.00 holding 0.1, 0.2 and 0.4 of the rank */
    const uint8_t is_min[] = {1, 1, 0, 1};
    const double fit[] = {1.0, 1.04, 5.0, 2.0};
    const double x[] = {0.1, 0.2, 0.3, 0.4};
    const double p[] = {0.0, 0.04, 0.05, 1.0};
    const double want[] = {0.1 / 0.7, 0.3 / 0.7, 0.3 / 0.7, 1.0};
    double cp[4];
    check(or_centrality(4, is_min, fit, x, 1.0, p, 4, cp) == OR_OK, "C_p: call");
    for (int k = 0; k < 4; ++k) check(close_rel(cp[k], want[k], 1e-15), "C_p: hand example");
}

static void splitmix(void) {
    const uint64_t g = 0x9E3779B97F4A7C15ULL;
    const uint64_t want[] = {0xE220A8397B1DCDAFULL, 0x6E789E6AA1B965F4ULL,
                             0x06C45D188009454FULL};
    for (uint64_t k = 0; k < 3; ++k)
        check(or_splitmix64(k * g) == want[k], "SplitMix64: published outputs from state 0");
}

int main(void) {
    raw_sizes();
    adjacent_example();
    chain();
    tournament();
    centrality();
    splitmix();
    if (failures) {
        printf("%d oracle self-checks failed\n", failures);
        return 1;
    }
    printf("oracle self-checks passed\n");
    return 0;
}
