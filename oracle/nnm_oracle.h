/*
 * nnm_oracle.h -- CPU oracle for nearest-neighbour-method (NNM) clustering.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path: only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is computed in IEEE binary64 with round-to-nearest and no fused
 * multiply-add (the file is compiled with -ffp-contract=off), in the plain order
 * written below, so that results are reproducible bit for bit.
 *
 * Definitions (Litvinenko, "Parallel algorithms for problems of cluster analysis
 * with very large amount of data", arXiv:1402.3789):
 *   D(i,j)   squared Euclidean distance of Eq. (1), summed feature by feature:
 *            D = ((t_0 + t_1) + t_2) + ... + t_{d-1},  t_k = e_k * e_k,
 *            e_k = (double)x_ik - (double)x_jk.  Decisions compare D; the reported
 *            distance is sqrt(D) (correctly rounded).
 *   key(i,j) (D, min(i,j), max(i,j)) compared lexicographically: a total order on
 *            pairs, so the single-linkage merge tree (the minimum spanning tree
 *            under this order) is unique.
 */
#ifndef NNM_ORACLE_H
#define NNM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One tree edge / candidate pair: a < b. */
typedef struct {
    uint32_t a;
    uint32_t b;
    double D;
} or_edge;

/* One accepted merge, in acceptance order. */
typedef struct {
    uint32_t a;        /* smaller row index of the joining pair */
    uint32_t b;        /* larger row index */
    double D;          /* squared distance of the pair */
    double dist;       /* sqrt(D) */
    int64_t new_size;  /* size of the cluster formed */
} or_merge;

/* Restrictions of the "Problem statement" / "Problem settings" sections.
 * Zero (or max_join_dist <= 0 / not finite) disables a restriction. */
typedef struct {
    double max_join_dist;
    int64_t kl1_stop_clusters;
    int64_t kl2_max_pre_size;
    int64_t kl3_max_size;
    int64_t kl4_min_size;
} or_restrictions;

/* Metrics: Eq. (1) (its square is D), and the two the paper leaves open to choose. */
#define OR_EUCLIDEAN 0
#define OR_MANHATTAN 1
#define OR_CHEBYSHEV 2

/* The metric of all later calls (default OR_EUCLIDEAN). */
void or_set_metric(int32_t metric);

/* D(x, y) in the canonical order (Eq. (1) squared for OR_EUCLIDEAN). */
double or_dist(const float *x, const float *y, int32_t d);

/* Fill out[m] = D(rows_i[m], rows_j[m]) for m < count. */
void or_dist_pairs(const float *X, int32_t d, const int64_t *rows_i, const int64_t *rows_j,
                   int64_t count, double *out);

/* Exact k nearest neighbours of each query row (self excluded), ordered by (D, j).
 * idx_out / D_out: [nq][k]. Returns 0, or -1 on bad arguments. */
int or_knn(const float *X, int64_t N, int32_t d, const int64_t *queries, int64_t nq,
           int32_t k, int32_t threads, uint32_t *idx_out, double *D_out);

/* Single-linkage merge tree by the paper's batched procedure: P minimal pairs per
 * pass, merged in order, pairs already inside one cluster skipped, repeated.
 * edges_out: capacity N-1, filled in key order. Returns edge count, or -1. */
int64_t or_nnm_batched(const float *X, int64_t N, int32_t d, int64_t P, int32_t threads,
                       or_edge *edges_out);

/* The same tree by Prim's algorithm (dense, O(N^2)), edges sorted by key. */
int64_t or_prim(const float *X, int64_t N, int32_t d, int32_t threads, or_edge *edges_out);

/* The same tree by Kruskal over all N(N-1)/2 pairs (small N only). */
int64_t or_kruskal_allpairs(const float *X, int64_t N, int32_t d, or_edge *edges_out);

/* Restrictions applied to a key-sorted tree (tree semantics). Returns merge count. */
int64_t or_restrict_tree(const or_edge *edges, int64_t m, int64_t N, const or_restrictions *r,
                         or_merge *merges_out);

/* Restrictions applied to every pair in key order (the paper-literal reading),
 * small N only. Returns merge count, or -1. */
int64_t or_restrict_literal(const float *X, int64_t N, int32_t d, const or_restrictions *r,
                            or_merge *merges_out);

/* Dense labels 0..K-1, ordered by each cluster's smallest member. Returns K. */
int64_t or_labels(const or_merge *merges, int64_t m, int64_t N, int32_t *labels_out);

/* Sort edges by key in place. */
void or_sort_edges(or_edge *e, int64_t m);

#ifdef __cplusplus
}
#endif
#endif
