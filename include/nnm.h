/*
 * nnm.h -- C ABI of the GB300 (sm_103a) nearest-neighbour-method clustering library.
 *
 * Method: N. Litvinenko, "Parallel algorithms for problems of cluster analysis with
 * very large amount of data" (arXiv:1402.3789).  Rows are records, columns features;
 * the distance is Eq. (1), the Euclidean distance.  Clusters are built by the nearest
 * neighbour method (single linkage): pairs join in increasing order of distance, a
 * pair already inside one cluster is skipped ("General description of the algorithm
 * for constructing the set of minimum distances"), and the restrictions of "Problem
 * statement" / "Problem settings" (maximum joining distance, KL1..KL4) decide which
 * joins happen.
 *
 * Definitions used by every entry point:
 *   D(i,j)    squared Eq. (1) distance in IEEE binary64, features summed in order:
 *             D = ((t_0 + t_1) + ...) + t_{d-1},  t_k = e_k*e_k,
 *             e_k = (double)X[i][k] - (double)X[j][k], round-to-nearest, no FMA.
 *   key(i,j)  (D(i,j), min(i,j), max(i,j)) compared lexicographically.  Ties in
 *             distance, which the paper leaves open, are broken by this order, so
 *             the merge tree and the labels are unique.
 *
 * Conventions:
 *   - Pointers named *_dev are CUDA device pointers on the current device; *_host
 *     are host pointers.  All buffers are caller-owned unless stated otherwise.
 *   - Work is enqueued on the stream given to nnm_create; every call returns after
 *     its work has completed (the call synchronises that stream).
 *   - Row indices are uint32; N < 2^31.
 *   - No call throws; each returns an nnm_status, also kept in the context and
 *     described by nnm_last_error().
 */
#ifndef NNM_H
#define NNM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NNM_OK = 0,
    NNM_EINVAL = 1,       /* bad argument (sizes, k, restrictions, null pointers)          */
    NNM_ENONFINITE = 2,   /* X holds NaN or +-Inf (the main module's data check)           */
    NNM_ENOMEM = 3,       /* device workspace could not be allocated                       */
    NNM_ECUDA = 4,        /* a CUDA runtime call failed                                    */
    NNM_ETIMEOUT = 5,     /* a bounded device-side wait gave up (the context stays usable) */
    NNM_EUNSUPPORTED = 6  /* metric / precision / size not provided by this build          */
} nnm_status;

/* Eq. (1) (Euclidean) is the default; the paper allows another metric where a task
 * needs one.  With
 * e_k = (double)x_ik - (double)x_jk in feature order, binary64, no contraction:
 *   NNM_EUCLIDEAN  D = sum of e_k^2 (Eq. (1) squared); a merge's length is sqrt(D) and the
 *                  maximum joining distance c admits D <= c*c.
 *   NNM_MANHATTAN  D = sum of |e_k|;  NNM_CHEBYSHEV  D = max |e_k|.  For these two the
 *                  length is D itself and c admits D <= c.  They use the FP32 direct
 *                  candidates (NNM_PREC_FP32); other precisions give EUNSUPPORTED. */
typedef enum { NNM_EUCLIDEAN = 0, NNM_MANHATTAN = 1, NNM_CHEBYSHEV = 2 } nnm_metric;

/* How candidate distances are produced before the exact binary64 re-rank.  Every
 * precision returns the same, exact result; they differ only in speed.
 *   NNM_PREC_FP32          direct differences sum((x-y)^2) in FP32 on CUDA cores.
 *   NNM_PREC_BF16_RERANK   |x|^2 + |y|^2 - 2 x.y as a BF16 tensor-core (tcgen05)
 *                          product with FP32 accumulation, centred data.
 *   NNM_PREC_FP16_RERANK   the same with FP16 operands and one power-of-two scale.
 *   NNM_PREC_BF16X3_RERANK BF16 operands with each value split as hi + lo (three
 *                          products per feature, K = 3d + 6 padded to 16): BF16 tensor
 *                          math with a 16-bit mantissa; d <= 30. */
typedef enum {
    NNM_PREC_FP32 = 0,
    NNM_PREC_BF16_RERANK = 1,
    NNM_PREC_FP16_RERANK = 2,
    NNM_PREC_BF16X3_RERANK = 3
} nnm_precision;

typedef struct nnm_ctx nnm_ctx;

/* Tuning knobs; zero-initialise for defaults. */
typedef struct {
    int32_t cache_k;       /* exact nearest neighbours cached per row for the merge rounds
                              (0: default per precision; 1..16)                           */
    int32_t freeze_at_cap; /* 1: stop extending the tree past the maximum joining distance
                              (the restricted result is unchanged; the merge tree returned
                              by nnm_get_tree then holds only edges within the cap)        */
    int32_t col_split;     /* 0: automatic; >0: number of column ranges per row tile      */
    int32_t no_tile_pruning; /* 1: evaluate every column tile (no skipping by bounding
                                spheres or landmark distances; results are identical,
                                only slower)                                               */
    int64_t wait_limit_ns; /* 0: 2 s.  Longest time one device-side wait of the tensor-core
                              sweep (for a copied tile, an accumulator, a planned tile or a
                              threshold) may take before the kernel gives up, raises its
                              error flag and exits; the call then returns NNM_ETIMEOUT and
                              the context stays usable.  1 .. 60e9 (larger is taken as 60 s);
                              negative: EINVAL.  See nnm_set_wait_limit.                   */
} nnm_options;

/* Restrictions ("Problem statement"; "Problem settings").  Zero disables each one.
 *   max_join_dist      > 0 and finite: a pair joins only if D <= fl64(c*c) (Euclidean;
 *                      D <= c for the other metrics).
 *   kl1_stop_clusters  KL1: no join once the number of clusters has reached KL1.
 *   kl2_max_pre_size   KL2: no join if either cluster already has more than KL2 rows
 *                      (a cluster may end larger than KL2, as the paper allows).
 *   kl3_max_size       KL3: no join if the two sizes add up to more than KL3 (KL3 > KL2).
 *   kl4_min_size       KL4: joins that touch a cluster with fewer than KL4 rows go
 *                      first: one pass in key order makes only those joins and defers
 *                      the rest, a second pass in key order handles the deferred ones.
 *   semantics          0: the gates act on the merge-tree edges in key order (tree
 *                      semantics, the default).  1: the gates act on every pair in key
 *                      order, as the paper's batched procedure over all pairs walks them
 *                      ("General description of the algorithm for constructing the set
 *                      of minimum distances"); with KL2 or KL3 a cluster may then join
 *                      through a pair that is not a tree edge.  Semantics 1 costs O(N^2)
 *                      pair evaluations per batch of joins and takes one instance of at
 *                      most 262,144 rows (else NNM_EUNSUPPORTED); the tree is not built.
 *                      Other values: NNM_EINVAL.
 * A join blocked by a gate is not retried (sizes only grow). */
typedef struct {
    double max_join_dist;
    int64_t kl1_stop_clusters;
    int64_t kl2_max_pre_size;
    int64_t kl3_max_size;
    int64_t kl4_min_size;
    int32_t semantics;
    int32_t reserved;
} nnm_restrictions;

/* One join, in the order the joins are made.  32 bytes. */
typedef struct {
    uint32_t a;        /* smaller row index of the joining pair */
    uint32_t b;        /* larger row index */
    double D;          /* D(a,b) */
    double dist;       /* length: sqrt(D) correctly rounded (Euclidean), D (others) */
    int64_t new_size;  /* rows in the cluster the join forms */
} nnm_merge;

/* One merge-tree edge (a < b).  16 bytes. */
typedef struct {
    uint32_t a;
    uint32_t b;
    double D;
} nnm_edge;

/* Per-context counters of the last nnm_nearest / nnm_cluster call. */
typedef struct {
    double ms_prep;          /* nnm_create: checks, centring, operand layout        */
    double ms_sweep;         /* all-pairs candidate sweeps (full and row rescans)  */
    double ms_rerank;        /* binary64 re-rank and candidate selection           */
    double ms_rounds;        /* component minima, hooking, pointer jumping         */
    double ms_sort;          /* device merge sort of the tree edges                */
    double ms_restrict;      /* restriction walk                                   */
    double ms_labels;        /* labels                                             */
    double ms_total;         /* whole call, CUDA events on the stream             */
    int64_t rounds;          /* merge rounds                                       */
    int64_t sweep_launches;  /* candidate-sweep kernel launches                    */
    int64_t pairs_evaluated; /* ordered (row, column) candidate evaluations        */
    int64_t rows_rescanned;  /* row rescans after the first sweep                  */
    int64_t rows_overflowed; /* rows whose candidate list needed the collect pass  */
    int64_t rerank_pairs;    /* binary64 distances computed                        */
    int64_t max_candidates;  /* most candidates re-ranked for one row              */
    double max_abs_err;      /* max |candidate distance - D| over re-ranked pairs  */
    double max_rel_err;      /* the same relative to D (pairs with D > 0)          */
    double sweep_ms_per_launch_full; /* mean duration of a full-matrix sweep launch */
    int64_t full_sweep_pairs;        /* pairs of one full-matrix sweep launch       */
    int32_t k_pad;           /* tensor-core K (0 on the FP32 path)                 */
    int32_t cache_k;         /* cached neighbours per row                          */
    double scale;            /* power-of-two operand scale (tensor paths)          */
    int64_t kernel_launches; /* kernels this library launched during the call      */
    int64_t tiles_skipped;   /* column tiles skipped by the bounding-sphere bound   */
    int64_t tiles_swept;     /* column tiles evaluated                              */
    int64_t full_sweep_pairs_computed; /* (row, column) pairs in the tiles the full-matrix
                                          sweep launch evaluated (256 rows x tile width
                                          per tile): the work the launch did            */
} nnm_stats;

/* nnm_create -- "main module" ("Objectives of the main module"): validate the data
 * array, derive auxiliary settings, fill the working fields.
 *   X_dev   row-major float32 [N][d] on the device; borrowed: it must stay alive and
 *           unchanged until nnm_destroy (the exact re-rank reads it).
 *   N       rows, 1 <= N < 2^31.   d  features, 1 <= d <= 32.
 *   metric  see nnm_metric.         precision  see nnm_precision.
 *   cuda_stream  cudaStream_t to enqueue on (NULL: the legacy default stream).
 *   options      may be NULL.
 *   out     receives the context (NULL on failure).
 * Errors: EINVAL (sizes, null pointers), ENONFINITE (NaN/Inf in X), EUNSUPPORTED
 * (metric or precision; NNM_PREC_BF16X3_RERANK with d > 30), ENOMEM, ECUDA.  The context owns its device workspace:
 * about N*(4*d_pad + 2*2*K_pad + 24*cache_k + 96) bytes. */
nnm_status nnm_create(const float *X_dev, int64_t N, int32_t d, nnm_metric metric,
                      nnm_precision precision, void *cuda_stream, const nnm_options *options,
                      nnm_ctx **out);

/* nnm_create_batched -- one context for many independent problems (instances) that share
 * d: instance b is rows [offsets_host[b], offsets_host[b+1]) of X_dev.  Distances,
 * neighbours and merges never cross instances: nnm_nearest gives each row its k nearest
 * within its own instance; nnm_cluster gives the merge forest (one tree per instance,
 * N - n_instances edges; nnm_get_tree returns it grouped by instance, each group in key
 * order), applies the restrictions to each instance on its own (KL1 counts the clusters
 * of that instance), returns the merges grouped by instance (each group in acceptance
 * order) and labels over all rows.  Instances with fewer
 * features are passed padded with zero columns: zero columns leave every distance and
 * therefore every result unchanged.  The paper runs one problem per program start; this
 * form serves many small problems in one pass of each kernel.
 *   offsets_host  int64 [n_instances + 1] host memory, 0 = offsets[0] < ... <
 *                 offsets[n_instances] = N < 2^31; read during the call only.
 *   n_instances   1 .. 65535.
 * Other arguments and errors as nnm_create; EINVAL also for bad offsets.  nnm_nearest
 * requires k < rows of the smallest instance. */
nnm_status nnm_create_batched(const float *X_dev, const int64_t *offsets_host, int64_t n_instances, int32_t d,
                              nnm_metric metric, nnm_precision precision, void *cuda_stream,
                              const nnm_options *options, nnm_ctx **out);

/* nnm_nearest -- exact k nearest neighbours of every row (self excluded), in order
 * of (D, index): the per-row minima of the second and third parallel items of
 * "Overall idea of the algorithm" (all pairwise distances, minimum selection).
 *   k        1 <= k <= 16 and k < N (EINVAL otherwise).
 *   idx_dev  uint32 [N][k] device, written.   D_dev  float64 [N][k] device, written. */
nnm_status nnm_nearest(nnm_ctx *ctx, int32_t k, uint32_t *idx_dev, double *D_dev);

/* nnm_cluster -- the NNM merge tree (single linkage, minimum spanning tree under
 * key order) and the restricted joins on it.
 *   restrictions  may be NULL (no restriction).  EINVAL: negative values, KL3 <= KL2
 *                 with both set (the paper takes KL3 above KL2), semantics not 0 or 1;
 *                 EUNSUPPORTED: semantics 1 beyond its limits (see nnm_restrictions).
 *   merges_dev    nnm_merge [N-1] device, the accepted joins in acceptance order.
 *   n_merges_host receives their number.
 *   labels_dev    int32 [N] device: cluster of every row, 0..K-1, numbered by each
 *                 cluster's smallest row index.
 *   n_clusters_host  receives K.
 * N >= 2 required.  Without KL2, KL3 and KL4 the accepted joins are a prefix of the
 * key-ordered tree and are computed in parallel; the first such call allocates up to
 * about 220 bytes per tree edge of scratch in the context (kept until nnm_destroy). */
nnm_status nnm_cluster(nnm_ctx *ctx, const nnm_restrictions *restrictions, nnm_merge *merges_dev,
                       int64_t *n_merges_host, int32_t *labels_dev, int64_t *n_clusters_host);

/* nnm_cluster_host -- nnm_create + nnm_cluster + nnm_destroy from and to host memory, for
 * callers whose rows live on the host: X is copied to the device, clustered, and the
 * merges and labels are copied back, all on cuda_stream.  The paper's program reads its
 * records from host memory and writes its results back ("Objectives of the main module").
 *   X_host          row-major float32 [N][d] host memory (page-locked memory copies
 *                   fastest); read during the call only.
 *   metric, precision, options   as for nnm_create;  restrictions  as for nnm_cluster.
 *   merges_host     nnm_merge [N-1] host memory, written;  n_merges_host receives the count.
 *   labels_host     int32 [N] host memory, written;  n_clusters_host receives K.
 * The device memory the call needs (X, merges, labels and the context's workspace) is
 * taken from the library's pool and given back inside the call (see nnm_destroy).  N >= 2.  Errors: those of nnm_create and
 * nnm_cluster. */
nnm_status nnm_cluster_host(const float *X_host, int64_t N, int32_t d, nnm_metric metric,
                            nnm_precision precision, const nnm_options *options,
                            const nnm_restrictions *restrictions, void *cuda_stream, nnm_merge *merges_host,
                            int64_t *n_merges_host, int32_t *labels_host, int64_t *n_clusters_host);

/* nnm_set_wait_limit -- change the context's wait limit (nnm_options.wait_limit_ns) for
 * the calls that follow; 0 restores the 2 s default.  EINVAL if wait_limit_ns < 0. */
nnm_status nnm_set_wait_limit(nnm_ctx *ctx, int64_t wait_limit_ns);

/* nnm_get_tree -- copy the merge tree of the last nnm_cluster call (edges sorted by
 * key; N-1 of them unless freeze_at_cap stopped it early).
 *   edges_dev  nnm_edge [N-1] device.   n_edges_host receives the count. */
nnm_status nnm_get_tree(nnm_ctx *ctx, nnm_edge *edges_dev, int64_t *n_edges_host);

/* nnm_get_stats -- counters of the last call. */
nnm_status nnm_get_stats(const nnm_ctx *ctx, nnm_stats *out);

/* nnm_last_error -- human-readable description of the last failure ("" if none).
 * Owned by the context; valid until the next call on it. */
const char *nnm_last_error(const nnm_ctx *ctx);

/* nnm_status_string -- static name of a status code. */
const char *nnm_status_string(nnm_status s);

/* nnm_destroy -- free the context and its device workspace.  NULL is ignored.
 * Device workspace (of contexts, of calls and of nnm_cluster_host) comes from a memory
 * pool of the library, one per device, allocated and freed in stream order on the
 * context's stream; freed workspace goes back to that pool, which keeps the memory it
 * has grown to for the life of the process (the default pool is not touched). */
void nnm_destroy(nnm_ctx *ctx);

/* Largest N accepted by nnm_restrict_static. */
#define NNM_STATIC_MAX_ROWS (1 << 20)

/* nnm_restrict_static -- the restriction walk and the labels of nnm_cluster, applied to
 * a merge tree the caller already holds, without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate at call time (device memory owned by an application pool or arena that must
 * not see foreign cudaMalloc/cudaFree, which synchronise the device and fragment the
 * pool; services with a memory budget fixed at start-up).  Its scratch is one fixed
 * device array of about 21 MB inside this library, held on every GPU that loads the
 * library until the process exits.
 *   tree_dev       nnm_edge [n_edges] device, one instance's tree sorted by key, as
 *                  nnm_get_tree returns it for a context of one instance (a batched
 *                  context's tree, grouped by instance, is not accepted);
 *                  0 <= n_edges <= N-1.  Checked on the device before the walk: every
 *                  endpoint below N, a < b, D finite and >= 0, keys strictly increasing;
 *                  a tree that fails gives NNM_EINVAL and no result.
 *   N              rows, 2 <= N <= NNM_STATIC_MAX_ROWS (larger N: NNM_EUNSUPPORTED, no launch).
 *   metric         the metric the tree's D values are in (the context's metric): it fixes
 *                  the cap's units and the merges' reported length, as for nnm_cluster;
 *                  an unknown value gives NNM_EINVAL.
 *   restrictions   as for nnm_cluster (may be NULL); same EINVAL rules; semantics 1 (which
 *                  needs the rows, not a tree) gives NNM_EUNSUPPORTED.
 *   merges_dev, n_merges_host, labels_dev, n_clusters_host  as for nnm_cluster.
 *   cuda_stream    cudaStream_t to enqueue on (NULL: the legacy default stream); the call
 *                  returns after its work has completed.
 * The first call on each device looks up the scratch array's device address, with that
 * device current; make it before any stream capture.  All calls share the array: calls
 * whose work overlaps on the GPU race and corrupt each other; calls ordered on one
 * stream are safe.  Errors: EINVAL, EUNSUPPORTED, ECUDA. */
nnm_status nnm_restrict_static(const nnm_edge *tree_dev, int64_t n_edges, int64_t N, nnm_metric metric,
                               const nnm_restrictions *restrictions, nnm_merge *merges_dev,
                               int64_t *n_merges_host, int32_t *labels_dev, int64_t *n_clusters_host,
                               void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
