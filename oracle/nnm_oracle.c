/*
 * nnm_oracle.c -- plain CPU oracle for nearest-neighbour-method (NNM) clustering.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  Compile with -ffp-contract=off (no FMA contraction):
 * every floating-point value here is an IEEE binary64 round-to-nearest result of
 * the operations written, in the order written.
 *
 * Paper: N. Litvinenko, "Parallel algorithms for problems of cluster analysis with
 * very large amount of data" (arXiv:1402.3789).
 */
#define _GNU_SOURCE
#include "nnm_oracle.h"

#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------- */
/* Distance and pair order                                                    */
/* ------------------------------------------------------------------------- */

/* The metric of every distance below (Eq. (1) is Euclidean; the paper allows another
 * metric where a task needs one); set once before a computation. */
static int32_t g_metric = OR_EUCLIDEAN;

void or_set_metric(int32_t metric) { g_metric = metric; }

/* D(x, y) with e_k = (double)x_k - (double)y_k in feature order:
 *   Euclidean: Eq. (1) squared, the e_k^2 summed one after another.  Decisions use
 *              the square, which orders pairs the same way as the root.
 *   Manhattan: the |e_k| summed one after another.
 *   Chebyshev: the largest |e_k|. */
double or_dist(const float *x, const float *y, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double e = (double)x[k] - (double)y[k];
        if (g_metric == OR_MANHATTAN) {
            s = s + fabs(e);
        } else if (g_metric == OR_CHEBYSHEV) {
            double a = fabs(e);
            if (a > s) s = a;
        } else {
            double t = e * e;
            s = s + t;
        }
    }
    return s;
}

/* The length of a pair from its D: the root of a squared Euclidean D, else D. */
static double pair_length(double D) { return g_metric == OR_EUCLIDEAN ? sqrt(D) : D; }

void or_dist_pairs(const float *X, int32_t d, const int64_t *rows_i, const int64_t *rows_j,
                   int64_t count, double *out)
{
    for (int64_t m = 0; m < count; ++m)
        out[m] = or_dist(X + rows_i[m] * d, X + rows_j[m] * d, d);
}

/* key(e) = (D, a, b) with a < b; the paper leaves ties open, this order closes them. */
static int edge_less(const or_edge *p, const or_edge *q)
{
    if (p->D != q->D) return p->D < q->D;
    if (p->a != q->a) return p->a < q->a;
    return p->b < q->b;
}

static int edge_cmp(const void *p, const void *q)
{
    const or_edge *x = (const or_edge *)p, *y = (const or_edge *)q;
    if (edge_less(x, y)) return -1;
    if (edge_less(y, x)) return 1;
    return 0;
}

void or_sort_edges(or_edge *e, int64_t m) { qsort(e, (size_t)m, sizeof(or_edge), edge_cmp); }

static or_edge make_edge(int64_t i, int64_t j, double D)
{
    or_edge e;
    e.a = (uint32_t)(i < j ? i : j);
    e.b = (uint32_t)(i < j ? j : i);
    e.D = D;
    return e;
}

/* ------------------------------------------------------------------------- */
/* Threads                                                                    */
/* ------------------------------------------------------------------------- */

static int resolve_threads(int32_t t)
{
    if (t > 0) return t;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

typedef struct {
    void (*fn)(void *ctx, int tid, int nthreads);
    void *ctx;
    int tid;
    int nthreads;
} or_job;

static void *or_job_main(void *p)
{
    or_job *j = (or_job *)p;
    j->fn(j->ctx, j->tid, j->nthreads);
    return NULL;
}

/* Run fn(ctx, tid, n) on n threads (tid 0 on the caller) and join. */
static void run_threads(int n, void (*fn)(void *, int, int), void *ctx)
{
    pthread_t *th = (pthread_t *)calloc((size_t)n, sizeof(pthread_t));
    or_job *jobs = (or_job *)calloc((size_t)n, sizeof(or_job));
    for (int t = 0; t < n; ++t) {
        jobs[t].fn = fn;
        jobs[t].ctx = ctx;
        jobs[t].tid = t;
        jobs[t].nthreads = n;
    }
    for (int t = 1; t < n; ++t) pthread_create(&th[t], NULL, or_job_main, &jobs[t]);
    fn(ctx, 0, n);
    for (int t = 1; t < n; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
}

/* Sense-reversing spin barrier: Prim needs two barriers per added vertex, and a
 * sleeping barrier's wake-up latency would dominate its run time. */
typedef struct {
    atomic_int count;
    atomic_int sense;
    int n;
} spin_barrier;

static void spin_barrier_init(spin_barrier *b, int n)
{
    atomic_init(&b->count, 0);
    atomic_init(&b->sense, 0);
    b->n = n;
}

static void spin_barrier_wait(spin_barrier *b)
{
    int s = atomic_load(&b->sense);
    if (atomic_fetch_add(&b->count, 1) == b->n - 1) {
        atomic_store(&b->count, 0);
        atomic_store(&b->sense, 1 - s);
        return;
    }
    for (long spins = 0; atomic_load(&b->sense) == s; ++spins)
        if (spins > 4096) sched_yield();
}

/* ------------------------------------------------------------------------- */
/* Union-find with sizes                                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t *parent;
    int64_t *size;
} uf_t;

static void uf_init(uf_t *u, int64_t n)
{
    u->parent = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    u->size = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        u->parent[i] = i;
        u->size[i] = 1;
    }
}

static void uf_free(uf_t *u)
{
    free(u->parent);
    free(u->size);
}

static int64_t uf_find(uf_t *u, int64_t x)
{
    while (u->parent[x] != x) {
        u->parent[x] = u->parent[u->parent[x]];
        x = u->parent[x];
    }
    return x;
}

/* Join the clusters with roots ra != rb; returns the new root. */
static int64_t uf_union(uf_t *u, int64_t ra, int64_t rb)
{
    if (u->size[ra] < u->size[rb]) {
        int64_t t = ra;
        ra = rb;
        rb = t;
    }
    u->parent[rb] = ra;
    u->size[ra] += u->size[rb];
    return ra;
}

/* ------------------------------------------------------------------------- */
/* k nearest neighbours by brute force                                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    const float *X;
    int64_t N;
    int32_t d;
    const int64_t *queries;
    int64_t nq;
    int32_t k;
    uint32_t *idx_out;
    double *D_out;
} knn_ctx;

static void knn_worker(void *p, int tid, int nt)
{
    knn_ctx *c = (knn_ctx *)p;
    int32_t k = c->k;
    for (int64_t q = tid; q < c->nq; q += nt) {
        int64_t i = c->queries[q];
        const float *xi = c->X + i * c->d;
        uint32_t *bi = c->idx_out + q * k;
        double *bd = c->D_out + q * k;
        int32_t cnt = 0;
        for (int64_t j = 0; j < c->N; ++j) {
            if (j == i) continue;
            double D = or_dist(xi, c->X + j * c->d, c->d);
            /* keep the k smallest (D, j) in a sorted array */
            if (cnt == k && !(D < bd[k - 1] || (D == bd[k - 1] && (uint32_t)j < bi[k - 1])))
                continue;
            int32_t pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && (D < bd[pos - 1] || (D == bd[pos - 1] && (uint32_t)j < bi[pos - 1]))) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = D;
            bi[pos] = (uint32_t)j;
            if (cnt < k) ++cnt;
        }
        for (int32_t m = cnt; m < k; ++m) {
            bd[m] = INFINITY;
            bi[m] = UINT32_MAX;
        }
    }
}

int or_knn(const float *X, int64_t N, int32_t d, const int64_t *queries, int64_t nq, int32_t k,
           int32_t threads, uint32_t *idx_out, double *D_out)
{
    if (N < 1 || d < 1 || k < 1 || nq < 0) return -1;
    knn_ctx c = {X, N, d, queries, nq, k, idx_out, D_out};
    run_threads(resolve_threads(threads), knn_worker, &c);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The paper's batched procedure ("General description of the algorithm for    */
/* constructing the set of minimum distances"): every pass selects the P pairs  */
/* with the smallest distance, sorts them, joins clusters along them in order   */
/* (a pair already inside one cluster is skipped), and repeats.                */
/* ------------------------------------------------------------------------- */

/* Bounded max-heap of pairs (largest key on top). */
typedef struct {
    or_edge *v;
    int64_t n;
    int64_t cap;
} pheap;

static void heap_sift_up(pheap *h, int64_t i)
{
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!edge_less(&h->v[p], &h->v[i])) break;
        or_edge t = h->v[p];
        h->v[p] = h->v[i];
        h->v[i] = t;
        i = p;
    }
}

static void heap_sift_down(pheap *h, int64_t i)
{
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < h->n && edge_less(&h->v[m], &h->v[l])) m = l;
        if (r < h->n && edge_less(&h->v[m], &h->v[r])) m = r;
        if (m == i) break;
        or_edge t = h->v[m];
        h->v[m] = h->v[i];
        h->v[i] = t;
        i = m;
    }
}

static void heap_offer(pheap *h, or_edge e)
{
    if (h->n < h->cap) {
        h->v[h->n++] = e;
        heap_sift_up(h, h->n - 1);
    } else if (edge_less(&e, &h->v[0])) {
        h->v[0] = e;
        heap_sift_down(h, 0);
    }
}

typedef struct {
    const float *X;
    int64_t N;
    int32_t d;
    const int64_t *comp;  /* cluster of every row, fixed during a pass */
    or_edge last;         /* pairs with key <= last were handled by earlier passes */
    int have_last;
    pheap *heaps;         /* one per thread */
} batch_ctx;

static void batch_worker(void *p, int tid, int nt)
{
    batch_ctx *c = (batch_ctx *)p;
    pheap *h = &c->heaps[tid];
    h->n = 0;
    for (int64_t i = tid; i < c->N; i += nt) {
        const float *xi = c->X + i * c->d;
        for (int64_t j = i + 1; j < c->N; ++j) {
            if (c->comp[i] == c->comp[j]) continue; /* would be skipped anyway */
            or_edge e = make_edge(i, j, or_dist(xi, c->X + j * c->d, c->d));
            if (c->have_last && !edge_less(&c->last, &e)) continue;
            heap_offer(h, e);
        }
    }
}

int64_t or_nnm_batched(const float *X, int64_t N, int32_t d, int64_t P, int32_t threads,
                       or_edge *edges_out)
{
    if (N < 1 || d < 1 || P < 1) return -1;
    int nt = resolve_threads(threads);
    uf_t uf;
    uf_init(&uf, N);
    int64_t *comp = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    pheap *heaps = (pheap *)calloc((size_t)nt, sizeof(pheap));
    for (int t = 0; t < nt; ++t) {
        heaps[t].cap = P;
        heaps[t].v = (or_edge *)malloc((size_t)P * sizeof(or_edge));
    }
    or_edge *batch = (or_edge *)malloc((size_t)P * (size_t)nt * sizeof(or_edge));
    batch_ctx c = {X, N, d, comp, {0, 0, 0.0}, 0, heaps};
    int64_t m = 0, clusters = N;
    while (clusters > 1) {
        for (int64_t i = 0; i < N; ++i) comp[i] = uf_find(&uf, i);
        run_threads(nt, batch_worker, &c);
        /* the first-level merge: the P smallest of all threads' P smallest */
        int64_t nb = 0;
        for (int t = 0; t < nt; ++t) {
            memcpy(batch + nb, heaps[t].v, (size_t)heaps[t].n * sizeof(or_edge));
            nb += heaps[t].n;
        }
        if (nb == 0) break;
        or_sort_edges(batch, nb);
        if (nb > P) nb = P;
        for (int64_t q = 0; q < nb; ++q) {
            int64_t ra = uf_find(&uf, batch[q].a), rb = uf_find(&uf, batch[q].b);
            if (ra == rb) continue; /* pair already inside one cluster */
            uf_union(&uf, ra, rb);
            edges_out[m++] = batch[q];
            --clusters;
        }
        c.last = batch[nb - 1];
        c.have_last = 1;
    }
    for (int t = 0; t < nt; ++t) free(heaps[t].v);
    free(heaps);
    free(batch);
    free(comp);
    uf_free(&uf);
    return m;
}

/* ------------------------------------------------------------------------- */
/* Prim's algorithm (dense): an independent route to the same unique tree.     */
/* ------------------------------------------------------------------------- */

typedef struct {
    const float *X;
    int64_t N;
    int32_t d;
    unsigned char *in_tree;
    double *best_D;     /* best known edge from each outside vertex into the tree */
    int64_t *best_p;    /* its tree endpoint (-1: none) */
    int64_t *thr_arg;   /* per-thread argmin of the outside vertices' best edge */
    int64_t u;          /* vertex added last */
    int done;
    spin_barrier bar;
} prim_ctx;

static or_edge prim_edge(const prim_ctx *c, int64_t v)
{
    return make_edge(c->best_p[v], v, c->best_D[v]);
}

static int prim_better(const prim_ctx *c, int64_t v, int64_t w)
{
    /* is v's best edge smaller than w's? (no edge counts as +infinity) */
    if (w < 0 || c->best_p[w] < 0) return c->best_p[v] >= 0;
    if (c->best_p[v] < 0) return 0;
    or_edge ev = prim_edge(c, v), ew = prim_edge(c, w);
    return edge_less(&ev, &ew);
}

/* One thread's share of a Prim step: relax the outside vertices against the
 * vertex added last and find the smallest outside edge among them. */
static void prim_scan(prim_ctx *c, int tid, int nt)
{
    int64_t u = c->u, arg = -1;
    const float *xu = c->X + u * c->d;
    int64_t lo = c->N * tid / nt, hi = c->N * (tid + 1) / nt; /* contiguous: no false sharing */
    for (int64_t v = lo; v < hi; ++v) {
        if (c->in_tree[v]) continue;
        or_edge e = make_edge(u, v, or_dist(xu, c->X + v * c->d, c->d));
        int improve = c->best_p[v] < 0;
        if (!improve) {
            or_edge cur = prim_edge(c, v);
            improve = edge_less(&e, &cur);
        }
        if (improve) {
            c->best_D[v] = e.D;
            c->best_p[v] = u;
        }
        if (prim_better(c, v, arg)) arg = v;
    }
    c->thr_arg[tid] = arg;
}

static void prim_worker(void *p, int tid, int nt)
{
    prim_ctx *c = (prim_ctx *)p;
    for (;;) {
        spin_barrier_wait(&c->bar);
        if (c->done) break;
        prim_scan(c, tid, nt);
        spin_barrier_wait(&c->bar);
    }
}

int64_t or_prim(const float *X, int64_t N, int32_t d, int32_t threads, or_edge *edges_out)
{
    if (N < 1 || d < 1) return -1;
    int nt = resolve_threads(threads);
    if ((int64_t)nt > N) nt = (int)N;
    prim_ctx c;
    c.X = X;
    c.N = N;
    c.d = d;
    c.in_tree = (unsigned char *)calloc((size_t)N, 1);
    c.best_D = (double *)malloc((size_t)N * sizeof(double));
    c.best_p = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    c.thr_arg = (int64_t *)malloc((size_t)nt * sizeof(int64_t));
    for (int64_t v = 0; v < N; ++v) c.best_p[v] = -1;
    c.done = 0;
    spin_barrier_init(&c.bar, nt);

    pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
    or_job *jobs = (or_job *)calloc((size_t)nt, sizeof(or_job));
    for (int t = 1; t < nt; ++t) {
        jobs[t].fn = prim_worker;
        jobs[t].ctx = &c;
        jobs[t].tid = t;
        jobs[t].nthreads = nt;
        pthread_create(&th[t], NULL, or_job_main, &jobs[t]);
    }
    int64_t m = 0;
    c.u = 0;
    c.in_tree[0] = 1;
    for (int64_t it = 1; it < N; ++it) {
        /* thread 0 is the caller: it runs its share between the two barriers */
        spin_barrier_wait(&c.bar);
        prim_scan(&c, 0, nt);
        spin_barrier_wait(&c.bar);
        int64_t best = -1;
        for (int t = 0; t < nt; ++t)
            if (c.thr_arg[t] >= 0 && prim_better(&c, c.thr_arg[t], best)) best = c.thr_arg[t];
        if (best < 0) break; /* cannot happen on a complete graph */
        edges_out[m++] = prim_edge(&c, best);
        c.in_tree[best] = 1;
        c.u = best;
    }
    c.done = 1;
    spin_barrier_wait(&c.bar);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    free(c.in_tree);
    free(c.best_D);
    free(c.best_p);
    free(c.thr_arg);
    or_sort_edges(edges_out, m);
    return m;
}

/* ------------------------------------------------------------------------- */
/* Kruskal over all pairs: the textbook definition of single linkage.          */
/* ------------------------------------------------------------------------- */

static or_edge *all_pairs_sorted(const float *X, int64_t N, int32_t d, int64_t *count)
{
    int64_t np = N * (N - 1) / 2;
    or_edge *e = (or_edge *)malloc((size_t)(np > 0 ? np : 1) * sizeof(or_edge));
    int64_t q = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j) e[q++] = make_edge(i, j, or_dist(X + i * d, X + j * d, d));
    or_sort_edges(e, np);
    *count = np;
    return e;
}

int64_t or_kruskal_allpairs(const float *X, int64_t N, int32_t d, or_edge *edges_out)
{
    if (N < 1 || d < 1 || N > 20000) return -1;
    int64_t np;
    or_edge *e = all_pairs_sorted(X, N, d, &np);
    uf_t uf;
    uf_init(&uf, N);
    int64_t m = 0;
    for (int64_t q = 0; q < np && m < N - 1; ++q) {
        int64_t ra = uf_find(&uf, e[q].a), rb = uf_find(&uf, e[q].b);
        if (ra == rb) continue;
        uf_union(&uf, ra, rb);
        edges_out[m++] = e[q];
    }
    uf_free(&uf);
    free(e);
    return m;
}

/* ------------------------------------------------------------------------- */
/* Restrictions ("Problem statement"; "Problem settings": KL1..KL4)            */
/*                                                                           */
/* A walk over candidate pairs in key order with a union-find that tracks       */
/* cluster sizes and the cluster count K (initially N):                        */
/*  - max joining distance c: a pair is admissible iff D <= c*c (rounded);     */
/*  - KL1: before every join, stop if K <= KL1 (KL1 read as the wanted number  */
/*    of clusters);                                                           */
/*  - KL2: no join if either cluster already has more than KL2 elements;       */
/*  - KL3: no join if the two sizes add up to more than KL3;                   */
/*  - KL4: pairs that touch a cluster with fewer than KL4 elements go first:   */
/*    one key-order walk joins only such pairs and defers the others, a second */
/*    key-order walk then handles the deferred pairs.  A pair whose gates       */
/*    block it is dropped for good (sizes only grow).                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    double cap2;
    int64_t kl1, kl2, kl3, kl4;
} gates_t;

static gates_t make_gates(const or_restrictions *r)
{
    gates_t g;
    g.cap2 = INFINITY;
    /* the cap in D units: squared for the squared Euclidean D */
    if (r->max_join_dist > 0.0 && isfinite(r->max_join_dist))
        g.cap2 = g_metric == OR_EUCLIDEAN ? r->max_join_dist * r->max_join_dist : r->max_join_dist;
    g.kl1 = r->kl1_stop_clusters;
    g.kl2 = r->kl2_max_pre_size;
    g.kl3 = r->kl3_max_size;
    g.kl4 = r->kl4_min_size;
    return g;
}

/* Decide one pair. Returns 1 if joined (merge recorded), 0 otherwise;
 * *stop set when KL1 ends the walk, *deferred set when KL4 defers it. */
static int walk_step(uf_t *uf, const gates_t *g, const or_edge *e, int phase, int64_t *K,
                     or_merge *out, int64_t *m, int *stop, int *deferred)
{
    *deferred = 0;
    int64_t ra = uf_find(uf, e->a), rb = uf_find(uf, e->b);
    if (ra == rb) return 0; /* already inside one cluster */
    if (!(e->D <= g->cap2)) return 0;
    if (g->kl4 > 0 && phase == 1 && uf->size[ra] >= g->kl4 && uf->size[rb] >= g->kl4) {
        *deferred = 1;
        return 0;
    }
    if (g->kl2 > 0 && (uf->size[ra] > g->kl2 || uf->size[rb] > g->kl2)) return 0;
    if (g->kl3 > 0 && uf->size[ra] + uf->size[rb] > g->kl3) return 0;
    if (g->kl1 > 0 && *K <= g->kl1) {
        *stop = 1;
        return 0;
    }
    int64_t r = uf_union(uf, ra, rb);
    or_merge mg;
    mg.a = e->a;
    mg.b = e->b;
    mg.D = e->D;
    mg.dist = pair_length(e->D);
    mg.new_size = uf->size[r];
    out[(*m)++] = mg;
    --*K;
    return 1;
}

static int64_t restrict_walk(const or_edge *cand, int64_t nc, int64_t N, const or_restrictions *r,
                             or_merge *out)
{
    gates_t g = make_gates(r);
    uf_t uf;
    uf_init(&uf, N);
    int64_t K = N, m = 0;
    int stop = 0, deferred;
    char *defer = (char *)calloc((size_t)(nc > 0 ? nc : 1), 1);
    int phase = g.kl4 > 0 ? 1 : 2;
    for (int64_t q = 0; q < nc && !stop; ++q) {
        walk_step(&uf, &g, &cand[q], phase, &K, out, &m, &stop, &deferred);
        defer[q] = (char)deferred;
    }
    if (g.kl4 > 0)
        for (int64_t q = 0; q < nc && !stop; ++q)
            if (defer[q]) walk_step(&uf, &g, &cand[q], 2, &K, out, &m, &stop, &deferred);
    free(defer);
    uf_free(&uf);
    return m;
}

int64_t or_restrict_tree(const or_edge *edges, int64_t m, int64_t N, const or_restrictions *r,
                         or_merge *merges_out)
{
    return restrict_walk(edges, m, N, r, merges_out);
}

int64_t or_restrict_literal(const float *X, int64_t N, int32_t d, const or_restrictions *r,
                            or_merge *merges_out)
{
    if (N < 1 || d < 1 || N > 20000) return -1;
    int64_t np;
    or_edge *e = all_pairs_sorted(X, N, d, &np);
    int64_t m = restrict_walk(e, np, N, r, merges_out);
    free(e);
    return m;
}

/* ------------------------------------------------------------------------- */
/* Final labels ("Objectives of the main module": the closing computations)    */
/* ------------------------------------------------------------------------- */

int64_t or_labels(const or_merge *merges, int64_t m, int64_t N, int32_t *labels_out)
{
    uf_t uf;
    uf_init(&uf, N);
    for (int64_t q = 0; q < m; ++q) {
        int64_t ra = uf_find(&uf, merges[q].a), rb = uf_find(&uf, merges[q].b);
        if (ra != rb) uf_union(&uf, ra, rb);
    }
    /* rows visited in increasing order: a cluster's label is fixed by its smallest member */
    int64_t *lab_of_root = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) lab_of_root[i] = -1;
    int64_t K = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t r = uf_find(&uf, i);
        if (lab_of_root[r] < 0) lab_of_root[r] = K++;
        labels_out[i] = (int32_t)lab_of_root[r];
    }
    free(lab_of_root);
    uf_free(&uf);
    return K;
}
