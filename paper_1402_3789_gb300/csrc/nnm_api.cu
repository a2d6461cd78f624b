// nnm_api.cu -- the C ABI (include/nnm.h) and the host-side driver of the device path.
//
// The paper's main module validates the data and runs the managers that keep the GPU
// busy ("Objectives of the main module", "Tasks of the first/second level manager").
// Here one host thread enqueues every step on the caller's stream; all arithmetic runs
// in this library's kernels:
//   nnm_create   K0 checks + operand preparation
//   nnm_nearest  K1/K2 candidate sweep -> K3 exact re-rank (-> collect pass)
//   nnm_cluster  round 0: cached exact k nearest neighbours of every row; merge rounds
//                (K4 component minima, masked rescans, K5 hooking + pointer jumping);
//                K6 edge sort; K7 restriction walk; K8 labels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>
#include <mutex>

#include "nnm_internal.cuh"

using namespace nnm;

#include <atomic>

namespace nnm {
static std::atomic<int64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace nnm

struct nnm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    const float *X = nullptr;
    int64_t N = 0;
    int d = 0;
    nnm_precision prec = NNM_PREC_FP32;
    nnm_options opt{};
    uint64_t wait_ns = 2000000000ull;   // device-side wait limit of the tensor-core sweep
    int64_t Npad = 0;
    int dp = 0;
    int kpad = 0;
    int fp16 = 0;
    int terms = 1;   // 3: split BF16 operands
    double scale = 1.0;
    Margin margin{};
    SelConst selc{};
    // spatial order of the operands (see prep.cu) and the column tiles' bounding spheres
    uint32_t *pos2row = nullptr, *row2pos = nullptr, *list_pos = nullptr, *group = nullptr;
    // batched contexts: independent instances of contiguous rows (n_inst == 1: none)
    int64_t n_inst = 1;
    int64_t min_inst_rows = 0;
    int64_t max_inst_rows = 0;
    int64_t *inst_off = nullptr;   // device [n_inst + 1]; positions = rows of each instance
    uint32_t *inst_pos = nullptr;  // device [N]: instance of each position (and row)
    int64_t *ebeg = nullptr, *eend = nullptr;   // edge range of each instance in the tree
    unsigned long long *inst_nm = nullptr;      // merges per instance (restriction walks)
    uint32_t *inst_edges = nullptr;             // tree edges per instance (merge rounds)
    nnm_merge *merges_tmp = nullptr;
    float *tile_c = nullptr, *tile_rho = nullptr, *mu_f = nullptr, *blk_c = nullptr, *blk_rho = nullptr;
    // landmark bounds: per row the FP32 squared distance to its nearest landmark (x units),
    // per position an upper bound of that distance and per tile / block a lower bound of
    // its columns' distances to any landmark (y units)
    float *land_d2 = nullptr, *lup = nullptr, *tile_lmin = nullptr, *blk_lmin = nullptr;
    int tile_w = 0;
    float lb_R2 = 0.f, lb_eps = 0.f, lb_gamma = 0.f;
    // operands
    float *Xs = nullptr;
    uint16_t *XA = nullptr, *XB = nullptr;
    float *r = nullptr, *P = nullptr, *E = nullptr;
    // sweep / re-rank scratch
    float *cand_v = nullptr;
    uint32_t *cand_j = nullptr;
    uint8_t *cand_ovf = nullptr;
    size_t cand_cap = 0;         // records (one per row slot and column range)
    uint32_t *ovf_row = nullptr, *ovf_blk = nullptr;
    float *ovf_thr = nullptr, *ovf_thr_slot = nullptr;
    uint8_t *ovf_flag = nullptr;
    unsigned int *slot_thr = nullptr;
    size_t ovf_cap = 0;          // slots
    uint32_t *coll_cnt = nullptr, *coll_j = nullptr;
    double *coll_D = nullptr;
    size_t coll_cap = 0;         // entries
    uint8_t *heavy_flag = nullptr;
    uint32_t *heavy_blk = nullptr, *heavy_rows = nullptr, *heavy_rows2 = nullptr;
    float *heavy_thr = nullptr, *heavy_thr2 = nullptr;
    size_t heavy_cap = 0;        // rows
    // cache and rounds
    int metric = 0;   // nnm_metric
    int kc = 0;   // cache width (neighbours kept per row by the first sweep)
    int kr = 0;   // neighbours kept by a rescan (<= kc)
    uint32_t *cache_j = nullptr;
    double *cache_D = nullptr;
    uint8_t *cache_n = nullptr, *cache_exh = nullptr;
    double *row_B = nullptr;
    unsigned long long *comp_bound = nullptr;
    uint32_t *comp_pos = nullptr, *tile_comp = nullptr;
    uint32_t *comp = nullptr, *parent = nullptr, *list = nullptr;
    unsigned long long *row_D = nullptr, *row_ab = nullptr, *best_D = nullptr, *best_ab = nullptr;
    uint8_t *row_state = nullptr, *frozen = nullptr, *flag_pos = nullptr;
    uint32_t *block_cnt = nullptr;
    nnm_edge *edges = nullptr, *edges_tmp = nullptr, *tree = nullptr;
    int64_t n_tree = 0;
    // restriction walk / labels
    uint32_t *uf_parent = nullptr, *uf_size = nullptr, *deferred = nullptr, *minm = nullptr, *flag = nullptr,
             *block_sums = nullptr;
    // restriction cut (no size gate): per-instance counts, level state, hash table
    unsigned long long *cut_cnt = nullptr, *cut_hkey = nullptr;
    uint32_t *cut_lab = nullptr, *cut_w = nullptr, *cut_slot = nullptr;
    uint32_t *cut_hpar = nullptr, *cut_hw = nullptr, *cut_hsum = nullptr, *cut_hlab = nullptr;
    int64_t cut_cap = 0, cut_H = 0;
    // KL2 / KL3 without KL4: safe edges in parallel, the walk only over the others
    nnm_merge *fw_cand = nullptr, *fw_walk = nullptr;
    uint8_t *fw_dec = nullptr, *fw_unsafe = nullptr;
    uint32_t *fw_pos = nullptr, *fw_blk = nullptr;
    nnm_edge *fw_edges = nullptr;
    unsigned long long *fw_cnt = nullptr;   // [0] walk joins [1] joined count (walk state) [2] stop flag
    int64_t fw_cap = 0;
    // small device block: counters and statistics
    uint32_t *dcount = nullptr;             // [0] ovf, [1..3] round counters, [4] n_edges
    unsigned long long *dstat = nullptr;    // [0] max_abs [1] max_rel [2] pairs [3] max_cand [4] n_merges [5] K [6] maxbits..
    int *derr = nullptr;                    // [0] sweep time-out, [1] collect retry, [2] non-finite, [3] cut union
    // events
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    nnm_stats stats{};
    int64_t launch_base = 0;
    nnm_status status = NNM_OK;
    std::string err;
};

namespace {

nnm_status fail(nnm_ctx *c, nnm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->status = s;
        c->err = buf;
    }
    return s;
}

#define NNM_CUDA(c, call)                                                                            \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail((c), e_ == cudaErrorMemoryAllocation ? NNM_ENOMEM : NNM_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                          \
    } while (0)

#define NNM_TRY(x)                         \
    do {                                           \
        nnm_status s_ = (x);                       \
        if (s_ != NNM_OK) return s_;               \
    } while (0)

// Device memory of the library comes from a memory pool of its own, allocated and freed
// in stream order on the context's stream: after the first context, creating and
// destroying contexts costs no cudaMalloc / cudaFree (the pool keeps what it has grown
// to), and the process's default pool is left as the user set it.
cudaMemPool_t lib_pool()
{
    static std::mutex m;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> g(m);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&pools[dev], &props) != cudaSuccess) {
            cudaGetLastError();
            pools[dev] = nullptr;
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return pools[dev];
}

// count elements of T in stream order on s (the library's pool; the default pool if it
// could not be created)
template <typename T>
cudaError_t pool_alloc(T **p, size_t count, cudaStream_t s)
{
    cudaMemPool_t pool = lib_pool();
    const size_t bytes = (count ? count : 1) * sizeof(T);
    return pool ? cudaMallocFromPoolAsync((void **)p, bytes, pool, s) : cudaMallocAsync((void **)p, bytes, s);
}

template <typename T>
nnm_status dalloc(nnm_ctx *c, T **p, size_t count)
{
    if (*p) {
        cudaFreeAsync(*p, c->stream);
        *p = nullptr;
    }
    cudaError_t e = pool_alloc(p, count, c->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, NNM_ENOMEM, "allocation of %zu bytes failed: %s", (count ? count : 1) * sizeof(T),
                    cudaGetErrorString(e));
    }
    return NNM_OK;
}

template <typename T>
void dfree(nnm_ctx *c, T *&p)
{
    if (p) cudaFreeAsync(p, c->stream);
    p = nullptr;
}

// Phase timer: a pair of CUDA events on the context's stream around a scope; the
// elapsed time is added to a stats field.  Phases may nest.
struct Phase {
    nnm_ctx *c;
    double *acc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Phase(nnm_ctx *c_, double *acc_) : c(c_), acc(acc_)
    {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, c->stream);
    }
    ~Phase()
    {
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *acc += ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// nnm_options.wait_limit_ns -> nanoseconds (0: 2 s; at most 60 s)
uint64_t wait_limit(int64_t ns)
{
    if (ns <= 0) return 2000000000ull;
    return ns > 60000000000ll ? 60000000000ull : (uint64_t)ns;
}

bool is_tensor(const nnm_ctx *c) { return c->prec != NNM_PREC_FP32; }

// Column ranges per row tile: enough CTAs to fill the 152 SMs a few times.  In a batched
// context a row tile sweeps its own instances' columns (one instance, or several when a
// short row list mixes instances); the kernels split that range, so the same rule applies
// (splits beyond a row tile's range are empty and cheap).
int choose_splits(const nnm_ctx *c, int64_t nslots)
{
    if (c->opt.col_split > 0) return c->opt.col_split < kMaxSplits ? c->opt.col_split : kMaxSplits;
    const int64_t row_ctas = (nslots + kRowTile - 1) / kRowTile;
    const int64_t target = is_tensor(c) ? 152 * 4 : 152 * 2 * 4;
    int64_t s = (target + row_ctas - 1) / row_ctas;
    // at least 32 tiles of 64 columns per range (FP32), one block of 32 tiles of 128 (tensor)
    const int64_t max_by_cols = is_tensor(c) ? (c->N + 4095) / 4096 : (c->N + 2047) / 2048;
    if (s > max_by_cols) s = max_by_cols;
    if (s > kMaxSplits) s = kMaxSplits;
    if (s < 1) s = 1;
    return (int)s;
}

nnm_status ensure_cand(nnm_ctx *c, size_t records)
{
    if (records <= c->cand_cap) return NNM_OK;
    NNM_TRY(dalloc(c, &c->cand_v, records * kListC));
    NNM_TRY(dalloc(c, &c->cand_j, records * kListC));
    NNM_TRY(dalloc(c, &c->cand_ovf, records));
    c->cand_cap = records;
    return NNM_OK;
}

uint32_t float_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

float bits_float(uint32_t u)
{
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// float >= x (round up)
float up_f(double x)
{
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}

// Host side of the sweeps' pruning constants (FP32, rounded up, enlarged by 2^-20).
SelConst make_selconst(const Margin &m)
{
    SelConst sc{};
    const double grow = 1.0 + 0x1p-20;
    sc.tensor = m.tensor;
    sc.c1 = up_f((1.0 + m.gamma) / (1.0 - m.gamma) * grow * grow);
    sc.c0 = up_f(m.alpha * grow + 1e-37);
    sc.gamma = up_f(m.gamma * grow);
    sc.R = up_f(m.R * grow);
    sc.Pmax = up_f(m.Pmax * grow);
    sc.Emax = up_f(m.Emax * grow);
    sc.c1_32 = up_f((1.0 + m.gamma32) / (1.0 - m.gamma32) * grow * grow);
    sc.c0_32 = up_f(m.alpha32 * grow + 1e-37);
    return sc;
}

nnm_status ensure_ovf(nnm_ctx *c, size_t slots)
{
    if (slots <= c->ovf_cap) return NNM_OK;
    NNM_TRY(dalloc(c, &c->ovf_row, slots));
    NNM_TRY(dalloc(c, &c->ovf_thr, slots));
    NNM_TRY(dalloc(c, &c->ovf_thr_slot, slots));
    NNM_TRY(dalloc(c, &c->ovf_flag, slots));
    NNM_TRY(dalloc(c, &c->ovf_blk, (size_t)compact_blocks((int64_t)slots)));
    NNM_TRY(dalloc(c, &c->coll_cnt, slots));
    NNM_TRY(dalloc(c, &c->slot_thr, slots));
    c->ovf_cap = slots;
    return NNM_OK;
}

nnm_status ensure_cut(nnm_ctx *c, int64_t m)
{
    if (!c->cut_cnt) NNM_TRY(dalloc(c, &c->cut_cnt, (size_t)c->n_inst + 1));
    if (m <= c->cut_cap) return NNM_OK;
    const int64_t H = cut_hash_slots(m);
    NNM_TRY(dalloc(c, &c->cut_lab, (size_t)(2 * m)));
    NNM_TRY(dalloc(c, &c->cut_w, (size_t)(2 * m)));
    NNM_TRY(dalloc(c, &c->cut_slot, (size_t)(2 * m)));
    NNM_TRY(dalloc(c, &c->cut_hkey, (size_t)H));
    NNM_TRY(dalloc(c, &c->cut_hpar, (size_t)H));
    NNM_TRY(dalloc(c, &c->cut_hw, (size_t)H));
    NNM_TRY(dalloc(c, &c->cut_hsum, (size_t)H));
    NNM_TRY(dalloc(c, &c->cut_hlab, (size_t)H));
    c->cut_cap = m;
    c->cut_H = H;
    return NNM_OK;
}

nnm_status ensure_fast(nnm_ctx *c)
{
    if (c->fw_cap >= c->N) return NNM_OK;
    const size_t n = (size_t)c->N;
    NNM_TRY(dalloc(c, &c->fw_cand, n));
    NNM_TRY(dalloc(c, &c->fw_walk, n));
    NNM_TRY(dalloc(c, &c->fw_dec, n));
    NNM_TRY(dalloc(c, &c->fw_unsafe, n));
    NNM_TRY(dalloc(c, &c->fw_pos, n));
    NNM_TRY(dalloc(c, &c->fw_blk, (size_t)compact_blocks(c->N)));
    NNM_TRY(dalloc(c, &c->fw_edges, n));
    NNM_TRY(dalloc(c, &c->fw_cnt, 4));
    c->fw_cap = c->N;
    return NNM_OK;
}

nnm_status ensure_heavy(nnm_ctx *c, size_t rows)
{
    if (rows <= c->heavy_cap) return NNM_OK;
    NNM_TRY(dalloc(c, &c->heavy_flag, rows));
    NNM_TRY(dalloc(c, &c->heavy_blk, (size_t)compact_blocks((int64_t)rows)));
    NNM_TRY(dalloc(c, &c->heavy_rows, rows));
    NNM_TRY(dalloc(c, &c->heavy_rows2, rows));
    NNM_TRY(dalloc(c, &c->heavy_thr, rows));
    NNM_TRY(dalloc(c, &c->heavy_thr2, rows));
    c->heavy_cap = rows;
    return NNM_OK;
}

nnm_status ensure_coll(nnm_ctx *c, size_t entries)
{
    if (entries <= c->coll_cap) return NNM_OK;
    NNM_TRY(dalloc(c, &c->coll_j, entries));
    NNM_TRY(dalloc(c, &c->coll_D, entries));
    c->coll_cap = entries;
    return NNM_OK;
}

SweepArgs base_sweep(nnm_ctx *c)
{
    SweepArgs a{};
    a.Xs = c->Xs;
    a.dp = c->dp;
    a.XA = c->XA;
    a.XB = c->XB;
    a.kpad = c->kpad;
    a.fp16 = c->fp16;
    a.band = c->prec == NNM_PREC_BF16_RERANK ? 64 : 32;
    a.N = c->N;
    a.col_begin = 0;
    a.col_end = c->N;
    a.pos2row = c->pos2row;
    a.err_flag = &c->derr[0];
    a.wait_ns = c->wait_ns;
    a.prune = c->opt.no_tile_pruning ? 0 : 1;
    a.tile_w = c->tile_w;
    a.tile_c = c->tile_c;
    a.tile_rho = c->tile_rho;
    a.lup = c->lup;
    a.tile_lmin = c->tile_lmin;
    a.blk_lmin = c->blk_lmin;
    a.group = c->group;
    a.metric = c->metric;
    a.inst_pos = c->inst_pos;
    a.inst_off = c->inst_off;
    a.blk_c = c->blk_c;
    a.blk_rho = c->blk_rho;
    a.mu_f = c->mu_f;
    a.scale_f = (float)c->scale;
    a.lb_R2 = c->lb_R2;
    a.lb_eps = c->lb_eps;
    a.lb_gamma = c->lb_gamma;
    a.X = c->X;
    a.d = c->d;
    a.st_tiles = &c->dstat[13];
    a.m = c->margin;
    a.sc = c->selc;
    a.kc = 1;
    return a;
}

nnm_status launch_sweep(nnm_ctx *c, const SweepArgs &a, bool collect)
{
    cudaError_t e = is_tensor(c) ? launch_sweep_tc(a, collect, c->stream)
                                 : launch_sweep_fp32(a, c->d, collect, c->stream);
    if (e != cudaSuccess) return fail(c, NNM_ECUDA, "candidate sweep launch: %s", cudaGetErrorString(e));
    c->stats.sweep_launches += 1;
    c->stats.pairs_evaluated += a.nslots * c->N;
    return NNM_OK;
}

nnm_status check_sweep_error(nnm_ctx *c)
{
    int h = 0;
    NNM_CUDA(c, cudaMemcpyAsync(&h, &c->derr[0], sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    NNM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h) {
        NNM_CUDA(c, cudaMemsetAsync(&c->derr[0], 0, sizeof(int), c->stream));
        return fail(c, NNM_ETIMEOUT, "a bounded wait in the tensor-core sweep gave up");
    }
    return NNM_OK;
}

constexpr size_t kCollectBytes = (size_t)4 << 30;   // collect buffers (uint32 + binary64 per entry)

// Collect pass over n rows (positions rows[], thresholds thr[]) with room for cap
// columns per row; rows that collected more are gathered and run again with room for
// their exact count.
nnm_status collect(nnm_ctx *c, const uint32_t *rows, const float *thr, int64_t n, int64_t cap, int k,
                   const uint32_t *comp, uint32_t *res_j, double *res_D, uint8_t *res_n, uint8_t *res_exh,
                   const double *row_B, int res_stride)
{
    cudaStream_t s = c->stream;
    NNM_TRY(ensure_heavy(c, (size_t)n));
    for (int pass = 0; n > 0; ++pass) {
        if (pass > 2) return fail(c, NNM_ECUDA, "collect pass did not converge");
        if (cap > c->N) cap = c->N;
        if (cap < 1) cap = 1;
        int64_t batch = (int64_t)(kCollectBytes / 12 / (size_t)cap);
        if (batch < 1) batch = 1;
        if (batch > n) batch = n;
        NNM_TRY(ensure_coll(c, (size_t)batch * cap));
        NNM_CUDA(c, cudaMemsetAsync(&c->dstat[12], 0, sizeof(unsigned long long), s));
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int64_t nb = n - b0 < batch ? n - b0 : batch;
            SweepArgs ca = base_sweep(c);
            ca.rows = rows + b0;
            ca.nslots = nb;
            ca.comp = comp;
            ca.comp_pos = comp ? c->comp_pos : nullptr;
            ca.tile_comp = comp ? c->tile_comp : nullptr;
            const int S2 = choose_splits(c, nb);
            ca.cols_per_split = round_up((c->N + S2 - 1) / S2, 128);
            ca.splits = (int)((c->N + ca.cols_per_split - 1) / ca.cols_per_split);
            ca.thr = thr + b0;
            ca.coll_cnt = c->coll_cnt;
            ca.coll_j = c->coll_j;
            ca.coll_cap = cap;
            {
                Phase ph(c, &c->stats.ms_sweep);
                NNM_CUDA(c, cudaMemsetAsync(c->coll_cnt, 0, nb * sizeof(uint32_t), s));
                NNM_TRY(launch_sweep(c, ca, true));
            }
            if (is_tensor(c)) NNM_TRY(check_sweep_error(c));
            Phase ph(c, &c->stats.ms_rerank);
            CollectRerankArgs ra{};
            ra.X = c->X;
            ra.d = c->d;
            ra.N = c->N;
            ra.rows = rows + b0;
            ra.pos2row = c->pos2row;
            ra.n = nb;
            ra.coll_cnt = c->coll_cnt;
            ra.coll_j = c->coll_j;
            ra.cap = cap;
            ra.scratch_D = c->coll_D;
            ra.k = k;
            ra.m = c->margin;
            ra.sc = c->selc;
            ra.res_j = res_j;
            ra.res_D = res_D;
            ra.res_n = res_n;
            ra.res_exh = res_exh;
            ra.res_stride = res_stride;
            ra.row_B = row_B;
            ra.retry_flag = &c->derr[1];
            ra.heavy_flag = c->heavy_flag;
            ra.heavy_base = b0;
            ra.heavy_max = &c->dstat[12];
            ra.st_pairs = &c->dstat[2];
            ra.st_max_cand = &c->dstat[3];
            NNM_CUDA(c, launch_collect_rerank(ra, s));
        }
        // heavy rows in collect-slot order (the order of the rows, hence spatial)
        NNM_CUDA(c, launch_compact(c->heavy_flag, n, rows, thr, c->heavy_blk, c->heavy_rows, c->heavy_thr,
                                   &c->dcount[5], s));
        uint32_t nheavy = 0;
        unsigned long long hmax = 0;
        NNM_CUDA(c, cudaMemcpyAsync(&nheavy, &c->dcount[5], sizeof nheavy, cudaMemcpyDeviceToHost, s));
        NNM_CUDA(c, cudaMemcpyAsync(&hmax, &c->dstat[12], sizeof hmax, cudaMemcpyDeviceToHost, s));
        NNM_CUDA(c, cudaStreamSynchronize(s));
        if (nheavy == 0) break;
        // the next pass runs only the heavy rows, with room for the largest exact count
        // swap: the gathered lists become this function's inputs
        std::swap(c->heavy_rows, c->heavy_rows2);
        std::swap(c->heavy_thr, c->heavy_thr2);
        rows = c->heavy_rows2;
        thr = c->heavy_thr2;
        n = nheavy;
        cap = (int64_t)hmax;
    }
    return NNM_OK;
}

// Exact k nearest eligible columns of the given rows (rows == nullptr: all rows).
// Eligible: j != i, and comp[j] != comp[i] if comp is given.  Results go to
// res_j/res_D [row][k] (and res_n / res_exh if given).
nnm_status run_knn(nnm_ctx *c, const uint32_t *rows, int64_t nslots, int k, const uint32_t *comp,
                   uint32_t *res_j, double *res_D, uint8_t *res_n, uint8_t *res_exh, bool full,
                   const double *row_B = nullptr, int res_stride = 0)
{
    if (nslots <= 0) return NNM_OK;
    if (res_stride < k) res_stride = k;
    const int S = choose_splits(c, nslots);
    const int64_t cps = round_up((c->N + S - 1) / S, 128);
    const int splits = (int)((c->N + cps - 1) / cps);
    NNM_TRY(ensure_cand(c, (size_t)nslots * splits));
    NNM_TRY(ensure_ovf(c, (size_t)nslots));

    SweepArgs sa = base_sweep(c);
    sa.rows = rows;
    sa.nslots = nslots;
    sa.comp = comp;
    sa.comp_pos = comp ? c->comp_pos : nullptr;
    sa.tile_comp = comp ? c->tile_comp : nullptr;
    sa.cols_per_split = cps;
    sa.splits = splits;
    sa.out_v = c->cand_v;
    sa.out_j = c->cand_j;
    sa.out_ovf = c->cand_ovf;
    sa.kc = k;
    sa.row_B = row_B;
    sa.slot_thr = c->slot_thr;
    if (splits > 1) NNM_CUDA(c, cudaMemsetAsync(c->slot_thr, 0xFF, (size_t)nslots * sizeof(unsigned int), c->stream));
    {
        Phase ph(c, &c->stats.ms_sweep);
        if (full) NNM_CUDA(c, cudaEventRecord(c->ev0, c->stream));
        NNM_TRY(launch_sweep(c, sa, false));
        if (full) NNM_CUDA(c, cudaEventRecord(c->ev1, c->stream));
    }
    if (full) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        c->stats.sweep_ms_per_launch_full = ms;
        c->stats.full_sweep_pairs = c->N * (c->N - 1);
        // the first sweep of the call: the tile counter holds this launch's tiles
        unsigned long long tiles = 0;
        NNM_CUDA(c, cudaMemcpyAsync(&tiles, &c->dstat[14], sizeof tiles, cudaMemcpyDeviceToHost, c->stream));
        NNM_CUDA(c, cudaStreamSynchronize(c->stream));
        c->stats.full_sweep_pairs_computed = (int64_t)tiles * kRowTile * c->tile_w;
    }
    if (is_tensor(c)) NNM_TRY(check_sweep_error(c));

    uint32_t novf = 0;
    {
        Phase ph(c, &c->stats.ms_rerank);
        FinalizeArgs fa{};
        fa.X = c->X;
        fa.d = c->d;
        fa.N = c->N;
        fa.rows = rows;
        fa.pos2row = c->pos2row;
        fa.nslots = nslots;
        fa.splits = splits;
        fa.in_v = c->cand_v;
        fa.in_j = c->cand_j;
        fa.in_ovf = c->cand_ovf;
        fa.k = k;
        fa.m = c->margin;
        fa.sc = c->selc;
        fa.res_j = res_j;
        fa.res_D = res_D;
        fa.res_n = res_n;
        fa.res_exh = res_exh;
        fa.res_stride = res_stride;
        fa.row_B = row_B;
        fa.ovf_flag = c->ovf_flag;
        fa.ovf_thr = c->ovf_thr_slot;
        fa.st_max_abs = &c->dstat[0];
        fa.st_max_rel = &c->dstat[1];
        fa.st_pairs = &c->dstat[2];
        fa.st_max_cand = &c->dstat[3];
        NNM_CUDA(c, launch_finalize(fa, c->stream));
        // incomplete rows in slot order, so that the collect pass keeps the spatial order
        NNM_CUDA(c, launch_compact(c->ovf_flag, nslots, rows, c->ovf_thr_slot, c->ovf_blk, c->ovf_row, c->ovf_thr,
                                   &c->dcount[0], c->stream));
        NNM_CUDA(c, cudaMemcpyAsync(&novf, &c->dcount[0], sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    }
    if (novf == 0) return NNM_OK;

    // Collect pass: every eligible column with value <= the row's threshold.  The first
    // pass gives each row room for cap columns and counts exactly; rows that had more are
    // run again with room for all of them.  Batches keep the buffers within kCollectBytes.
    c->stats.rows_overflowed += novf;
    NNM_TRY(collect(c, c->ovf_row, c->ovf_thr, novf, is_tensor(c) ? 1024 : 256, k, comp, res_j, res_D, res_n,
                    res_exh, row_B, res_stride));
    return NNM_OK;
}

void reset_stats(nnm_ctx *c)
{
    const double prep = c->stats.ms_prep;
    const int32_t kp = c->stats.k_pad;
    const double sc = c->stats.scale;
    memset(&c->stats, 0, sizeof c->stats);
    c->stats.ms_prep = prep;
    c->stats.k_pad = kp;
    c->stats.scale = sc;
    c->stats.cache_k = c->kc;
    c->launch_base = launches_so_far();
    cudaMemsetAsync(c->dstat, 0, 4 * sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(&c->dstat[13], 0, 2 * sizeof(unsigned long long), c->stream);
}

nnm_status read_stats(nnm_ctx *c)
{
    unsigned long long h[4], ht[2];
    NNM_CUDA(c, cudaMemcpyAsync(h, c->dstat, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    NNM_CUDA(c, cudaMemcpyAsync(ht, &c->dstat[13], sizeof ht, cudaMemcpyDeviceToHost, c->stream));
    NNM_CUDA(c, cudaStreamSynchronize(c->stream));
    double a, r;
    memcpy(&a, &h[0], 8);
    memcpy(&r, &h[1], 8);
    c->stats.max_abs_err = a;
    c->stats.max_rel_err = r;
    c->stats.rerank_pairs = (int64_t)h[2];
    c->stats.max_candidates = (int64_t)h[3];
    c->stats.kernel_launches = launches_so_far() - c->launch_base;
    c->stats.tiles_skipped = (int64_t)ht[0];
    c->stats.tiles_swept = (int64_t)ht[1];
    return NNM_OK;
}

nnm_status prepare(nnm_ctx *c)
{
    cudaStream_t s = c->stream;
    c->Npad = round_up(c->N, 256);
    NNM_TRY(dalloc(c, &c->dcount, 8));
    NNM_TRY(dalloc(c, &c->dstat, 16));
    NNM_TRY(dalloc(c, &c->derr, 4));
    NNM_CUDA(c, cudaMemsetAsync(c->dcount, 0, 8 * sizeof(uint32_t), s));
    NNM_CUDA(c, cudaMemsetAsync(c->dstat, 0, 16 * sizeof(unsigned long long), s));
    NNM_CUDA(c, cudaMemsetAsync(c->derr, 0, 4 * sizeof(int), s));

    // the main module's data check ("Objectives of the main module")
    NNM_CUDA(c, launch_check_finite(c->X, c->N * c->d, &c->derr[2], s));
    int bad = 0;
    NNM_CUDA(c, cudaMemcpyAsync(&bad, &c->derr[2], sizeof(int), cudaMemcpyDeviceToHost, s));
    NNM_CUDA(c, cudaStreamSynchronize(s));
    if (bad) return fail(c, NNM_ENONFINITE, "X holds NaN or infinite values");

    // spatial order: landmark groups along a chain of coarse landmarks, isolated rows last
    {
        NNM_TRY(dalloc(c, &c->pos2row, (size_t)c->N));
        NNM_TRY(dalloc(c, &c->row2pos, (size_t)c->N));
        NNM_TRY(dalloc(c, &c->list_pos, (size_t)c->N));
        NNM_TRY(dalloc(c, &c->group, (size_t)c->N));
        int64_t L = c->N / 512;
        if (L > kMaxGroups) L = kMaxGroups;
        if (L < 1) L = 1;
        const int64_t S = L < 1024 ? L : 1024;
        nnm_edge *keys = nullptr, *tmp = nullptr, *sorted = nullptr, *lkeys = nullptr, *ltmp = nullptr,
                 *lsorted = nullptr;
        uint32_t *crank = nullptr, *larg = nullptr, *lpos = nullptr, *lrank = nullptr, *rarg = nullptr;
        float *ldist = nullptr, *rdist = nullptr, *tau = nullptr;
        unsigned int *hist = nullptr;
        auto free_all = [&]() {
            if (keys) cudaFreeAsync(keys, s);
            if (tmp) cudaFreeAsync(tmp, s);
            if (lkeys) cudaFreeAsync(lkeys, s);
            if (ltmp) cudaFreeAsync(ltmp, s);
            if (crank) cudaFreeAsync(crank, s);
            if (larg) cudaFreeAsync(larg, s);
            if (lpos) cudaFreeAsync(lpos, s);
            if (lrank) cudaFreeAsync(lrank, s);
            if (rarg) cudaFreeAsync(rarg, s);
            if (ldist) cudaFreeAsync(ldist, s);
            if (tau) cudaFreeAsync(tau, s);
            if (hist) cudaFreeAsync(hist, s);
        };
        nnm_status st = NNM_OK;
        do {
            if ((st = dalloc(c, &keys, (size_t)c->N)) != NNM_OK) break;
            if ((st = dalloc(c, &tmp, (size_t)c->N)) != NNM_OK) break;
            if ((st = dalloc(c, &lkeys, (size_t)L)) != NNM_OK) break;
            if ((st = dalloc(c, &ltmp, (size_t)L)) != NNM_OK) break;
            if ((st = dalloc(c, &crank, (size_t)S)) != NNM_OK) break;
            if ((st = dalloc(c, &larg, (size_t)L)) != NNM_OK) break;
            if ((st = dalloc(c, &lpos, (size_t)L)) != NNM_OK) break;
            if ((st = dalloc(c, &lrank, (size_t)L)) != NNM_OK) break;
            if ((st = dalloc(c, &ldist, (size_t)L)) != NNM_OK) break;
            if ((st = dalloc(c, &rarg, (size_t)c->N)) != NNM_OK) break;
            if ((st = dalloc(c, &c->land_d2, (size_t)c->N)) != NNM_OK) break;
            rdist = c->land_d2;   // kept for the landmark bounds of the tiles
            if ((st = dalloc(c, &tau, 1)) != NNM_OK) break;
            if ((st = dalloc(c, &hist, 4096)) != NNM_OK) break;
        } while (0);
        if (st != NNM_OK) {
            free_all();
            return st;
        }
        cudaError_t e = launch_landmark_chain(c->X, c->N, c->d, S, crank, s);
        if (e == cudaSuccess) e = launch_nearest_ref(c->X, c->N, c->d, L, S, larg, ldist, s);
        if (e == cudaSuccess)
            e = launch_spatial_keys(larg, ldist, L, crank, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr,
                                    lkeys, nullptr, 0, s);
        if (e == cudaSuccess) e = launch_sort_edges(lkeys, ltmp, L, s, &lsorted);
        if (e == cudaSuccess) e = launch_order_from_keys(lsorted, L, lpos, lrank, nullptr, s);
        if (e == cudaSuccess) e = launch_nearest_ref(c->X, c->N, c->d, c->N, L, rarg, rdist, s);
        if (e == cudaSuccess)
            e = launch_spatial_keys(nullptr, nullptr, 0, nullptr, rarg, rdist, c->N, lrank, c->inst_pos, hist, tau,
                                    nullptr, keys, 1, s);
        if (e == cudaSuccess) e = launch_sort_edges(keys, tmp, c->N, s, &sorted);
        if (e == cudaSuccess) e = launch_order_from_keys(sorted, c->N, c->pos2row, c->row2pos, c->group, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        free_all();
        if (e != cudaSuccess) return fail(c, NNM_ECUDA, "spatial order: %s", cudaGetErrorString(e));
    }
    if (!is_tensor(c)) {
        c->dp = (c->d + 3) & ~3;
        NNM_TRY(dalloc(c, &c->Xs, (size_t)c->Npad * c->dp));
        NNM_CUDA(c, launch_pad_fp32(c->X, c->N, c->d, c->dp, c->Npad, c->pos2row, c->Xs, s));
        c->tile_w = 64;
        c->scale = 1.0;
        const double u = 0x1p-24;
        c->margin.tensor = 0;
        c->margin.gamma = (c->d + 2) * u / (1.0 - (c->d + 2) * u);
        c->margin.alpha = (c->d + 2) * 0x1p-149;
        c->margin.inv_scale2 = 1.0;
    } else {
        c->fp16 = c->prec == NNM_PREC_FP16_RERANK;
        c->terms = c->prec == NNM_PREC_BF16X3_RERANK ? 3 : 1;
        c->kpad = (int)round_up(c->terms * c->d + 6, 16);
        const int mb = mean_blocks(c->N);
        double *partial = nullptr, *mu = nullptr;
        NNM_TRY(dalloc(c, &partial, (size_t)mb * c->d));
        NNM_TRY(dalloc(c, &mu, (size_t)c->d));
        NNM_CUDA(c, launch_mean(c->X, c->N, c->d, partial, mb, mu, s));
        NNM_CUDA(c, launch_max_sqnorm(c->X, c->N, c->d, mu, &c->dstat[8], s));
        unsigned long long mbits = 0;
        NNM_CUDA(c, cudaMemcpyAsync(&mbits, &c->dstat[8], 8, cudaMemcpyDeviceToHost, s));
        NNM_CUDA(c, cudaStreamSynchronize(s));
        double M;
        memcpy(&M, &mbits, 8);
        // one power-of-two scale so that every |x_hat|^2 stays below 2^14 (FP16 range
        // for the norm pieces and the accumulator well inside FP32)
        c->scale = 1.0;
        if (M > 0.0) c->scale = ldexp(1.0, (int)floor(log2(sqrt(16384.0 / M))));
        NNM_TRY(dalloc(c, &c->XA, (size_t)c->Npad * c->kpad));
        NNM_TRY(dalloc(c, &c->XB, (size_t)c->Npad * c->kpad));
        NNM_TRY(dalloc(c, &c->r, (size_t)c->Npad));
        NNM_TRY(dalloc(c, &c->P, (size_t)c->Npad));
        NNM_TRY(dalloc(c, &c->E, (size_t)c->Npad));
        NNM_CUDA(c, launch_tc_operands(c->X, c->N, c->d, mu, c->scale, c->fp16, c->terms, c->kpad, c->Npad, c->pos2row, c->XA,
                                       c->XB, c->r, c->P, c->E, &c->dstat[9], s));
        unsigned long long mx[3];
        NNM_CUDA(c, cudaMemcpyAsync(mx, &c->dstat[9], sizeof mx, cudaMemcpyDeviceToHost, s));
        double mu_h[32];
        float muf_h[32];
        NNM_CUDA(c, cudaMemcpyAsync(mu_h, mu, c->d * sizeof(double), cudaMemcpyDeviceToHost, s));
        NNM_CUDA(c, cudaStreamSynchronize(s));
        for (int k = 0; k < c->d; ++k) muf_h[k] = (float)mu_h[k];
        NNM_TRY(dalloc(c, &c->mu_f, (size_t)c->d));
        NNM_CUDA(c, cudaMemcpyAsync(c->mu_f, muf_h, c->d * sizeof(float), cudaMemcpyHostToDevice, s));
        NNM_CUDA(c, cudaStreamSynchronize(s));
        cudaFreeAsync(partial, s);
        cudaFreeAsync(mu, s);
        c->tile_w = 128;
        c->margin.tensor = 1;
        // FP32 accumulation of kpad exact products, order and rounding mode unknown:
        // at most kpad additions, each off by < 2^-23 of the partial-sum magnitude
        c->margin.gamma = (c->kpad + 2) * 0x1p-23;
        c->margin.alpha = 0.0;
        memcpy(&c->margin.R, &mx[0], 8);
        memcpy(&c->margin.Pmax, &mx[1], 8);
        memcpy(&c->margin.Emax, &mx[2], 8);
        c->margin.inv_scale2 = 1.0 / (c->scale * c->scale);
        c->margin.r = c->r;
        c->margin.P = c->P;
        c->margin.E = c->E;
        c->stats.k_pad = c->kpad;
        c->stats.scale = c->scale;
    }
    {
        const double u = 0x1p-24;
        c->margin.gamma32 = (c->d + 2) * u / (1.0 - (c->d + 2) * u);
        c->margin.alpha32 = (c->d + 2) * 0x1p-149;
    }
    // bounding spheres of the column tiles and the constants of their lower bound
    {
        const int64_t nt = (c->N + c->tile_w - 1) / c->tile_w;
        NNM_TRY(dalloc(c, &c->tile_c, (size_t)nt * 2 * c->d));
        NNM_TRY(dalloc(c, &c->tile_rho, (size_t)nt * 2));
        // landmark bounds: y = x exactly on the FP32 path; on the tensor path the rounding
        // of y = (x - mu) * scale moves a distance by at most 2^-23 of the largest |y|
        // (<= Pmax + R), far inside the slack
        const float land_slack = is_tensor(c) ? up_f((c->margin.Pmax + c->margin.R) * 0x1p-12 * (1.0 + 0x1p-10)) : 0.0f;
        NNM_TRY(dalloc(c, &c->lup, (size_t)c->N));
        NNM_TRY(dalloc(c, &c->tile_lmin, (size_t)nt));
        NNM_CUDA(c, launch_tile_spheres(c->X, c->N, c->d, c->pos2row, c->group, c->mu_f, (float)c->scale, c->tile_w,
                                        c->tile_c, c->tile_rho, c->land_d2, land_slack, c->lup, c->tile_lmin, s));
        const int64_t nb = (nt + 31) / 32;
        NNM_TRY(dalloc(c, &c->blk_c, (size_t)nb * c->d));
        NNM_TRY(dalloc(c, &c->blk_rho, (size_t)nb));
        NNM_TRY(dalloc(c, &c->blk_lmin, (size_t)nb));
        NNM_CUDA(c, launch_block_spheres(c->tile_c, c->tile_rho, nt, c->d, c->blk_c, c->blk_rho, c->tile_lmin,
                                         c->blk_lmin, s));
        const double grow = 1.0 + 0x1p-20;
        if (is_tensor(c)) {
            c->lb_R2 = up_f(2.0 * c->margin.R * grow);
            c->lb_eps = up_f((c->margin.gamma * 4.0 * c->margin.Pmax * c->margin.Pmax + 2.0 * c->margin.Emax) * grow);
            c->lb_gamma = 0.0f;
        } else {
            c->lb_R2 = 0.0f;
            c->lb_eps = up_f(c->margin.alpha * grow + 1e-37);
            c->lb_gamma = up_f(c->margin.gamma * grow);
        }
    }
    c->selc = make_selconst(c->margin);
    return NNM_OK;
}

nnm_status ensure_rounds(nnm_ctx *c)
{
    if (c->comp) return NNM_OK;
    const int64_t N = c->N;
    NNM_TRY(dalloc(c, &c->cache_j, (size_t)N * c->kc));
    NNM_TRY(dalloc(c, &c->cache_D, (size_t)N * c->kc));
    NNM_TRY(dalloc(c, &c->cache_n, (size_t)N));
    NNM_TRY(dalloc(c, &c->cache_exh, (size_t)N));
    NNM_TRY(dalloc(c, &c->row_B, (size_t)N));
    NNM_TRY(dalloc(c, &c->comp_bound, (size_t)N));
    NNM_TRY(dalloc(c, &c->comp_pos, (size_t)N));
    if (c->n_inst > 1) {
        NNM_TRY(dalloc(c, &c->ebeg, (size_t)c->n_inst));
        NNM_TRY(dalloc(c, &c->eend, (size_t)c->n_inst));
        NNM_TRY(dalloc(c, &c->inst_nm, (size_t)c->n_inst + 1));
        NNM_TRY(dalloc(c, &c->inst_edges, (size_t)c->n_inst));
        NNM_TRY(dalloc(c, &c->merges_tmp, (size_t)N));
    }
    NNM_TRY(dalloc(c, &c->tile_comp, (size_t)((N + c->tile_w - 1) / c->tile_w)));
    NNM_TRY(dalloc(c, &c->parent, (size_t)N));
    NNM_TRY(dalloc(c, &c->list, (size_t)N));
    NNM_TRY(dalloc(c, &c->row_D, (size_t)N));
    NNM_TRY(dalloc(c, &c->row_ab, (size_t)N));
    NNM_TRY(dalloc(c, &c->best_D, (size_t)N));
    NNM_TRY(dalloc(c, &c->best_ab, (size_t)N));
    NNM_TRY(dalloc(c, &c->row_state, (size_t)N));
    NNM_TRY(dalloc(c, &c->frozen, (size_t)N));
    NNM_TRY(dalloc(c, &c->flag_pos, (size_t)N));
    NNM_TRY(dalloc(c, &c->block_cnt, (size_t)((N + 1023) / 1024)));
    NNM_TRY(dalloc(c, &c->edges, (size_t)N));
    NNM_TRY(dalloc(c, &c->edges_tmp, (size_t)N));
    NNM_TRY(dalloc(c, &c->uf_parent, (size_t)N));
    NNM_TRY(dalloc(c, &c->uf_size, (size_t)N));
    NNM_TRY(dalloc(c, &c->deferred, (size_t)N));
    NNM_TRY(dalloc(c, &c->minm, (size_t)N));
    NNM_TRY(dalloc(c, &c->flag, (size_t)N));
    NNM_TRY(dalloc(c, &c->block_sums, (size_t)labels_scratch_blocks(N)));
    NNM_TRY(dalloc(c, &c->comp, (size_t)N));   // last: marks the set as allocated
    return NNM_OK;
}

template <typename T>
nnm_status read_dev(nnm_ctx *c, T *host, const T *dev)
{
    NNM_CUDA(c, cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    NNM_CUDA(c, cudaStreamSynchronize(c->stream));
    return NNM_OK;
}

// The merge tree: exact k-NN cache, then rounds until one component remains (or, with
// freeze_at_cap, until no component has an admissible outgoing pair).
nnm_status build_tree(nnm_ctx *c, double cap2)
{
    NNM_TRY(ensure_rounds(c));
    cudaStream_t s = c->stream;
    NNM_TRY(run_knn(c, nullptr, c->N, c->kc, nullptr, c->cache_j, c->cache_D, c->cache_n, c->cache_exh, true));

    RoundState st{};
    st.N = c->N;
    st.k = c->kc;
    st.comp = c->comp;
    st.parent = c->parent;
    st.cache_j = c->cache_j;
    st.cache_D = c->cache_D;
    st.cache_n = c->cache_n;
    st.cache_exh = c->cache_exh;
    st.row_B = c->row_B;
    st.comp_bound = c->comp_bound;
    // a rescan reaches a little beyond the bound it needs, so that the next rounds'
    // (similar, slightly larger) bounds are often covered by its cache already
    st.overscan = 1.25;
    st.X = c->X;
    st.d = c->d;
    st.inst_pos = c->inst_pos;
    st.inst_off = c->inst_off;
    st.inst_edges = c->n_inst > 1 ? c->inst_edges : nullptr;
    st.metric = c->metric;
    st.row_D = c->row_D;
    st.row_ab = c->row_ab;
    st.row_state = c->row_state;
    st.best_D = c->best_D;
    st.best_ab = c->best_ab;
    st.list = c->list;
    st.list_pos = c->list_pos;
    st.flag_pos = c->flag_pos;
    st.block_cnt = c->block_cnt;
    st.row2pos = c->row2pos;
    st.pos2row = c->pos2row;
    st.counters = &c->dcount[1];
    st.edges = c->edges;
    st.n_edges = &c->dcount[4];
    st.frozen = c->frozen;
    st.cap2 = cap2;
    {
        Phase ph(c, &c->stats.ms_rounds);
        NNM_CUDA(c, launch_round_init(st, s));
        NNM_CUDA(c, cudaMemsetAsync(&c->dcount[1], 0, 4 * sizeof(uint32_t), s));
        if (st.inst_edges) NNM_CUDA(c, cudaMemsetAsync(c->inst_edges, 0, (size_t)c->n_inst * sizeof(uint32_t), s));
    }
    int64_t ncomp = c->N;
    // NNM_TRACE=1 in the environment: one line per merge round on stderr
    const char *trace_env = getenv("NNM_TRACE");
    const bool trace = trace_env && trace_env[0] == '1';
    auto tiles_now = [&](unsigned long long *t) {
        cudaMemcpyAsync(t, &c->dstat[13], 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
    };
    if (trace) {
        unsigned long long t[2];
        tiles_now(t);
        fprintf(stderr, "nnm initial k=%d: sweep %.2f ms, rerank %.2f ms, tiles swept %llu skipped %llu, overflowed %lld\n",
                c->kc, c->stats.ms_sweep, c->stats.ms_rerank, t[1], t[0], (long long)c->stats.rows_overflowed);
    }
    for (int round = 0; ncomp > 1; ++round) {
        const double sweep0 = c->stats.ms_sweep, rerank0 = c->stats.ms_rerank;
        unsigned long long t0[2] = {0, 0}, t1[2] = {0, 0};
        if (trace) tiles_now(t0);
        if (round > 64) return fail(c, NNM_ECUDA, "merge rounds did not converge");
        c->stats.rounds = round + 1;
        uint32_t nres = 0;
        {
            Phase ph(c, &c->stats.ms_rounds);
            NNM_CUDA(c, launch_resolve(st, nullptr, c->N, s));
            NNM_CUDA(c, launch_component_min(st, s));
            NNM_CUDA(c, launch_flag_rescans(st, s));
        }
        NNM_TRY(read_dev(c, &nres, &c->dcount[1]));
        std::vector<double> trace_B;
        std::vector<uint32_t> trace_rows;
        if (trace && nres > 0) {
            // rescan bounds of the flagged rows
            std::vector<uint32_t> lst(nres);
            std::vector<double> rb(c->N);
            cudaMemcpyAsync(lst.data(), c->list, nres * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(rb.data(), c->row_B, c->N * sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            for (uint32_t q = 0; q < nres; ++q) trace_B.push_back(rb[lst[q]]);
            trace_rows = lst;
        }
        if (nres > 0) {
            c->stats.rows_rescanned += nres;
            NNM_CUDA(c, launch_position_comps(st, c->tile_w, c->comp_pos, c->tile_comp, s));
            NNM_TRY(run_knn(c, c->list_pos, nres, c->kr, c->comp, c->cache_j, c->cache_D, c->cache_n, c->cache_exh,
                            false, c->row_B, c->kc));
            Phase ph(c, &c->stats.ms_rounds);
            NNM_CUDA(c, launch_resolve(st, c->list, nres, s));
            NNM_CUDA(c, launch_component_min(st, s));
        }
        if (trace && nres > 0) {
            // how far the rescan bound (without the overscan) was from the minimum the
            // component's rescan found: per component, sqrt(bound / minimum)
            std::vector<uint32_t> comp(c->N);
            std::vector<unsigned long long> best(c->N);
            cudaMemcpyAsync(comp.data(), c->comp, c->N * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(best.data(), c->best_D, c->N * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            std::vector<double> ratio;
            std::vector<uint8_t> seen(c->N, 0);
            for (size_t q = 0; q < trace_rows.size(); ++q) {
                const uint32_t cc = comp[trace_rows[q]];
                if (seen[cc] || best[cc] == kMaxKey) continue;
                seen[cc] = 1;
                double bd;
                memcpy(&bd, &best[cc], 8);
                const double B = trace_B[q] / st.overscan;
                if (B < INFINITY && bd > 0.0) ratio.push_back(sqrt(B / bd));
            }
            if (!ratio.empty()) {
                std::sort(ratio.begin(), ratio.end());
                const size_t m = ratio.size();
                size_t over = 0;
                for (double r : ratio) over += r > 1.1;
                fprintf(stderr, "    bound / found minimum (distance ratio) over %zu components: 10/50/90%%: %.3f %.3f %.3f, "
                                "above 1.1: %zu\n", m, ratio[m / 10], ratio[m / 2], ratio[(9 * m) / 10], over);
            }
        }
        uint32_t nedge = 0;
        {
            Phase ph(c, &c->stats.ms_rounds);
            NNM_CUDA(c, cudaMemsetAsync(&c->dcount[2], 0, sizeof(uint32_t), s));
            NNM_CUDA(c, launch_hook(st, s));
        }
        NNM_TRY(read_dev(c, &nedge, &c->dcount[2]));
        if (nedge == 0) break;
        {
            Phase ph(c, &c->stats.ms_rounds);
            for (int it = 0;; ++it) {
                if (it > 64) return fail(c, NNM_ECUDA, "pointer jumping did not converge");
                uint32_t changed = 0;
                NNM_CUDA(c, cudaMemsetAsync(&c->dcount[3], 0, sizeof(uint32_t), s));
                NNM_CUDA(c, launch_jump(st, s));
                NNM_TRY(read_dev(c, &changed, &c->dcount[3]));
                if (!changed) break;
            }
            NNM_CUDA(c, launch_relabel(st, s));
        }
        ncomp -= nedge;
        // a batched context is done when every instance is one component
        if (c->n_inst > 1 && ncomp == c->n_inst) break;
        if (trace) {
            tiles_now(t1);
            fprintf(stderr, "nnm round %d: rescans %u, sweep %.2f ms, rerank %.2f ms, tiles swept %llu skipped %llu, "
                            "edges %u, components %lld\n",
                    round, nres, c->stats.ms_sweep - sweep0, c->stats.ms_rerank - rerank0, t1[1] - t0[1],
                    t1[0] - t0[0], nedge, (long long)ncomp);
            if (!trace_B.empty()) {
                std::sort(trace_B.begin(), trace_B.end());
                const size_t m = trace_B.size();
                size_t ninf = 0;
                for (double b : trace_B) ninf += !(b < INFINITY);
                fprintf(stderr, "    rescan bounds: unbounded %zu, quantiles 10/50/90%%: %.4g %.4g %.4g\n", ninf,
                        trace_B[m / 10], trace_B[m / 2], trace_B[(9 * m) / 10]);
            }
        }
    }
    uint32_t ne = 0;
    NNM_TRY(read_dev(c, &ne, &c->dcount[4]));
    c->n_tree = ne;
    {
        Phase ph(c, &c->stats.ms_sort);
        // a batched context keeps each instance's edges together (then in key order)
        NNM_CUDA(c, launch_sort_edges(c->edges, c->edges_tmp, c->n_tree, s, &c->tree,
                                      c->n_inst > 1 ? c->inst_pos : nullptr));
        if (c->n_inst > 1)
            NNM_CUDA(c, launch_edge_ranges(c->tree, c->n_tree, c->inst_pos, c->n_inst, c->ebeg, c->eend, s));
    }
    return NNM_OK;
}

// KL2 / KL3 without KL4 on one instance (dendro.cu has the argument): the unrestricted
// endpoint sizes of every admissible edge from the cut's levels, the safe edges joined in
// parallel, the walk over the unsafe ones only, then the joins in key order, cut after
// N - KL1 of them.  Leaves the final partition in uf_parent and the count in dstat[4].
nnm_status restrict_fast(nnm_ctx *c, const nnm_restrictions &r, double cap2, nnm_merge *merges_dev)
{
    cudaStream_t s = c->stream;
    const int64_t N = c->N;
    NNM_TRY(ensure_cut(c, c->n_tree));
    NNM_TRY(ensure_fast(c));
    CutArgs ca{};
    ca.edges = c->tree;
    ca.m = c->n_tree;
    ca.N = N;
    ca.cap2 = cap2;
    ca.kl1 = 0;
    ca.metric = c->metric;
    ca.n_inst = 1;
    ca.merges = c->fw_cand;
    ca.n_merges = &c->dstat[4];
    ca.uf_parent = c->uf_parent;
    ca.err_flag = &c->derr[3];
    ca.cnt = c->cut_cnt;
    ca.lab = c->cut_lab;
    ca.w = c->cut_w;
    ca.slot = c->cut_slot;
    ca.hkey = c->cut_hkey;
    ca.hpar = c->cut_hpar;
    ca.hw = c->cut_hw;
    ca.hsum = c->cut_hsum;
    ca.hlab = c->cut_hlab;
    ca.H = c->cut_H;
    int64_t M = 0;
    NNM_CUDA(c, launch_restrict_cut(ca, &M, s));
    FastWalkArgs f{};
    f.N = N;
    f.M = M;
    f.kl2 = r.kl2_max_pre_size;
    f.kl3 = r.kl3_max_size;
    f.cand = c->fw_cand;
    f.w = c->cut_w;
    f.dec = c->fw_dec;
    f.unsafe = c->fw_unsafe;
    f.pos = c->fw_pos;
    f.unsafe_edges = c->fw_edges;
    f.walk_out = c->fw_walk;
    f.uf_parent = c->uf_parent;
    f.uf_size = c->uf_size;
    f.merges = merges_dev;
    f.err_flag = &c->derr[3];
    NNM_CUDA(c, launch_fast_walk_steps(f, 0, 0, s));
    NNM_CUDA(c, launch_fast_walk_steps(f, 1, 0, s));
    uint32_t n_unsafe = 0;
    NNM_CUDA(c, launch_compact(c->fw_unsafe, M, nullptr, nullptr, c->fw_blk, c->fw_pos, nullptr, &c->dcount[6], s));
    NNM_TRY(read_dev(c, &n_unsafe, &c->dcount[6]));
    if (n_unsafe > 0) {
        NNM_CUDA(c, launch_fast_walk_steps(f, 2, n_unsafe, s));
        NNM_CUDA(c, cudaMemsetAsync(c->fw_cnt, 0, 4 * sizeof(unsigned long long), s));
        RestrictArgs ra{};
        ra.edges = c->fw_edges;
        ra.m = n_unsafe;
        ra.N = N;
        ra.cap2 = cap2;
        ra.kl2 = r.kl2_max_pre_size;
        ra.kl3 = r.kl3_max_size;
        ra.uf_parent = c->uf_parent;
        ra.uf_size = c->uf_size;
        ra.merges = c->fw_walk;
        ra.n_merges = &c->fw_cnt[0];
        ra.err_flag = &c->derr[3];
        ra.n_inst = 1;
        ra.metric = c->metric;
        ra.persist = 1;
        ra.lit_phase = 2;
        ra.joined_io = reinterpret_cast<long long *>(&c->fw_cnt[1]);
        ra.stop_io = reinterpret_cast<int *>(&c->fw_cnt[2]);
        NNM_CUDA(c, launch_restrict(ra, s));
        unsigned long long n_acc = 0;
        NNM_TRY(read_dev(c, &n_acc, &c->fw_cnt[0]));
        NNM_CUDA(c, launch_fast_walk_steps(f, 3, (int64_t)n_acc, s));
    }
    uint32_t n_dec = 0;
    NNM_CUDA(c, launch_compact(c->fw_dec, M, nullptr, nullptr, c->fw_blk, c->fw_pos, nullptr, &c->dcount[6], s));
    NNM_TRY(read_dev(c, &n_dec, &c->dcount[6]));
    int64_t n_out = n_dec;
    if (r.kl1_stop_clusters > 0) {
        const int64_t room = N > r.kl1_stop_clusters ? N - r.kl1_stop_clusters : 0;
        if (n_out > room) n_out = room;
    }
    NNM_CUDA(c, launch_fast_walk_steps(f, 4, n_out, s));
    NNM_CUDA(c, launch_fast_walk_steps(f, 5, n_out, s));
    const unsigned long long nm = (unsigned long long)n_out;
    NNM_CUDA(c, cudaMemcpyAsync(&c->dstat[4], &nm, sizeof nm, cudaMemcpyHostToDevice, s));
    NNM_CUDA(c, cudaStreamSynchronize(s));
    return NNM_OK;
}

constexpr int64_t kLiteralMaxRows = 262144;

// Device buffers of one call, freed (in stream order) when it returns.
struct CallScratch {
    explicit CallScratch(cudaStream_t st) : s(st) {}
    cudaStream_t s;
    std::vector<void *> ptrs;
    template <typename T>
    cudaError_t get(T **p, size_t count)
    {
        *p = nullptr;
        cudaError_t e = pool_alloc(p, count, s);
        if (e != cudaSuccess) {
            *p = nullptr;
            cudaGetLastError();
            return e;
        }
        ptrs.push_back(*p);
        return cudaSuccess;
    }
    void release(void *p)
    {
        for (auto &q : ptrs)
            if (q == p) {
                cudaFreeAsync(q, s);
                q = nullptr;
            }
    }
    ~CallScratch()
    {
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, s);
    }
};

float down_f(double x)
{
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

// The restrictions in the paper's all-pairs reading (semantics = 1): batches of the pairs
// that cross two clusters and pass every gate at the batch start, each complete for a
// key range above the last one, walked in key order (literal.cu has the argument).  Two
// phases with KL4.  The tree is not needed; the labels come from the walk's union-find.
nnm_status cluster_literal(nnm_ctx *c, const nnm_restrictions &r, double cap2, nnm_merge *merges_dev,
                           int64_t *n_merges_host, int32_t *labels_dev, int64_t *n_clusters_host)
{
    if (c->n_inst > 1) return fail(c, NNM_EUNSUPPORTED, "the all-pairs reading (semantics 1) takes one instance");
    if (c->N > kLiteralMaxRows)
        return fail(c, NNM_EUNSUPPORTED, "the all-pairs reading (semantics 1) takes N <= %lld", (long long)kLiteralMaxRows);
    const int64_t N = c->N;
    cudaStream_t s = c->stream;
    CallScratch sc(c->stream);
    LitArgs a{};
    a.X = c->X;
    a.d = c->d;
    a.N = N;
    a.metric = c->metric;
    a.cap2 = cap2;
    a.cap2f = cap2 < INFINITY ? up_f(cap2) : INFINITY;
    a.kl2 = r.kl2_max_pre_size;
    a.kl3 = r.kl3_max_size;
    a.kl4 = r.kl4_min_size;
    a.c0 = c->selc.c0_32;
    a.c1 = c->selc.c1_32;
    a.c1inv = down_f(1.0 / (double)a.c1);
    const int fine_bins = literal_fine_bins();
    unsigned long long *cnt = nullptr;   // [0] emitted [1] kept [2] merges [3] K
    long long *joined = nullptr;
    int *stop = nullptr;
    uint32_t *minm = nullptr, *lflag = nullptr, *bsums = nullptr;
    cudaError_t e = sc.get(&a.uf_parent, N);
    if (e == cudaSuccess) e = sc.get(&a.uf_size, N);
    if (e == cudaSuccess) e = sc.get(&a.comp, N);
    if (e == cudaSuccess) e = sc.get(&a.csize, N);
    if (e == cudaSuccess) e = sc.get(&a.tD, N);
    if (e == cudaSuccess) e = sc.get(&a.tab, N);
    if (e == cudaSuccess) e = sc.get(&a.w0, N);
    if (e == cudaSuccess) e = sc.get(&a.w1, N);
    if (e == cudaSuccess) e = sc.get(&a.w2, N);
    if (e == cudaSuccess) e = sc.get(&a.w3, N);
    if (e == cudaSuccess) e = sc.get(&a.w4, N);
    if (e == cudaSuccess) e = sc.get(&a.hist, (size_t)fine_bins);
    if (e == cudaSuccess) e = sc.get(&cnt, 4);
    if (e == cudaSuccess) e = sc.get(&joined, 1);
    if (e == cudaSuccess) e = sc.get(&stop, 1);
    if (e == cudaSuccess) e = sc.get(&minm, N);
    if (e == cudaSuccess) e = sc.get(&lflag, N);
    if (e == cudaSuccess) e = sc.get(&bsums, (size_t)labels_scratch_blocks(N));
    if (e != cudaSuccess) return fail(c, NNM_ENOMEM, "all-pairs reading: scratch allocation failed");
    a.n_emit = &cnt[0];
    a.n_kept = &cnt[1];
    NNM_CUDA(c, cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s));
    NNM_CUDA(c, cudaMemsetAsync(joined, 0, sizeof(long long), s));
    NNM_CUDA(c, cudaMemsetAsync(stop, 0, sizeof(int), s));
    NNM_CUDA(c, launch_lit_init(a, a.kl4 > 0 ? INFINITY : -1.0, s));
    // pairs per batch: large enough that the all-pairs passes stay a small share
    int64_t P = 8 * N;
    if (P < (int64_t(1) << 20)) P = int64_t(1) << 20;
    if (P > (int64_t(1) << 24)) P = int64_t(1) << 24;
    int64_t cap = 0;
    nnm_edge *tmp = nullptr;
    std::vector<unsigned long long> h(fine_bins);
    const double c0 = a.c0, c1inv = a.c1inv;
    // tau(E): every pair with D <= tau has an FP32 value <= E
    auto tau_of = [&](float E) -> double {
        if (!(E < INFINITY)) return INFINITY;
        double t = ((double)E - c0) * c1inv - c0;
        t = nextafter(t, -INFINITY);
        return t > 0.0 ? t : 0.0;
    };
    for (int phase = a.kl4 > 0 ? 1 : 2; phase <= 2; ++phase) {
        int hstop = 0;
        NNM_CUDA(c, cudaMemcpyAsync(&hstop, stop, sizeof(int), cudaMemcpyDeviceToHost, s));
        NNM_CUDA(c, cudaStreamSynchronize(s));
        if (hstop) break;
        if (phase == 2 && a.kl4 > 0) {
            unsigned long long n1 = 0;
            NNM_TRY(read_dev(c, &n1, &cnt[2]));
            NNM_CUDA(c, launch_lit_reach(a, merges_dev, (int64_t)n1, s));
        }
        a.phase = phase;
        a.have_last = 0;
        a.last_D = -INFINITY;
        for (int batch = 0;; ++batch) {
            if (batch > (1 << 20)) return fail(c, NNM_ECUDA, "all-pairs reading did not converge");
            NNM_CUDA(c, launch_lit_flatten(a, s));
            NNM_CUDA(c, cudaMemsetAsync(a.hist, 0, 256 * sizeof(unsigned long long), s));
            NNM_CUDA(c, launch_lit_pass(a, 0, s));
            NNM_CUDA(c, cudaMemcpyAsync(h.data(), a.hist, 256 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            NNM_CUDA(c, cudaStreamSynchronize(s));
            unsigned long long total = 0;
            for (int q = 0; q < 256; ++q) total += h[q];
            if (total == 0) break;
            // the smallest cut that moves past the last batch
            float Emin = 0.0f;
            if (a.have_last) {
                Emin = up_f((a.last_D + c0) / c1inv + c0);
                Emin = nextafterf(Emin, INFINITY);
            }
            const unsigned emin_oct = a.have_last ? (unsigned)(float_bits(Emin) >> 23) : 0u;
            unsigned oct = 0, last_nz = 0;
            unsigned long long cum = 0, below = 0;
            bool found = false;
            for (unsigned q = 0; q < 256; ++q) {
                if (h[q]) last_nz = q;
                if (!found && cum + h[q] >= (unsigned long long)P) {
                    oct = q;
                    found = true;
                }
                if (!found) cum += h[q];
            }
            if (!found) oct = last_nz;
            if (oct < emin_oct) oct = emin_oct;
            below = 0;
            for (unsigned q = 0; q < oct && q < 256; ++q) below += h[q];
            float E;
            unsigned long long count;
            if (oct >= 255) {
                E = INFINITY;
                count = total;
            } else {
                NNM_CUDA(c, cudaMemsetAsync(a.hist, 0, (size_t)fine_bins * sizeof(unsigned long long), s));
                a.octave = oct;
                NNM_CUDA(c, launch_lit_pass(a, 1, s));
                NNM_CUDA(c, cudaMemcpyAsync(h.data(), a.hist, (size_t)fine_bins * sizeof(unsigned long long),
                                            cudaMemcpyDeviceToHost, s));
                NNM_CUDA(c, cudaStreamSynchronize(s));
                unsigned b = (unsigned)fine_bins - 1, fnz = 0;
                bool fb = false;
                unsigned long long fc = below;
                for (unsigned q = 0; q < (unsigned)fine_bins; ++q) {
                    if (h[q]) fnz = q;
                    if (!fb && fc + h[q] >= (unsigned long long)P) {
                        b = q;
                        fb = true;
                    }
                    fc += h[q];
                }
                if (!fb) b = fnz;
                if (oct == emin_oct && a.have_last) {
                    const unsigned bmin = (float_bits(Emin) >> 11) & (unsigned)(fine_bins - 1);
                    if (b < bmin) b = bmin;
                }
                E = bits_float((oct << 23) | (b << 11) | 0x7FFu);
                count = below;
                for (unsigned q = 0; q <= b; ++q) count += h[q];
            }
            const double tau = tau_of(E);
            if (a.have_last && !(tau > a.last_D)) return fail(c, NNM_ECUDA, "all-pairs reading: no progress");
            if (count > (unsigned long long)cap) {
                if (a.emit) sc.release(a.emit);
                if (a.kept) sc.release(a.kept);
                if (tmp) sc.release(tmp);
                cap = (int64_t)count;
                if (sc.get(&a.emit, (size_t)cap) != cudaSuccess || sc.get(&a.kept, (size_t)cap) != cudaSuccess ||
                    sc.get(&tmp, (size_t)cap) != cudaSuccess)
                    return fail(c, NNM_ENOMEM, "all-pairs reading: %llu pairs in one batch", count);
            }
            a.emit_cap = cap;
            a.cut = E;
            a.tau_D = tau;
            NNM_CUDA(c, cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s));
            NNM_CUDA(c, launch_lit_pass(a, 2, s));
            unsigned long long ne = 0;
            NNM_TRY(read_dev(c, &ne, &cnt[0]));
            if (ne > (unsigned long long)cap) return fail(c, NNM_ECUDA, "all-pairs reading: emitted more than counted");
            a.n_emitted = (int64_t)ne;
            NNM_CUDA(c, launch_lit_exact(a, s));
            unsigned long long nk = 0;
            NNM_TRY(read_dev(c, &nk, &cnt[1]));
            if (nk > 0) {
                nnm_edge *sorted = nullptr;
                NNM_CUDA(c, launch_sort_edges(a.kept, tmp, (int64_t)nk, s, &sorted));
                RestrictArgs ra{};
                ra.edges = sorted;
                ra.m = (int64_t)nk;
                ra.N = N;
                ra.cap2 = cap2;
                ra.kl1 = r.kl1_stop_clusters;
                ra.kl2 = r.kl2_max_pre_size;
                ra.kl3 = r.kl3_max_size;
                ra.kl4 = r.kl4_min_size;
                ra.uf_parent = a.uf_parent;
                ra.uf_size = a.uf_size;
                ra.merges = merges_dev;
                ra.n_merges = &cnt[2];
                ra.metric = c->metric;
                ra.n_inst = 1;
                ra.persist = 1;
                ra.lit_phase = phase;
                ra.joined_io = joined;
                ra.stop_io = stop;
                NNM_CUDA(c, launch_restrict(ra, s));
                int hs = 0;
                NNM_TRY(read_dev(c, &hs, stop));
                if (hs) break;
            }
            a.have_last = 1;
            a.last_D = tau;
            if (!(tau < INFINITY)) break;
        }
    }
    LabelArgs la{};
    la.N = N;
    la.uf_parent = a.uf_parent;
    la.minm = minm;
    la.flag = lflag;
    la.block_sums = bsums;
    la.labels = labels_dev;
    la.K = &cnt[3];
    NNM_CUDA(c, launch_labels(la, s));
    unsigned long long hk[2];
    NNM_CUDA(c, cudaMemcpyAsync(hk, &cnt[2], sizeof hk, cudaMemcpyDeviceToHost, s));
    NNM_CUDA(c, cudaStreamSynchronize(s));
    *n_merges_host = (int64_t)hk[0];
    *n_clusters_host = (int64_t)hk[1];
    return NNM_OK;
}

}  // namespace

extern "C" {

const char *nnm_status_string(nnm_status s)
{
    switch (s) {
    case NNM_OK: return "NNM_OK";
    case NNM_EINVAL: return "NNM_EINVAL";
    case NNM_ENONFINITE: return "NNM_ENONFINITE";
    case NNM_ENOMEM: return "NNM_ENOMEM";
    case NNM_ECUDA: return "NNM_ECUDA";
    case NNM_ETIMEOUT: return "NNM_ETIMEOUT";
    case NNM_EUNSUPPORTED: return "NNM_EUNSUPPORTED";
    }
    return "unknown";
}

static nnm_status create_impl(const float *X_dev, int64_t N, int32_t d, const int64_t *offsets, int64_t n_inst,
                              nnm_metric metric, nnm_precision precision, void *cuda_stream,
                              const nnm_options *options, nnm_ctx **out)
{
    if (!out) return NNM_EINVAL;
    *out = nullptr;
    if (!X_dev || N < 1 || N >= (int64_t(1) << 31) || d < 1 || d > 32) return NNM_EINVAL;
    if (metric != NNM_EUCLIDEAN && metric != NNM_MANHATTAN && metric != NNM_CHEBYSHEV) return NNM_EUNSUPPORTED;
    // the tensor-core candidates rest on |x|^2 + |y|^2 - 2 x.y: Euclidean only
    if (metric != NNM_EUCLIDEAN && precision != NNM_PREC_FP32) return NNM_EUNSUPPORTED;
    if (precision != NNM_PREC_FP32 && precision != NNM_PREC_BF16_RERANK && precision != NNM_PREC_FP16_RERANK &&
        precision != NNM_PREC_BF16X3_RERANK)
        return NNM_EUNSUPPORTED;
    if (precision == NNM_PREC_BF16X3_RERANK && d > 30) return NNM_EUNSUPPORTED;
    if (options && (options->cache_k < 0 || options->cache_k > 16 || options->col_split < 0 ||
                    options->wait_limit_ns < 0))
        return NNM_EINVAL;
    int64_t min_rows = N, max_rows = N;
    if (offsets) {
        if (n_inst < 1 || n_inst > 65535 || offsets[0] != 0 || offsets[n_inst] != N) return NNM_EINVAL;
        max_rows = 0;
        for (int64_t b = 0; b < n_inst; ++b) {
            if (offsets[b + 1] <= offsets[b]) return NNM_EINVAL;
            if (offsets[b + 1] - offsets[b] < min_rows) min_rows = offsets[b + 1] - offsets[b];
            if (offsets[b + 1] - offsets[b] > max_rows) max_rows = offsets[b + 1] - offsets[b];
        }
    }
    nnm_ctx *c = new nnm_ctx();
    c->X = X_dev;
    c->N = N;
    c->d = d;
    c->prec = precision;
    c->metric = (int)metric;
    c->margin.metric = (int)metric;
    if (options) c->opt = *options;
    c->wait_ns = wait_limit(c->opt.wait_limit_ns);
    c->stream = (cudaStream_t)cuda_stream;
    c->kc = c->opt.cache_k > 0 ? c->opt.cache_k : (precision == NNM_PREC_BF16_RERANK ? 2 : 8);
    if (c->kc > N - 1) c->kc = N > 1 ? (int)(N - 1) : 1;
    c->kr = c->kc;
    c->min_inst_rows = min_rows;
    c->max_inst_rows = max_rows;
    cudaGetDevice(&c->device);
    cudaEventCreate(&c->ev0);
    cudaEventCreate(&c->ev1);
    nnm_status st = NNM_OK;
    if (offsets && n_inst > 1) {
        c->n_inst = n_inst;
        st = dalloc(c, &c->inst_off, (size_t)(n_inst + 1));
        if (st == NNM_OK) st = dalloc(c, &c->inst_pos, (size_t)N);
        if (st == NNM_OK &&
            (cudaMemcpyAsync(c->inst_off, offsets, (size_t)(n_inst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                             c->stream) != cudaSuccess ||
             launch_instance_ids(c->inst_off, n_inst, N, c->inst_pos, c->stream) != cudaSuccess))
            st = fail(c, NNM_ECUDA, "instance ids");
    }
    if (st == NNM_OK) {
        Phase ph(c, &c->stats.ms_prep);
        st = prepare(c);
    }
    if (st != NNM_OK) {
        nnm_destroy(c);
        return st;
    }
    *out = c;
    return NNM_OK;
}

nnm_status nnm_create(const float *X_dev, int64_t N, int32_t d, nnm_metric metric, nnm_precision precision,
                      void *cuda_stream, const nnm_options *options, nnm_ctx **out)
{
    return create_impl(X_dev, N, d, nullptr, 1, metric, precision, cuda_stream, options, out);
}

nnm_status nnm_create_batched(const float *X_dev, const int64_t *offsets_host, int64_t n_instances, int32_t d,
                              nnm_metric metric, nnm_precision precision, void *cuda_stream,
                              const nnm_options *options, nnm_ctx **out)
{
    if (!offsets_host || n_instances < 1) {
        if (out) *out = nullptr;
        return NNM_EINVAL;
    }
    return create_impl(X_dev, offsets_host[n_instances], d, offsets_host, n_instances, metric, precision,
                       cuda_stream, options, out);
}

nnm_status nnm_nearest(nnm_ctx *c, int32_t k, uint32_t *idx_dev, double *D_dev)
{
    if (!c) return NNM_EINVAL;
    c->err.clear();
    c->status = NNM_OK;
    if (!idx_dev || !D_dev) return fail(c, NNM_EINVAL, "null output buffer");
    if (k < 1 || k > kMaxK || (int64_t)k >= c->min_inst_rows)
        return fail(c, NNM_EINVAL, "k=%d outside 1..min(16, rows of the smallest instance - 1)", k);
    reset_stats(c);
    {
        Phase total(c, &c->stats.ms_total);
        NNM_TRY(run_knn(c, nullptr, c->N, k, nullptr, idx_dev, D_dev, nullptr, nullptr, true));
    }
    return read_stats(c);
}

nnm_status nnm_cluster(nnm_ctx *c, const nnm_restrictions *restr, nnm_merge *merges_dev, int64_t *n_merges_host,
                       int32_t *labels_dev, int64_t *n_clusters_host)
{
    if (!c) return NNM_EINVAL;
    c->err.clear();
    c->status = NNM_OK;
    if (!merges_dev || !n_merges_host || !labels_dev || !n_clusters_host)
        return fail(c, NNM_EINVAL, "null output pointer");
    if (c->N < 2) return fail(c, NNM_EINVAL, "nnm_cluster needs N >= 2");
    nnm_restrictions r{};
    if (restr) r = *restr;
    if (r.semantics != 0 && r.semantics != 1) return fail(c, NNM_EINVAL, "semantics must be 0 or 1");
    if (isnan(r.max_join_dist) || r.kl1_stop_clusters < 0 || r.kl2_max_pre_size < 0 || r.kl3_max_size < 0 ||
        r.kl4_min_size < 0)
        return fail(c, NNM_EINVAL, "negative restriction");
    if (r.kl2_max_pre_size > 0 && r.kl3_max_size > 0 && r.kl3_max_size <= r.kl2_max_pre_size)
        return fail(c, NNM_EINVAL, "KL3 must exceed KL2");
    // the cap in D units: squared for the squared Euclidean D, else the length itself
    const double cap2 = (r.max_join_dist > 0.0 && isfinite(r.max_join_dist))
                            ? (c->metric == NNM_EUCLIDEAN ? r.max_join_dist * r.max_join_dist : r.max_join_dist)
                            : INFINITY;
    reset_stats(c);
    if (r.semantics == 1) {
        {
            Phase total(c, &c->stats.ms_total);
            Phase ph(c, &c->stats.ms_restrict);
            NNM_TRY(cluster_literal(c, r, cap2, merges_dev, n_merges_host, labels_dev, n_clusters_host));
        }
        return read_stats(c);
    }
    {
        Phase total(c, &c->stats.ms_total);
        NNM_TRY(build_tree(c, c->opt.freeze_at_cap ? cap2 : INFINITY));
        const bool size_gates = r.kl2_max_pre_size > 0 || r.kl3_max_size > 0 || r.kl4_min_size > 0;
        // Many instances, none large: the per-instance walks (one CTA each, in parallel,
        // about 0.3 us per edge of the largest instance) beat the cut's levels over every
        // edge of the batch (about 9 ns per edge once its hash table leaves L2).
        const bool walk_instances = c->n_inst > 1 && c->max_inst_rows * 32 < c->N;
        int64_t n_cut = 0;
        if (!size_gates && !walk_instances) {
            // only the cap and KL1: a parallel cut, new sizes by halving rank ranges
            Phase ph(c, &c->stats.ms_restrict);
            NNM_TRY(ensure_cut(c, c->n_tree));
            CutArgs ca{};
            ca.edges = c->tree;
            ca.m = c->n_tree;
            ca.N = c->N;
            ca.cap2 = cap2;
            ca.kl1 = r.kl1_stop_clusters;
            ca.metric = c->metric;
            ca.n_inst = c->n_inst;
            ca.inst_off = c->inst_off;
            ca.ebeg = c->ebeg;
            ca.eend = c->eend;
            ca.inst_of_row = c->inst_pos;
            ca.merges = merges_dev;
            ca.n_merges = &c->dstat[4];
            ca.uf_parent = c->uf_parent;
            ca.err_flag = &c->derr[3];
            ca.cnt = c->cut_cnt;
            ca.lab = c->cut_lab;
            ca.w = c->cut_w;
            ca.slot = c->cut_slot;
            ca.hkey = c->cut_hkey;
            ca.hpar = c->cut_hpar;
            ca.hw = c->cut_hw;
            ca.hsum = c->cut_hsum;
            ca.hlab = c->cut_hlab;
            ca.H = c->cut_H;
            NNM_CUDA(c, launch_restrict_cut(ca, &n_cut, c->stream));
        } else if (r.kl4_min_size == 0 && c->n_inst == 1) {
            // KL2 / KL3 only: safe edges in parallel, the walk over the others
            Phase ph(c, &c->stats.ms_restrict);
            NNM_TRY(restrict_fast(c, r, cap2, merges_dev));
        } else {
            Phase ph(c, &c->stats.ms_restrict);
            RestrictArgs ra{};
            ra.edges = c->tree;
            ra.m = c->n_tree;
            ra.N = c->N;
            ra.cap2 = cap2;
            ra.kl1 = r.kl1_stop_clusters;
            ra.kl2 = r.kl2_max_pre_size;
            ra.kl3 = r.kl3_max_size;
            ra.kl4 = r.kl4_min_size;
            ra.uf_parent = c->uf_parent;
            ra.uf_size = c->uf_size;
            ra.deferred = c->deferred;
            ra.merges = merges_dev;
            ra.n_merges = &c->dstat[4];
            ra.err_flag = &c->derr[3];
            ra.n_inst = c->n_inst;
            ra.metric = c->metric;
            ra.inst_off = c->inst_off;
            ra.ebeg = c->ebeg;
            ra.eend = c->eend;
            ra.inst_nm = c->inst_nm;
            ra.merges_tmp = c->merges_tmp;
            NNM_CUDA(c, launch_restrict(ra, c->stream));
        }
        {
            Phase ph(c, &c->stats.ms_labels);
            LabelArgs la{};
            la.N = c->N;
            la.uf_parent = c->uf_parent;
            la.minm = c->minm;
            la.flag = c->flag;
            la.block_sums = c->block_sums;
            la.labels = labels_dev;
            la.K = &c->dstat[5];
            NNM_CUDA(c, launch_labels(la, c->stream));
        }
    }
    unsigned long long h[2];
    int uf_err = 0;
    NNM_CUDA(c, cudaMemcpyAsync(h, &c->dstat[4], sizeof h, cudaMemcpyDeviceToHost, c->stream));
    NNM_CUDA(c, cudaMemcpyAsync(&uf_err, &c->derr[3], sizeof uf_err, cudaMemcpyDeviceToHost, c->stream));
    NNM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (uf_err) {
        NNM_CUDA(c, cudaMemsetAsync(&c->derr[3], 0, sizeof(int), c->stream));
        return fail(c, NNM_ECUDA, "a union-find join in the restriction cut gave up");
    }
    *n_merges_host = (int64_t)h[0];
    *n_clusters_host = (int64_t)h[1];
    return read_stats(c);
}

nnm_status nnm_set_wait_limit(nnm_ctx *c, int64_t wait_limit_ns)
{
    if (!c) return NNM_EINVAL;
    if (wait_limit_ns < 0) return fail(c, NNM_EINVAL, "negative wait limit");
    c->opt.wait_limit_ns = wait_limit_ns;
    c->wait_ns = wait_limit(wait_limit_ns);
    return NNM_OK;
}

nnm_status nnm_cluster_host(const float *X_host, int64_t N, int32_t d, nnm_metric metric, nnm_precision precision,
                            const nnm_options *options, const nnm_restrictions *restrictions, void *cuda_stream,
                            nnm_merge *merges_host, int64_t *n_merges_host, int32_t *labels_host,
                            int64_t *n_clusters_host)
{
    if (!X_host || !merges_host || !n_merges_host || !labels_host || !n_clusters_host) return NNM_EINVAL;
    if (N < 2 || N >= (int64_t(1) << 31) || d < 1 || d > 32) return NNM_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float *X = nullptr;
    nnm_merge *mg = nullptr;
    int32_t *lab = nullptr;
    nnm_ctx *ctx = nullptr;
    nnm_status st = NNM_OK;
    auto cuda_status = [](cudaError_t e) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? NNM_ENOMEM : NNM_ECUDA;
    };
    do {
        cudaError_t e = pool_alloc(&X, (size_t)N * d, s);
        if (e == cudaSuccess) e = pool_alloc(&mg, (size_t)(N - 1), s);
        if (e == cudaSuccess) e = pool_alloc(&lab, (size_t)N, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(X, X_host, (size_t)N * d * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            st = cuda_status(e);
            break;
        }
        st = nnm_create(X, N, d, metric, precision, cuda_stream, options, &ctx);
        if (st != NNM_OK) break;
        int64_t nm = 0, K = 0;
        st = nnm_cluster(ctx, restrictions, mg, &nm, lab, &K);
        if (st != NNM_OK) break;
        e = cudaMemcpyAsync(merges_host, mg, (size_t)nm * sizeof(nnm_merge), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(labels_host, lab, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_status(e);
            break;
        }
        *n_merges_host = nm;
        *n_clusters_host = K;
    } while (0);
    nnm_destroy(ctx);   // synchronises the stream before freeing
    if (!ctx) cudaStreamSynchronize(s);
    if (X) cudaFreeAsync(X, s);
    if (mg) cudaFreeAsync(mg, s);
    if (lab) cudaFreeAsync(lab, s);
    cudaStreamSynchronize(s);
    return st;
}

nnm_status nnm_get_tree(nnm_ctx *c, nnm_edge *edges_dev, int64_t *n_edges_host)
{
    if (!c) return NNM_EINVAL;
    if (!edges_dev || !n_edges_host) return fail(c, NNM_EINVAL, "null output pointer");
    if (!c->tree) return fail(c, NNM_EINVAL, "no tree: call nnm_cluster first");
    NNM_CUDA(c, cudaMemcpyAsync(edges_dev, c->tree, c->n_tree * sizeof(nnm_edge), cudaMemcpyDeviceToDevice,
                                c->stream));
    NNM_CUDA(c, cudaStreamSynchronize(c->stream));
    *n_edges_host = c->n_tree;
    return NNM_OK;
}

nnm_status nnm_get_stats(const nnm_ctx *c, nnm_stats *out)
{
    if (!c || !out) return NNM_EINVAL;
    *out = c->stats;
    return NNM_OK;
}

const char *nnm_last_error(const nnm_ctx *c) { return c ? c->err.c_str() : "null context"; }

void nnm_destroy(nnm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    dfree(c, c->pos2row);
    dfree(c, c->tile_c);
    dfree(c, c->tile_rho);
    dfree(c, c->land_d2);
    dfree(c, c->lup);
    dfree(c, c->tile_lmin);
    dfree(c, c->blk_lmin);
    dfree(c, c->group);
    dfree(c, c->inst_off);
    dfree(c, c->inst_pos);
    dfree(c, c->ebeg);
    dfree(c, c->eend);
    dfree(c, c->inst_nm);
    dfree(c, c->inst_edges);
    dfree(c, c->merges_tmp);
    dfree(c, c->cut_cnt);
    dfree(c, c->cut_lab);
    dfree(c, c->cut_w);
    dfree(c, c->cut_slot);
    dfree(c, c->cut_hkey);
    dfree(c, c->cut_hpar);
    dfree(c, c->cut_hw);
    dfree(c, c->cut_hsum);
    dfree(c, c->cut_hlab);
    dfree(c, c->fw_cand);
    dfree(c, c->fw_walk);
    dfree(c, c->fw_dec);
    dfree(c, c->fw_unsafe);
    dfree(c, c->fw_pos);
    dfree(c, c->fw_blk);
    dfree(c, c->fw_edges);
    dfree(c, c->fw_cnt);
    dfree(c, c->blk_c);
    dfree(c, c->blk_rho);
    dfree(c, c->mu_f);
    dfree(c, c->row2pos);
    dfree(c, c->list_pos);
    dfree(c, c->Xs);
    dfree(c, c->XA);
    dfree(c, c->XB);
    dfree(c, c->r);
    dfree(c, c->P);
    dfree(c, c->E);
    dfree(c, c->cand_v);
    dfree(c, c->cand_j);
    dfree(c, c->cand_ovf);
    dfree(c, c->ovf_row);
    dfree(c, c->ovf_thr);
    dfree(c, c->ovf_thr_slot);
    dfree(c, c->ovf_flag);
    dfree(c, c->ovf_blk);
    dfree(c, c->slot_thr);
    dfree(c, c->coll_cnt);
    dfree(c, c->coll_j);
    dfree(c, c->coll_D);
    dfree(c, c->heavy_flag);
    dfree(c, c->heavy_blk);
    dfree(c, c->heavy_rows);
    dfree(c, c->heavy_rows2);
    dfree(c, c->heavy_thr);
    dfree(c, c->heavy_thr2);
    dfree(c, c->cache_j);
    dfree(c, c->cache_D);
    dfree(c, c->cache_n);
    dfree(c, c->cache_exh);
    dfree(c, c->row_B);
    dfree(c, c->comp_bound);
    dfree(c, c->comp_pos);
    dfree(c, c->tile_comp);
    dfree(c, c->comp);
    dfree(c, c->parent);
    dfree(c, c->list);
    dfree(c, c->row_D);
    dfree(c, c->row_ab);
    dfree(c, c->best_D);
    dfree(c, c->best_ab);
    dfree(c, c->row_state);
    dfree(c, c->frozen);
    dfree(c, c->flag_pos);
    dfree(c, c->block_cnt);
    dfree(c, c->edges);
    dfree(c, c->edges_tmp);
    dfree(c, c->uf_parent);
    dfree(c, c->uf_size);
    dfree(c, c->deferred);
    dfree(c, c->minm);
    dfree(c, c->flag);
    dfree(c, c->block_sums);
    dfree(c, c->dcount);
    dfree(c, c->dstat);
    dfree(c, c->derr);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

}  // extern "C"
