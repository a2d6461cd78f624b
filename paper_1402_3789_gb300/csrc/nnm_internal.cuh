// nnm_internal.cuh -- internal declarations of the sm_103a NNM clustering library.
//
// Layout of the device workspace, kernel argument blocks and launch wrappers shared
// between the translation units.  Nothing here is part of the C ABI (include/nnm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nnm.h"

namespace nnm {

// Process-wide count of kernel launches made by this library (read per call).
void count_launches(int n);
int64_t launches_so_far();

constexpr uint32_t kInvalid = 0xFFFFFFFFu;
constexpr int kListC = 80;        // record slots per (row, column range): 16 top + up to 64 band
constexpr int kMaxK = 16;         // largest k of nnm_nearest / cache width
constexpr int kRowTile = 256;     // rows per sweep CTA (both candidate paths)
constexpr int kMaxSplits = 32;    // column ranges per row tile
constexpr uint64_t kMaxKey = 0xFFFFFFFFFFFFFFFFull;
// Kernels whose dynamic shared memory depends on the launch set their limit to the
// largest the device allows them (its opt-in maximum less the kernel's static shared
// memory), one value per kernel: the limit is a per-function attribute, and host threads
// launching on different streams must not lower it below each other's requests (the
// request at launch still decides the occupancy).
template <typename Kernel>
inline cudaError_t set_max_dynamic_smem(Kernel *k)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

// State of a row's neighbour cache after a scan for its k nearest eligible columns:
constexpr uint8_t kCacheFull = 0;      // k found: every other eligible column has a larger key
constexpr uint8_t kCacheAll = 1;       // fewer found: they are every eligible column
constexpr uint8_t kCacheBounded = 2;   // fewer found: every other eligible column has D > the row's bound

// The exact D of a pair, e_k = x_ik - x_jk, each operation binary64 round-to-nearest,
// no contraction (the same value for (i, j) and (j, i)):
//   Euclidean (metric 0): Eq. (1) squared, ((t_0 + t_1) + ...) + t_{d-1}, t_k = e_k * e_k;
//   Manhattan (1): ((|e_0| + |e_1|) + ...) + |e_{d-1}|;  Chebyshev (2): max |e_k|.
__device__ __forceinline__ double canon_D(const float *__restrict__ xi, const float *__restrict__ xj, int d,
                                          int metric = 0)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double e = __dsub_rn((double)xi[k], (double)xj[k]);
        if (metric == 1) s = __dadd_rn(s, fabs(e));
        else if (metric == 2) s = fmax(s, fabs(e));
        else s = __dadd_rn(s, __dmul_rn(e, e));
    }
    return s;
}

struct Margin {
    int tensor;         // 0: FP32 direct candidates; 1: tensor-core candidates
    int metric;         // 0 Euclidean (D squared), 1 Manhattan, 2 Chebyshev
    double gamma;       // relative error bound of one candidate value
    double alpha;       // absolute slack (underflow)
    double R;           // tensor: max rounding radius over rows (scaled units)
    double Pmax;        // tensor: max |x_hat| over rows
    double Emax;        // tensor: max norm-split error over rows
    double inv_scale2;  // 1 / scale^2 (tensor candidates are in scaled units)
    const float *r;     // tensor: per-row rounding radius
    const float *P;     // tensor: per-row |x_hat|
    const float *E;     // tensor: per-row norm-split error
    double gamma32;     // FP32 direct refinement: relative bound gamma_{d+2}, u = 2^-24
    double alpha32;     //   and its underflow slack
};

// Per-launch constants of the sweeps' pruning threshold (an FP32 upper bound, rounded
// up, of the re-rank's binary64 threshold T; see select.cuh and rerank.cu).
struct SelConst {
    int tensor;
    float c1, c0;   // FP32 path: T = (v + c0) * c1 + c0
    float gamma;    // tensor path: accumulation bound
    float R, Pmax, Emax;
    float c1_32, c0_32;   // the re-rank's FP32 refinement: T32 = (v + c0_32) * c1_32 + c0_32
};

// ---------------------------------------------------------------------------------
// Candidate sweep (K1 FP32 direct / K2 tensor core): for each row slot, either keep
// the kListC smallest candidate values per column range (top-C mode) or append every
// eligible column whose value is <= the slot's threshold (collect mode).
// ---------------------------------------------------------------------------------
struct SweepArgs {
    // operands
    const float *Xs;          // FP32 path: [Npad][dp] padded copy of X
    int dp;
    const uint16_t *XA;       // tensor path: row operand, core-matrix interleaved [Npad][kpad]
    const uint16_t *XB;       // tensor path: column operand, same layout
    int kpad;
    int fp16;                 // tensor path: 1 FP16 operands, 0 BF16
    int band;                 // tensor path: band slots per row (32 or 64)
    int64_t N;
    // rows and columns are positions in the spatial order of the operands
    const uint32_t *rows;     // slot -> row position (nullptr: slot q is position q)
    int64_t nslots;
    const uint32_t *inst_pos;   // batched contexts: instance of each position (nullptr:
    const int64_t *inst_off;    // one instance); instance b = positions [inst_off[b], inst_off[b+1])
    const uint32_t *comp_pos;   // with comp: component of each position
    const uint32_t *tile_comp;  // with comp: component of each column tile of tile_w
                                // positions when they all share one, else kInvalid
    int metric;               // FP32 path: 0 Euclidean (squared), 1 Manhattan, 2 Chebyshev
    const double *row_B;      // per original row: only columns with exact D <= row_B are
                              // wanted (nullptr: no bound); a bound lowers the starting
                              // threshold of the row
    const uint32_t *pos2row;  // position -> original row index
    // eligibility
    const uint32_t *comp;     // nullptr: every column j != i is eligible; else comp[row(j)] != comp[row(i)]
    // columns
    int64_t col_begin, col_end, cols_per_split;
    int splits;
    // selection
    int kc;                   // the re-rank needs the kc smallest (1..16)
    Margin m;                 // per-row bound arrays (tensor path)
    SelConst sc;
    // top-C output: [nslots][splits][kListC] records and [nslots][splits] overflow flags
    float *out_v;
    uint32_t *out_j;
    uint8_t *out_ovf;
    // collect mode
    const float *thr;         // per slot, values <= thr are appended
    uint32_t *coll_cnt;       // per slot counters
    uint32_t *coll_j;         // [nslots][coll_cap]
    int64_t coll_cap;
    // bounded waits of the tensor kernel: a wait for work gives up after wait_ns
    // nanoseconds and raises *err_flag (the call returns NNM_ETIMEOUT)
    int *err_flag;
    uint64_t wait_ns;
    // tile pruning: bounding spheres of the column tiles (width tile_w positions) over
    // y = (x - mu_f) * scale_f, and the constants of the lower bound on candidate values
    int prune;
    int tile_w;
    const float *tile_c;      // [ntiles][2][d] two spheres per tile (split at a group change)
    const float *tile_rho;    // [ntiles][2] (-1: empty part)
    const uint32_t *group;    // [N] landmark group of each position (row tiles split alike)
    const float *blk_c;       // tensor path: [nblocks][d] sphere of each block of 32 tiles
    const float *blk_rho;     // [nblocks]
    // landmark bounds (triangle inequality through the landmark of a row): every pair
    // (i, j) has |y_i - y_j| >= lmin(j) - lup(i)
    const float *lup;         // [N] per position: upper bound on |y - y_l|, l its landmark
    const float *tile_lmin;   // [ntiles] lower bound on every column's distance to any landmark
    const float *blk_lmin;    // tensor path: [nblocks] the same over each block of 32 tiles
    const float *mu_f;        // [d] (nullptr: 0)
    float scale_f;
    float lb_R2;              // tensor: 2 * max rounding radius (scaled); FP32: 0
    float lb_eps;             // tensor: max candidate error; FP32: underflow slack
    float lb_gamma;           // FP32: relative candidate error; tensor: 0
    const float *X;           // original rows (row-tile spheres)
    int d;
    unsigned long long *st_tiles;   // [0] skipped, [1] evaluated column tiles
    unsigned int *slot_thr;   // [nslots] threshold shared by a row's column ranges (splits > 1)
};

// Bounding sphere of a set of points y (float, rounded up with a generous slack so that
// float rounding of y and of the distances can never make a bound invalid).
__device__ __forceinline__ float sphere_slack(float rho, float ymax)
{
    return __fadd_ru(__fmul_ru(rho, 1.0f + 0x1p-12f), __fmul_ru(ymax, 0x1p-12f)) + 1e-30f;
}

// Lower bound on the candidate value of any pair (row of the sphere (cR, rhoR), column
// of the sphere (cC, rhoC)): |y_i - y_j| >= |cR - cC| - rhoR - rhoC, the 16-bit operands
// differ from y by at most R each, and a candidate value differs from the squared
// operand distance by at most lb_eps (tensor) or a relative lb_gamma (FP32).
// Other metrics (FP32 path only): the Euclidean gap bounds them too, since
// |v|_1 >= |v|_2 and |v|_inf >= |v|_2 / sqrt(d); the candidate value is then the gap
// (Manhattan) or gap / sqrt(d) (Chebyshev) instead of its square.
// The bound from dist, a lower bound of the centre distance.
__device__ __forceinline__ float dist_lower_bound(float dist, float rhoR, float rhoC, int d, float lb_R2,
                                                  float lb_eps, float lb_gamma, int metric = 0)
{
    const float gap = dist - rhoR - rhoC - lb_R2;
    if (!(gap > 0.0f)) return -INFINITY;
    const float sq = metric == 0 ? gap * gap * (1.0f - 0x1p-12f)
                     : (metric == 1 ? gap : gap * rsqrtf((float)d) * (1.0f - 0x1p-12f));
    return sq * (1.0f - lb_gamma) - lb_eps;
}

// The bound from s = the FP32 sum of (cR_k - cC_k)^2 (the squared centre distance).
__device__ __forceinline__ float gap_lower_bound(float s, float rhoR, float rhoC, int d, float lb_R2, float lb_eps,
                                                 float lb_gamma, int metric = 0)
{
    return dist_lower_bound(sqrtf(s) * (1.0f - 0x1p-12f), rhoR, rhoC, d, lb_R2, lb_eps, lb_gamma, metric);
}

// Landmark bound: every column j of a tile has |y_j - y_l| >= lmin for every landmark l,
// and every row i of a part has |y_i - y_l(i)| <= dmax, so |y_i - y_j| >= lmin - dmax.
__device__ __forceinline__ float land_lower_bound(float lmin, float dmax, int d, float lb_R2, float lb_eps,
                                                  float lb_gamma, int metric = 0)
{
    return dist_lower_bound(lmin, dmax, 0.0f, d, lb_R2, lb_eps, lb_gamma, metric);
}

__device__ __forceinline__ float tile_lower_bound(const float *cR, float rhoR, const float *cC, float rhoC, int d,
                                                  float lb_R2, float lb_eps, float lb_gamma, int metric = 0)
{
    // fully unrolled so that the (predicated) loads of cC issue together
    float c[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) c[k] = k < d ? cC[k] : 0.0f;
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (k < d) {
            const float e = cR[k] - c[k];
            s = fmaf(e, e, s);
        }
    }
    return gap_lower_bound(s, rhoR, rhoC, d, lb_R2, lb_eps, lb_gamma, metric);
}

// Launch the FP32 direct sweep (template on d).
cudaError_t launch_sweep_fp32(const SweepArgs &a, int d, bool collect, cudaStream_t s);
// Launch the tcgen05 sweep.
cudaError_t launch_sweep_tc(const SweepArgs &a, bool collect, cudaStream_t s);
size_t sweep_tc_smem_bytes(int kpad, int band);

// ---------------------------------------------------------------------------------
// Exact re-rank (K3)
// ---------------------------------------------------------------------------------
struct FinalizeArgs {
    const float *X;            // user's rows [N][d]
    int d;
    int64_t N;
    const uint32_t *rows;      // slot -> row position (nullptr: identity)
    const uint32_t *pos2row;   // position -> original row index
    int64_t nslots;
    int splits;
    const float *in_v;         // [nslots][splits][kListC]
    const uint32_t *in_j;
    const uint8_t *in_ovf;     // [nslots][splits]
    int k;                     // results per row
    Margin m;
    SelConst sc;               // FP32 upper bounds of the thresholds (as the sweeps use them)
    // results (indexed by row)
    uint32_t *res_j;           // [N][k]
    double *res_D;             // [N][k]
    uint8_t *res_n;            // valid results per row (nullable)
    uint8_t *res_exh;          // cache state per row (kCache*, nullable)
    int res_stride;            // row stride of res_j / res_D (>= k)
    const double *row_B;       // per original row: keep only D <= row_B (nullptr: no bound)
    // incomplete rows -> collect pass (compacted afterwards in slot order, so that the
    // collect pass keeps the spatial order of the rows)
    uint8_t *ovf_flag;         // [nslots] 1: the slot's candidate lists are incomplete
    float *ovf_thr;            // [nslots] its threshold (rounded up), where flagged
    // statistics
    unsigned long long *st_max_abs;   // double bits
    unsigned long long *st_max_rel;
    unsigned long long *st_pairs;
    unsigned long long *st_max_cand;
};

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s);

struct CollectRerankArgs {
    const float *X;
    int d;
    int64_t N;
    const uint32_t *rows;      // collect slot p -> row position
    const uint32_t *pos2row;   // position -> original row index
    int64_t n;                 // collect slots
    const uint32_t *coll_cnt;  // [n]
    const uint32_t *coll_j;    // [n][cap]
    int64_t cap;
    double *scratch_D;         // [n][cap]
    int k;
    Margin m;
    SelConst sc;               // FP32 refinement bounds
    uint32_t *res_j;
    double *res_D;
    uint8_t *res_n;
    uint8_t *res_exh;
    int res_stride;
    const double *row_B;       // as in FinalizeArgs
    int *retry_flag;           // set when a slot collected more than cap
    uint8_t *heavy_flag;       // [heavy_base + p] 1: slot p collected more than cap
    int64_t heavy_base;
    unsigned long long *heavy_max;   // largest such count
    unsigned long long *st_pairs;
    unsigned long long *st_max_cand;
};

cudaError_t launch_collect_rerank(const CollectRerankArgs &a, cudaStream_t s);

// ---------------------------------------------------------------------------------
// Preparation
// ---------------------------------------------------------------------------------
cudaError_t launch_check_finite(const float *X, int64_t n, int *flag, cudaStream_t s);
// Spatial order (prep.cu): chain rank of S <= 1024 coarse landmarks; nearest reference
// row of each query row (queries and references at regular strides of X); sort keys of
// the landmarks (which = 0) or of the rows (which = 1, with the isolation threshold from
// a histogram of 4096 bins); positions from sorted keys.
constexpr int kMaxGroups = 4096;
cudaError_t launch_landmark_chain(const float *X, int64_t N, int d, int64_t L, uint32_t *rank, cudaStream_t s);
cudaError_t launch_nearest_ref(const float *X, int64_t N, int d, int64_t Q, int64_t R, uint32_t *arg, float *dist,
                               cudaStream_t s);
cudaError_t launch_spatial_keys(const uint32_t *larg, const float *ldist, int64_t L, const uint32_t *crank,
                                const uint32_t *rarg, const float *rdist, int64_t N, const uint32_t *lrank,
                                const uint32_t *inst /* nullable: instance of each row, most significant */,
                                unsigned int *hist, float *tau, nnm_edge *lkeys, nnm_edge *rkeys, int which,
                                cudaStream_t s);
// inst[p] = b for p in [off[b], off[b+1])
cudaError_t launch_instance_ids(const int64_t *off, int64_t B, int64_t N, uint32_t *inst, cudaStream_t s);
cudaError_t launch_order_from_keys(const nnm_edge *keys, int64_t N, uint32_t *pos2row, uint32_t *row2pos,
                                   uint32_t *group /* nullable: landmark group per position */, cudaStream_t s);
// out[q] = map[in[q]]
cudaError_t launch_gather_u32(const uint32_t *in, const uint32_t *map, int64_t n, uint32_t *out, cudaStream_t s);
// Ordered compaction: for every q < n with flag[q] != 0, in increasing q, append
// rows[q] (q itself if rows is null) to out_rows and vals[q] to out_vals; the number
// appended goes to *count.  block_cnt holds compact_blocks(n) words of scratch.
int64_t compact_blocks(int64_t n);
cudaError_t launch_compact(const uint8_t *flag, int64_t n, const uint32_t *rows, const float *vals, uint32_t *block_cnt,
                           uint32_t *out_rows, float *out_vals, uint32_t *count, cudaStream_t s);
cudaError_t launch_gather_f32(const uint32_t *in, const float *map, int64_t n, float *out, cudaStream_t s);
// padded FP32 copy in position order
cudaError_t launch_pad_fp32(const float *X, int64_t N, int d, int dp, int64_t Npad, const uint32_t *pos2row,
                            float *Xs, cudaStream_t s);
// column means in binary64 (deterministic order); partial: [blocks][d]
cudaError_t launch_mean(const float *X, int64_t N, int d, double *partial, int blocks, double *mu,
                        cudaStream_t s);
int mean_blocks(int64_t N);
cudaError_t launch_max_sqnorm(const float *X, int64_t N, int d, const double *mu,
                              unsigned long long *out_bits, cudaStream_t s);
// operands written at each row's position; r, P, E stay indexed by original row
// Bounding spheres of the column tiles (tile_w consecutive positions).
// Bounding spheres of blocks of 32 consecutive tiles, from the tiles' two spheres each.
cudaError_t launch_block_spheres(const float *tile_c, const float *tile_rho, int64_t ntiles, int d, float *blk_c,
                                 float *blk_rho, const float *tile_lmin, float *blk_lmin, cudaStream_t s);
// With land_d2 (per row: FP32 squared distance to the nearest landmark, x units), also
// lup [N] and tile_lmin [ntiles] in y units (scale_f times x units, plus land_slack for
// the rounding of y = (x - mu) * scale).
cudaError_t launch_tile_spheres(const float *X, int64_t N, int d, const uint32_t *pos2row, const uint32_t *group,
                                const float *mu_f, float scale_f, int tile_w, float *tile_c, float *tile_rho,
                                const float *land_d2, float land_slack, float *lup, float *tile_lmin, cudaStream_t s);
cudaError_t launch_tc_operands(const float *X, int64_t N, int d, const double *mu, double scale,
                               int fp16, int terms, int kpad, int64_t Npad, const uint32_t *pos2row, uint16_t *XA,
                               uint16_t *XB,
                               float *r, float *P, float *E, unsigned long long *max_bits /*[3]*/,
                               cudaStream_t s);

// ---------------------------------------------------------------------------------
// Merge rounds (K4/K5)
// ---------------------------------------------------------------------------------
struct RoundState {
    int64_t N;
    int k;                         // cache width
    uint32_t *comp;                // [N] component id (= root row id)
    uint32_t *parent;              // [N] hook target per component root
    const uint32_t *cache_j;       // [N][k]
    const double *cache_D;
    const uint8_t *cache_n;
    const uint8_t *cache_exh;
    double *row_B;                 // [N] bound of the row's last (re)scan: a cache with fewer
                                   // than k entries holds every eligible column with
                                   // D <= row_B (+inf: unbounded; then cache_exh is set)
    unsigned long long *comp_bound;   // [N] per component: D bits of some outgoing pair
    double overscan;               // rescan bound = overscan * the component's bound
    const float *X;                // [N][d] the rows (exact distances of the bound search)
    int d;
    int metric;
    const uint32_t *inst_pos;      // batched contexts: instance of each position (nullable)
    const int64_t *inst_off;       // batched: first row of each instance, and N
    uint32_t *inst_edges;          // batched: tree edges found so far per instance; an
                                   // instance with rows - 1 of them is one component, so
                                   // its rows have no outgoing pair and are not rescanned
    unsigned long long *row_D;     // [N] key of the row's best outgoing candidate (D bits)
    unsigned long long *row_ab;    // [N] (min << 32) | max
    uint8_t *row_state;            // 0 none, 1 resolved, 2 unresolved (row_D/row_ab: bound)
    unsigned long long *best_D;    // [N] per component
    unsigned long long *best_ab;
    uint32_t *list;                // [N] rescan rows (original indices, position order)
    uint32_t *list_pos;            // [N] their positions, increasing
    uint8_t *flag_pos;             // [N] rescan flag per position
    uint32_t *block_cnt;           // [ceil(N / 1024)] compaction scratch
    const uint32_t *row2pos, *pos2row;
    uint32_t *counters;            // [0] rescans, [1] edges this round, [2] jump changes
    nnm_edge *edges;               // [N-1]
    uint32_t *n_edges;             // device count
    uint8_t *frozen;               // [N] per component root
    double cap2;                   // freeze threshold (inf: none)
};

cudaError_t launch_round_init(RoundState &st, cudaStream_t s);
cudaError_t launch_resolve(RoundState &st, const uint32_t *rows, int64_t nrows, cudaStream_t s);
cudaError_t launch_component_min(RoundState &st, cudaStream_t s);
cudaError_t launch_flag_rescans(RoundState &st, cudaStream_t s);
cudaError_t launch_hook(RoundState &st, cudaStream_t s);
cudaError_t launch_jump(RoundState &st, cudaStream_t s);
cudaError_t launch_relabel(RoundState &st, cudaStream_t s);
// comp_pos[p] = comp[pos2row[p]]; tile_comp[t] = the component of tile t (tile_w
// consecutive positions) if it is one for the whole tile, else kInvalid
cudaError_t launch_position_comps(const RoundState &st, int tile_w, uint32_t *comp_pos, uint32_t *tile_comp,
                                  cudaStream_t s);

// ---------------------------------------------------------------------------------
// Sort (K6), restriction walk (K7), labels (K8)
// ---------------------------------------------------------------------------------
cudaError_t launch_sort_edges(nnm_edge *e, nnm_edge *tmp, int64_t m, cudaStream_t s,
                              nnm_edge **sorted_out, const uint32_t *major = nullptr);

struct RestrictArgs {
    const nnm_edge *edges;     // key-sorted tree edges
    int64_t m;
    int64_t N;
    double cap2;               // inf: none
    int64_t kl1, kl2, kl3, kl4;
    uint32_t *uf_parent;       // [N] scratch
    uint32_t *uf_size;         // [N] scratch
    uint32_t *deferred;        // [m] scratch (KL4 second walk)
    nnm_merge *merges;         // [N-1] out
    unsigned long long *n_merges; // device out
    int *err_flag;
    int metric;                // a merge's length: sqrt(D) (Euclidean) or D
    // batched contexts: one walk per instance (CTA b), the edges sorted by (instance,
    // key); instance b = rows [inst_off[b], inst_off[b+1]), edges [ebeg[b], eend[b]).
    // Each walk writes its merges at merges_tmp[ebeg[b]..] and their count to inst_nm[b];
    // launch_restrict then packs them into merges in instance order.
    int64_t n_inst;
    const int64_t *inst_off;
    const int64_t *ebeg, *eend;
    unsigned long long *inst_nm;   // [n_inst + 1] scratch
    nnm_merge *merges_tmp;         // [m] scratch
    // the all-pairs reading (literal.cu): one walk over a key-sorted batch of pairs that
    // continues the union-find, the merges, the join count and the KL1 stop of the batches
    // before it (persist = 1: no initialisation; merges appended at *n_merges; *joined_io
    // and *stop_io carried in and out).  lit_phase 1 skips a pair whose clusters both
    // have at least KL4 rows (it waits for the second phase); 2 applies no KL4 test.
    int persist;
    int lit_phase;
    long long *joined_io;
    int *stop_io;
};

cudaError_t launch_restrict(const RestrictArgs &a, cudaStream_t s);
// ebeg[b], eend[b]: the edge range of each instance in edges sorted by (instance, key)
cudaError_t launch_edge_ranges(const nnm_edge *edges, int64_t m, const uint32_t *inst_of_row, int64_t n_inst,
                               int64_t *ebeg, int64_t *eend, cudaStream_t s);

// Restriction step when no gate reads cluster sizes (cap and KL1 only): a parallel
// cut of each instance's key-ordered edges and the new sizes by halving rank ranges
// (dendro.cu).  Instances as in RestrictArgs.
struct CutArgs {
    const nnm_edge *edges;     // tree edges sorted by (instance, key)
    int64_t m;
    int64_t N;
    double cap2;               // inf: none
    int64_t kl1;
    int metric;
    int64_t n_inst;
    const int64_t *inst_off, *ebeg, *eend;   // batched only
    const uint32_t *inst_of_row;             // batched only
    nnm_merge *merges;         // [m] out: the accepted joins, (instance, key) order
    unsigned long long *n_merges;   // device out
    uint32_t *uf_parent;       // [N] out: a union-find of the final clusters
    int *err_flag;             // set if a union gave up (never expected)
    // scratch
    unsigned long long *cnt;   // [n_inst + 1]
    uint32_t *lab, *w, *slot;  // [2m] each
    unsigned long long *hkey;  // [H]
    uint32_t *hpar, *hw, *hsum, *hlab;   // [H]
    int64_t H;                 // cut_hash_slots(m)
};

int64_t cut_hash_slots(int64_t m);
// Returns after one synchronisation (the accepted count decides the levels).
cudaError_t launch_restrict_cut(const CutArgs &a, int64_t *n_merges_host, cudaStream_t s);

// The restrictions in the all-pairs reading (literal.cu): batches of pairs that cross two
// clusters and pass every gate at the batch start, cut by FP32 value and kept exactly.
struct LitArgs {
    const float *X;            // the caller's rows [N][d]
    int d;
    int64_t N;
    int metric;
    double cap2;               // cap in D units (inf: none)
    float cap2f;               // an FP32 value >= cap2
    int64_t kl2, kl3, kl4;
    int phase;                 // 1: pairs touching a cluster below KL4 only; 2: the rest
    uint32_t *uf_parent, *uf_size;       // [N] union-find of the walk
    uint32_t *comp, *csize;              // [N] per row: root and its size at the batch start
    double *tD;                          // [N] per row: key of the phase-1 join that brought
    unsigned long long *tab;             //     its cluster to KL4 rows (D, a << 32 | b)
    uint32_t *w0, *w1, *w2, *w3, *w4;    // [N] scratch of k_lit_reach
    float c0, c1, c1inv;       // FP32 margin: D <= (s + c0) c1 + c0, D >= (s - c0) c1inv - c0
    int have_last;             // 0 before the first batch of a phase
    double last_D;             // the previous batch covered every pair with D <= last_D
    double tau_D;              // this batch: pairs with last_D < D <= tau_D
    unsigned int octave;       // fine histogram: the FP32 exponent field it refines
    float cut;                 // emit: pairs with FP32 value <= cut
    unsigned long long *hist;  // [256] (by exponent) or [literal_fine_bins()]
    nnm_edge *emit;            // [emit_cap] emitted pairs
    int64_t emit_cap;
    unsigned long long *n_emit;
    int64_t n_emitted;
    nnm_edge *kept;            // [emit_cap] pairs kept by the binary64 test
    unsigned long long *n_kept;
};
int literal_fine_bins();
// mode 0: histogram by exponent; 1: histogram of one octave; 2: emit up to the cut
cudaError_t launch_lit_pass(const LitArgs &a, int mode, cudaStream_t s);
cudaError_t launch_lit_exact(const LitArgs &a, cudaStream_t s);
cudaError_t launch_lit_flatten(const LitArgs &a, cudaStream_t s);
cudaError_t launch_lit_init(const LitArgs &a, double t0, cudaStream_t s);
cudaError_t launch_lit_reach(const LitArgs &a, const nnm_merge *merges, int64_t n1, cudaStream_t s);

// KL2 / KL3 without KL4, one instance (dendro.cu): safe edges joined in parallel, the
// walk only over the others.  cand: the admissible edges as nnm_merge records in key
// order with their unrestricted new sizes, w: the two unrestricted endpoint sizes.
struct FastWalkArgs {
    int64_t N, M;
    int64_t kl2, kl3;
    nnm_merge *cand;           // [M] admissible edges (key order); new sizes fixed here
    const uint32_t *w;         // [2M] unrestricted sizes of both endpoints' clusters before each edge
    uint8_t *dec;              // [M] 1: joined
    uint8_t *unsafe;           // [M] 1: the walk decides it
    uint32_t *pos;             // [M] positions (compaction output)
    nnm_edge *unsafe_edges;    // [M] the unsafe edges in key order (the walk's input)
    nnm_merge *walk_out;       // [M] the walk's joins (key order)
    uint32_t *uf_parent, *uf_size;   // [N]
    nnm_merge *merges;         // [N-1] out
    int *err_flag;
};
// step 0 mark, 1 join safe edges and size the clusters, 2 gather n unsafe edges (pos),
// 3 place n accepted unsafe joins, 4 emit n joins (pos), 5 final union-find of n joins
cudaError_t launch_fast_walk_steps(const FastWalkArgs &f, int step, int64_t n, cudaStream_t s);

struct LabelArgs {
    int64_t N;
    uint32_t *uf_parent;       // union-find after the restriction walk
    uint32_t *minm;            // [N] scratch
    uint32_t *flag;            // [N] scratch (first member flags -> ranks)
    uint32_t *block_sums;      // scratch
    int32_t *labels;           // out
    unsigned long long *K;     // device out
};

cudaError_t launch_labels(const LabelArgs &a, cudaStream_t s);
int64_t labels_scratch_blocks(int64_t N);

}  // namespace nnm
