// sweep_fp32.cu -- K1: all-pairs candidate sweep with FP32 direct differences.
//
// The second and third parallel items of the paper ("Overall idea of the algorithm":
// distances between all pairs, then selection of the minimum distances) fused into
// one pass over row tile x column range (the paper pairs two blocks of the data in
// each step of its pair construction).  Each thread owns two rows (registers) and each step
// evaluates two columns from shared memory (cp.async, double buffered):
//     s~(i,j) = fl32( sum_k (x_ik - x_jk)^2 ),   k = 0..d-1 in order, one FMA per k.
// Features beyond d are zero in both operands (adding +0 leaves the sum unchanged), so
// one instantiation per multiple of four covers every d; d = 25 has its own.
// A value passes the fast test only if it is <= the row's pruning threshold (see
// select.cuh); the slow path checks eligibility (j != i, j inside the range, and with
// a mask comp[j] != comp[i]) and updates the row's selection, or in collect mode
// appends j to the row's global segment.
//
// Error bound used by the re-rank: |s~ - s| <= gamma_{d+2} * s (u = 2^-24) plus an
// underflow term, s the exact squared distance of the FP32 inputs.
#include <cuda_pipeline_primitives.h>

#include <type_traits>

#include "select.cuh"

namespace nnm {

namespace {

constexpr int kThreads = 128;
constexpr int kTile = 64;   // columns per shared-memory tile
constexpr int kBand = 32;   // band slots per row (the FP32 band is narrow)

template <int D, int KC, bool COLLECT>
__global__ void __launch_bounds__(kThreads, 2) k_sweep_fp32(const SweepArgs a)
{
    constexpr int DP = (D + 3) & ~3;
    __shared__ __align__(16) float sy[2][kTile * DP];
    extern __shared__ __align__(16) uint8_t dsm[];
    float *band_v = reinterpret_cast<float *>(dsm);                       // [kBand][kRowTile]
    uint32_t *band_j = reinterpret_cast<uint32_t *>(band_v + kBand * kRowTile);

    const int t = threadIdx.x;
    const int64_t slot[2] = {(int64_t)blockIdx.x * kRowTile + t, (int64_t)blockIdx.x * kRowTile + t + kThreads};
    bool valid[2];
    uint32_t row[2], crow[2];
    float x[2][D];
    float cthr[2];
    RowSel<KC, kBand> sel[2];
    const RowConst rc{0.f, 0.f};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        valid[r] = slot[r] < a.nslots;
        row[r] = valid[r] ? (a.rows ? a.rows[slot[r]] : (uint32_t)slot[r]) : 0u;   // position
        crow[r] = (valid[r] && a.comp) ? a.comp_pos[row[r]] : 0u;
        const float *xr = a.Xs + (int64_t)row[r] * a.dp;
#pragma unroll
        for (int k = 0; k < D; ++k) x[r][k] = k < a.dp ? xr[k] : 0.0f;
        cthr[r] = (COLLECT && valid[r]) ? a.thr[slot[r]] : -INFINITY;
        sel[r].init(valid[r]);
    }

    // Column tiles in the order of the operands, starting at this row tile's own place and
    // wrapping around (near neighbours first); split s takes the s-th range of that order.
    // In a batched context only the tiles of the row tile's instances, [rtb, rte).
    const int split = blockIdx.y;
    const int64_t slot_first = (int64_t)blockIdx.x * kRowTile;
    const int64_t p_first = a.rows ? a.rows[slot_first] : slot_first;
    int64_t rtb = 0, rte = (a.N + kTile - 1) / kTile;
    if (a.inst_pos) {
        const int64_t last = (slot_first + kRowTile < a.nslots ? slot_first + kRowTile : a.nslots) - 1;
        const int64_t p_last = a.rows ? a.rows[last] : last;
        rtb = a.inst_off[a.inst_pos[p_first]] / kTile;
        rte = (a.inst_off[a.inst_pos[p_last] + 1] + kTile - 1) / kTile;
    }
    const int64_t ntile_all = rte - rtb;
    const int64_t tile0 = p_first / kTile - rtb;
    // tiles per column range: of the whole matrix, or (batched) of this row tile's range
    const int64_t tps = a.inst_pos ? (ntile_all + a.splits - 1) / a.splits : a.cols_per_split / kTile;
    const int64_t t_begin = (int64_t)split * tps;
    const int64_t t_end = t_begin + tps < ntile_all ? t_begin + tps : ntile_all;
    const int64_t ntiles = t_end > t_begin ? t_end - t_begin : 0;
    const int64_t start = (tile0 + t_begin) % ntile_all;
    auto tile_col = [&](int64_t tile) -> int64_t {
        const int64_t x = start + tile;
        return (rtb + (x >= ntile_all ? x - ntile_all : x)) * kTile;
    };
    // the columns of each row's instance (all columns when not batched)
    int64_t ibeg[2] = {0, 0}, iend[2] = {a.N, a.N};
    if (a.inst_pos) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (valid[r]) {
                ibeg[r] = a.inst_off[a.inst_pos[row[r]]];
                iend[r] = a.inst_off[a.inst_pos[row[r]] + 1];
            }
    }

    // operand rows hold a.dp floats; the tile keeps DP >= a.dp per column (rest zero)
    if (a.dp < DP)
        for (int q = t; q < 2 * kTile * DP; q += kThreads) (&sy[0][0])[q] = 0.0f;
    // Tile pruning: bounding spheres of this CTA's rows (the operands are the raw rows)
    // in two parts, the rows of the first landmark group and the rest, and each part's
    // largest row threshold after each tile.
    __shared__ float cR[2][32], wthr[2][kThreads / 32], blk_thr[2];
    __shared__ unsigned int rho_bits[2], ymax_bits, cmin, cmax, lup_bits[2];
    __shared__ int nvalid[2];
    if (t < 64) (&cR[0][0])[t] = 0.0f;
    if (t == 0) {
        rho_bits[0] = rho_bits[1] = 0u;
        lup_bits[0] = lup_bits[1] = 0u;
        ymax_bits = 0u;
        nvalid[0] = nvalid[1] = 0;
        blk_thr[0] = blk_thr[1] = INFINITY;
        cmin = 0xFFFFFFFFu;
        cmax = 0u;
    }
    int part[2] = {0, 0};
    if (a.prune) {
        const uint32_t g0 = a.group[a.rows ? a.rows[(int64_t)blockIdx.x * kRowTile] : (uint32_t)(blockIdx.x * kRowTile)];
#pragma unroll
        for (int r = 0; r < 2; ++r) part[r] = (valid[r] && a.group[row[r]] != g0) ? 1 : 0;
    }
    __syncthreads();
    if (a.comp) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (valid[r]) {
                atomicMin(&cmin, crow[r]);
                atomicMax(&cmax, crow[r]);
            }
    }
    if (a.prune) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!valid[r]) continue;
            float ny = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                ny = fmaf(x[r][k], x[r][k], ny);
                atomicAdd(&cR[part[r]][k], x[r][k]);
            }
            atomicAdd(&nvalid[part[r]], 1);
            atomicMax(&ymax_bits, __float_as_uint(sqrtf(ny)));
            if (a.lup) atomicMax(&lup_bits[part[r]], __float_as_uint(a.lup[row[r]]));
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!valid[r]) continue;
            float dd = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float e = x[r][k] - cR[part[r]][k] / (float)nvalid[part[r]];
                dd = fmaf(e, e, dd);
            }
            atomicMax(&rho_bits[part[r]], __float_as_uint(sqrtf(dd)));
        }
        __syncthreads();
        if (t < 64 && (t & 31) < D) cR[t >> 5][t & 31] /= (float)(nvalid[t >> 5] > 0 ? nvalid[t >> 5] : 1);
    }
    __syncthreads();
    float rhoR[2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
        rhoR[h] = nvalid[h] > 0 ? sphere_slack(__uint_as_float(rho_bits[h]), __uint_as_float(ymax_bits)) : -1.0f;
    // First kept tile at or after `from`.  Every thread takes the same decision; the lower
    // bounds of kThreads consecutive tiles are computed together (one per thread) into
    // lb_s when the scan leaves the current batch.
    // A masked sweep whose rows all lie in one component skips that component's tiles.
    __shared__ float lb_s[kThreads];
    __shared__ uint8_t own_s[kThreads];
    const uint32_t rcomp = (a.comp && cmin == cmax) ? cmin : kInvalid;
    int64_t lb_base = -(int64_t)kThreads;
    __shared__ float lb_s2[kThreads];
    auto next_kept = [&](int64_t from) -> int64_t {
        if (!a.prune && rcomp == kInvalid) return from;
        const float thr0 = blk_thr[0], thr1 = blk_thr[1];
        for (int64_t q = from; q < ntiles; ++q) {
            if (q >= lb_base + kThreads) {
                __syncthreads();   // the previous batch is no longer read
                lb_base = q;
                float lb[2] = {-INFINITY, -INFINITY};
                uint8_t own = 0;
                if (q + t < ntiles) {
                    const int64_t ct = tile_col(q + t) / kTile;
                    own = rcomp != kInvalid && a.tile_comp[ct] == rcomp;
                    if (a.prune && !own) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            lb[h] = INFINITY;
                            if (rhoR[h] >= 0.0f) {
                                for (int hc = 0; hc < 2; ++hc) {
                                    const float rc = a.tile_rho[ct * 2 + hc];
                                    if (rc >= 0.0f)
                                        lb[h] = fminf(lb[h], tile_lower_bound(cR[h], rhoR[h], a.tile_c + (ct * 2 + hc) * a.d,
                                                                              rc, a.d, 0.0f, a.lb_eps, a.lb_gamma,
                                                                              a.metric));
                                }
                                // the landmark bound of the tile (see tile_lower_bound's notes on metrics)
                                if (a.lup && a.tile_lmin[ct] > 0.0f)
                                    lb[h] = fmaxf(lb[h], land_lower_bound(a.tile_lmin[ct], __uint_as_float(lup_bits[h]),
                                                                          a.d, 0.0f, a.lb_eps, a.lb_gamma, a.metric));
                            }
                        }
                    }
                }
                lb_s[t] = lb[0];
                lb_s2[t] = lb[1];
                own_s[t] = own;
                __syncthreads();
            }
            const int e = (int)(q - lb_base);
            if (!own_s[e] && (!(lb_s[e] > thr0) || !(lb_s2[e] > thr1))) return q;
        }
        return ntiles;
    };
    auto load_tile = [&](int64_t tile, int buf) {
        const int64_t j0 = tile_col(tile);
        int64_t n = a.N - j0;
        if (n > kTile) n = kTile;
        const int per = a.dp / 4;
        const int chunks = (int)n * per;
        const float *src = a.Xs + j0 * a.dp;
        for (int q = t; q < chunks; q += kThreads) {
            const int c = q / per, w = q - c * per;
            __pipeline_memcpy_async(&sy[buf][c * DP + w * 4], src + (int64_t)q * 4, 16);
        }
    };

    uint32_t tcomp = kInvalid;   // component of the current column tile (kInvalid: mixed)
    auto consider = [&](int r, float v, uint32_t j) {
        if ((int64_t)j >= a.N || j == row[r]) return;
        if ((int64_t)j < ibeg[r] || (int64_t)j >= iend[r]) return;   // another instance
        if (a.comp && (tcomp != kInvalid ? tcomp == crow[r] : a.comp_pos[j] == crow[r])) return;
        if (COLLECT) {
            if (!(v <= cthr[r])) return;
            const uint32_t p = atomicAdd(&a.coll_cnt[slot[r]], 1u);
            if ((int64_t)p < a.coll_cap) a.coll_j[slot[r] * a.coll_cap + p] = j;
        } else {
            if (!(v <= sel[r].thr)) return;
            sel[r].insert(v, j, a.sc, rc, band_v + t + r * kThreads, band_j + t + r * kThreads, kRowTile);
        }
    };

    // the block's largest row threshold, for the tile decisions of every thread
    // (an empty part keeps -inf: its lower bound never keeps a tile)
    auto publish = [&](float th0, float th1) {
        float wt[2] = {-INFINITY, -INFINITY};
        wt[part[0]] = th0;
        wt[part[1]] = fmaxf(wt[part[1]], th1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wt[h] = fmaxf(wt[h], __shfl_xor_sync(0xffffffffu, wt[h], o));
            if ((t & 31) == 0) wthr[h][t >> 5] = wt[h];
        }
        __syncthreads();
        if (t < 2) {
            float m = wthr[t][0];
            for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, wthr[t][w]);
            blk_thr[t] = m;
        }
        __syncthreads();
    };
    // Thresholds already published for these rows by other column ranges; a collect pass
    // knows its thresholds from the start.
    if (!COLLECT && a.row_B) {
        // a bounded row starts at the threshold of its bound
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!valid[r]) continue;
            const double B = a.row_B[a.pos2row[row[r]]];
            if (B < INFINITY) sel[r].bound(sel_threshold(a.sc, rc, __double2float_ru(B / a.m.inv_scale2)));
        }
    }
    if (!COLLECT && a.splits > 1) {
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (valid[r]) sel[r].bound(shared_thr_exchange(&a.slot_thr[slot[r]], INFINITY));
    }
    if (a.prune) publish(COLLECT ? cthr[0] : sel[0].thr, COLLECT ? cthr[1] : sel[1].thr);

    int64_t tile = next_kept(0);
    int buf = 0;
    int64_t swept = 0;
    if (tile < ntiles) load_tile(tile, 0);
    __pipeline_commit();
    while (tile < ntiles) {
        const int64_t nxt = next_kept(tile + 1);
        if (nxt < ntiles) load_tile(nxt, buf ^ 1);
        __pipeline_commit();
        __pipeline_wait_prior(1);
        __syncthreads();
        const float *ys = sy[buf];
        const int64_t j0 = tile_col(tile);
        const int n = (int)(a.N - j0 < kTile ? a.N - j0 : kTile);
        float th0 = COLLECT ? cthr[0] : sel[0].thr;
        float th1 = COLLECT ? cthr[1] : sel[1].thr;
        tcomp = a.comp ? a.tile_comp[tile_col(tile) / kTile] : kInvalid;
        // rows of the tile's own component have nothing eligible in it
        const bool own0 = !valid[0] || (a.comp && tcomp != kInvalid && tcomp == crow[0]);
        const bool own1 = !valid[1] || (a.comp && tcomp != kInvalid && tcomp == crow[1]);
        // the column loop, one copy per metric (the branch is outside the loop)
        auto columns = [&](auto metric_tag) {
            constexpr int M = decltype(metric_tag)::value;
            for (int c = (own0 && own1) ? n : 0; c < n; c += 2) {
                const float4 *ya = reinterpret_cast<const float4 *>(ys + c * DP);
                const float4 *yb = reinterpret_cast<const float4 *>(ys + (c + 1) * DP);
                float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll
                for (int q = 0; q < DP / 4; ++q) {
                    const float4 A = ya[q], B = yb[q];
                    const float av[4] = {A.x, A.y, A.z, A.w};
                    const float bv[4] = {B.x, B.y, B.z, B.w};
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int k = q * 4 + w;
                        if (k < D) {
                            const float e00 = x[0][k] - av[w], e01 = x[0][k] - bv[w];
                            const float e10 = x[1][k] - av[w], e11 = x[1][k] - bv[w];
                            if constexpr (M == 0) {   // Euclidean: e^2 summed (one FMA)
                                s00 = fmaf(e00, e00, s00);
                                s01 = fmaf(e01, e01, s01);
                                s10 = fmaf(e10, e10, s10);
                                s11 = fmaf(e11, e11, s11);
                            } else if constexpr (M == 1) {   // Manhattan: |e| summed
                                s00 += fabsf(e00);
                                s01 += fabsf(e01);
                                s10 += fabsf(e10);
                                s11 += fabsf(e11);
                            } else {   // Chebyshev: largest |e|
                                s00 = fmaxf(s00, fabsf(e00));
                                s01 = fmaxf(s01, fabsf(e01));
                                s10 = fmaxf(s10, fabsf(e10));
                                s11 = fmaxf(s11, fabsf(e11));
                            }
                        }
                    }
                }
                if ((s00 <= th0) | (s01 <= th0) | (s10 <= th1) | (s11 <= th1)) {
                    const uint32_t ja = (uint32_t)(j0 + c), jb = ja + 1;
                    consider(0, s00, ja);
                    consider(0, s01, jb);
                    consider(1, s10, ja);
                    consider(1, s11, jb);
                    th0 = COLLECT ? cthr[0] : sel[0].thr;
                    th1 = COLLECT ? cthr[1] : sel[1].thr;
                }
            }
        };
        if (a.metric == 1) columns(std::integral_constant<int, 1>{});
        else if (a.metric == 2) columns(std::integral_constant<int, 2>{});
        else columns(std::integral_constant<int, 0>{});
        if (!COLLECT && a.splits > 1) {
#pragma unroll
            for (int r = 0; r < 2; ++r)
                if (valid[r]) sel[r].bound(shared_thr_exchange(&a.slot_thr[slot[r]], sel[r].thr));
            th0 = sel[0].thr;
            th1 = sel[1].thr;
        }
        if (a.prune) publish(th0, th1);
        else __syncthreads();
        tile = nxt;
        buf ^= 1;
        ++swept;
    }
    if (t == 0 && a.st_tiles) {
        atomicAdd(&a.st_tiles[0], (unsigned long long)(ntiles - swept));
        atomicAdd(&a.st_tiles[1], (unsigned long long)swept);
    }

    if (!COLLECT) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!valid[r]) continue;
            const int64_t rec = slot[r] * a.splits + split;
            sel[r].write(a.out_v + rec * kListC, a.out_j + rec * kListC, a.out_ovf + rec, band_v + t + r * kThreads,
                         band_j + t + r * kThreads, kRowTile);
        }
    }
}

template <int D>
cudaError_t launch_d(const SweepArgs &a, bool collect, cudaStream_t s)
{
    dim3 grid((unsigned)((a.nslots + kRowTile - 1) / kRowTile), (unsigned)a.splits);
    const size_t dsm = (size_t)kBand * kRowTile * 8;
    cudaError_t e = cudaSuccess;
#define NNM_GO(KC_, COLL_)                                                                                  \
    do {                                                                                                    \
        e = cudaFuncSetAttribute(k_sweep_fp32<D, KC_, COLL_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)dsm);                                                                 \
        if (e != cudaSuccess) return e;                                                                     \
        k_sweep_fp32<D, KC_, COLL_><<<grid, kThreads, dsm, s>>>(a);                                          \
    } while (0)
    if (collect) NNM_GO(1, true);
    else if (a.kc <= 1) NNM_GO(1, false);
    else if (a.kc <= 2) NNM_GO(2, false);
    else if (a.kc <= 4) NNM_GO(4, false);
    else if (a.kc <= 8) NNM_GO(8, false);
    else NNM_GO(16, false);
#undef NNM_GO
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

// One width D per translation unit (this file is compiled once per D, with
// -DNNM_SWEEP_FP32_D=D, so that the instantiations compile in parallel); the dispatcher
// lives in the D = 32 unit.
cudaError_t launch_sweep_fp32_d4(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d8(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d12(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d16(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d20(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d24(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d25(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d28(const SweepArgs &a, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_d32(const SweepArgs &a, bool collect, cudaStream_t s);

#ifdef NNM_SWEEP_FP32_D
#define NNM_FP32_UNIT_NAME2(x) launch_sweep_fp32_d##x
#define NNM_FP32_UNIT_NAME(x) NNM_FP32_UNIT_NAME2(x)
cudaError_t NNM_FP32_UNIT_NAME(NNM_SWEEP_FP32_D)(const SweepArgs &a, bool collect, cudaStream_t s)
{
    return launch_d<NNM_SWEEP_FP32_D>(a, collect, s);
}
#undef NNM_FP32_UNIT_NAME
#undef NNM_FP32_UNIT_NAME2

#if NNM_SWEEP_FP32_D == 32
cudaError_t launch_sweep_fp32(const SweepArgs &a, int d, bool collect, cudaStream_t s)
{
    if (d <= 4) return launch_sweep_fp32_d4(a, collect, s);
    if (d <= 8) return launch_sweep_fp32_d8(a, collect, s);
    if (d <= 12) return launch_sweep_fp32_d12(a, collect, s);
    if (d <= 16) return launch_sweep_fp32_d16(a, collect, s);
    if (d <= 20) return launch_sweep_fp32_d20(a, collect, s);
    if (d <= 24) return launch_sweep_fp32_d24(a, collect, s);
    if (d == 25) return launch_sweep_fp32_d25(a, collect, s);
    if (d <= 28) return launch_sweep_fp32_d28(a, collect, s);
    return launch_sweep_fp32_d32(a, collect, s);
}
#endif
#endif

}  // namespace nnm
