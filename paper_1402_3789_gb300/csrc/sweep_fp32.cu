// sweep_fp32.cu -- K1: all-pairs candidate sweep with FP32 direct differences.
//
// The second and third parallel items of the paper ("Overall idea of the algorithm":
// distances between all pairs, then selection of the minimum distances) fused into
// one pass over row tile x column range, the "two logical blocks of data" of the
// paper's pair construction.  Each thread owns two rows (registers), columns stream
// through shared memory (cp.async, double buffered), and the candidate value
//     s~(i,j) = fl32( sum_k (x_ik - x_jk)^2 ),   summed k = 0..d-1 with one FMA per k,
// is compared against the row's running threshold.  Only values below it reach the
// slow path, which checks eligibility (j != i, j inside the range, and with a mask
// comp[j] != comp[i]) and then either inserts into the row's sorted top-C list kept
// in registers, or, in collect mode, appends j to the row's global segment.
//
// Error bound used by the re-rank: |s~ - s| <= gamma_{d+2} * s (u = 2^-24) plus an
// underflow term, s the exact squared distance of the FP32 inputs.
#include <cuda_pipeline_primitives.h>

#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr int kThreads = 128;
constexpr int kTile = 64;   // columns per shared-memory tile

// Insert (v, j) into the ascending list (lv, lj); the largest entry falls out.
template <int C>
__device__ __forceinline__ void list_insert(float (&lv)[C], uint32_t (&lj)[C], float v, uint32_t j)
{
#pragma unroll
    for (int m = 0; m < C; ++m) {
        bool sw = v < lv[m];
        float tv = sw ? lv[m] : v;
        uint32_t tj = sw ? lj[m] : j;
        lv[m] = sw ? v : lv[m];
        lj[m] = sw ? j : lj[m];
        v = tv;
        j = tj;
    }
}

template <int D, bool COLLECT>
__global__ void __launch_bounds__(kThreads, 2) k_sweep_fp32(const SweepArgs a)
{
    constexpr int C = kListC;
    constexpr int DP = (D + 3) & ~3;
    __shared__ __align__(16) float sy[2][kTile * DP];

    const int t = threadIdx.x;
    const int64_t slot[2] = {(int64_t)blockIdx.x * kRowTile + t, (int64_t)blockIdx.x * kRowTile + t + kThreads};
    bool valid[2];
    uint32_t row[2], crow[2];
    float x[2][D];
    float thr[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        valid[r] = slot[r] < a.nslots;
        row[r] = valid[r] ? (a.rows ? a.rows[slot[r]] : (uint32_t)slot[r]) : 0u;
        crow[r] = (valid[r] && a.comp) ? a.comp[row[r]] : 0u;
        const float *xr = a.Xs + (int64_t)row[r] * DP;
#pragma unroll
        for (int k = 0; k < D; ++k) x[r][k] = xr[k];
        if (COLLECT) thr[r] = valid[r] ? a.thr[slot[r]] : -INFINITY;
        else thr[r] = valid[r] ? INFINITY : -INFINITY;
    }
    float lv[2][C];
    uint32_t lj[2][C];
    if (!COLLECT) {
#pragma unroll
        for (int m = 0; m < C; ++m) {
            lv[0][m] = INFINITY;
            lv[1][m] = INFINITY;
            lj[0][m] = kInvalid;
            lj[1][m] = kInvalid;
        }
    }

    const int split = blockIdx.y;
    const int64_t cb = a.col_begin + (int64_t)split * a.cols_per_split;
    int64_t ce = cb + a.cols_per_split;
    if (ce > a.col_end) ce = a.col_end;
    const int64_t ntiles = ce > cb ? (ce - cb + kTile - 1) / kTile : 0;

    auto load_tile = [&](int64_t tile, int buf) {
        const int64_t j0 = cb + tile * kTile;
        int64_t n = ce - j0;
        if (n > kTile) n = kTile;
        const int chunks = (int)n * (DP / 4);
        const float *src = a.Xs + j0 * DP;
        for (int q = t; q < chunks; q += kThreads)
            __pipeline_memcpy_async(&sy[buf][q * 4], src + q * 4, 16);
    };

    auto consider = [&](int r, float v, uint32_t j) {
        if ((int64_t)j >= ce || j == row[r]) return;
        if (a.comp && a.comp[j] == crow[r]) return;
        if (COLLECT) {
            if (!(v <= thr[r])) return;
            uint32_t p = atomicAdd(&a.coll_cnt[slot[r]], 1u);
            if ((int64_t)p < a.coll_cap) a.coll_j[slot[r] * a.coll_cap + p] = j;
        } else {
            if (!(v < thr[r])) return;
            if (r == 0) {
                list_insert<C>(lv[0], lj[0], v, j);
                thr[0] = lv[0][C - 1];
            } else {
                list_insert<C>(lv[1], lj[1], v, j);
                thr[1] = lv[1][C - 1];
            }
        }
    };

    if (ntiles > 0) load_tile(0, 0);
    __pipeline_commit();
    for (int64_t tile = 0; tile < ntiles; ++tile) {
        if (tile + 1 < ntiles) load_tile(tile + 1, (int)((tile + 1) & 1));
        __pipeline_commit();
        __pipeline_wait_prior(1);
        __syncthreads();
        const float *ys = sy[tile & 1];
        const int64_t j0 = cb + tile * kTile;
        int n = (int)(ce - j0 < kTile ? ce - j0 : kTile);
        for (int c = 0; c < n; c += 2) {
            const float4 *ya = reinterpret_cast<const float4 *>(ys + c * DP);
            const float4 *yb = reinterpret_cast<const float4 *>(ys + (c + 1) * DP);
            float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f;
#pragma unroll
            for (int q = 0; q < DP / 4; ++q) {
                float4 A = ya[q], B = yb[q];
                float av[4] = {A.x, A.y, A.z, A.w};
                float bv[4] = {B.x, B.y, B.z, B.w};
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int k = q * 4 + w;
                    if (k < D) {
                        float e;
                        e = x[0][k] - av[w];
                        s00 = fmaf(e, e, s00);
                        e = x[0][k] - bv[w];
                        s01 = fmaf(e, e, s01);
                        e = x[1][k] - av[w];
                        s10 = fmaf(e, e, s10);
                        e = x[1][k] - bv[w];
                        s11 = fmaf(e, e, s11);
                    }
                }
            }
            bool hit;
            if (COLLECT) hit = (s00 <= thr[0]) | (s01 <= thr[0]) | (s10 <= thr[1]) | (s11 <= thr[1]);
            else hit = (s00 < thr[0]) | (s01 < thr[0]) | (s10 < thr[1]) | (s11 < thr[1]);
            if (hit) {
                const uint32_t ja = (uint32_t)(j0 + c), jb = ja + 1;
                consider(0, s00, ja);
                consider(0, s01, jb);
                consider(1, s10, ja);
                consider(1, s11, jb);
            }
        }
        __syncthreads();
    }

    if (!COLLECT) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!valid[r]) continue;
            int64_t base = (slot[r] * a.splits + split) * C;
#pragma unroll
            for (int m = 0; m < C; ++m) {
                a.out_v[base + m] = lv[r][m];
                a.out_j[base + m] = lj[r][m];
            }
        }
    }
}

template <int D>
cudaError_t launch_d(const SweepArgs &a, bool collect, cudaStream_t s)
{
    dim3 grid((unsigned)((a.nslots + kRowTile - 1) / kRowTile), (unsigned)a.splits);
    if (collect) k_sweep_fp32<D, true><<<grid, kThreads, 0, s>>>(a);
    else k_sweep_fp32<D, false><<<grid, kThreads, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

// one half of the instantiations per translation unit (compiled twice)
cudaError_t launch_sweep_fp32_lo(const SweepArgs &a, int d, bool collect, cudaStream_t s);
cudaError_t launch_sweep_fp32_hi(const SweepArgs &a, int d, bool collect, cudaStream_t s);

#ifdef NNM_SWEEP_FP32_LO
cudaError_t launch_sweep_fp32_lo(const SweepArgs &a, int d, bool collect, cudaStream_t s)
{
    switch (d) {
#define NNM_CASE(D) case D: return launch_d<D>(a, collect, s);
        NNM_CASE(1) NNM_CASE(2) NNM_CASE(3) NNM_CASE(4) NNM_CASE(5) NNM_CASE(6) NNM_CASE(7) NNM_CASE(8)
        NNM_CASE(9) NNM_CASE(10) NNM_CASE(11) NNM_CASE(12) NNM_CASE(13) NNM_CASE(14) NNM_CASE(15) NNM_CASE(16)
#undef NNM_CASE
    default: return cudaErrorInvalidValue;
    }
}
#endif

#ifdef NNM_SWEEP_FP32_HI
cudaError_t launch_sweep_fp32_hi(const SweepArgs &a, int d, bool collect, cudaStream_t s)
{
    switch (d) {
#define NNM_CASE(D) case D: return launch_d<D>(a, collect, s);
        NNM_CASE(17) NNM_CASE(18) NNM_CASE(19) NNM_CASE(20) NNM_CASE(21) NNM_CASE(22) NNM_CASE(23) NNM_CASE(24)
        NNM_CASE(25) NNM_CASE(26) NNM_CASE(27) NNM_CASE(28) NNM_CASE(29) NNM_CASE(30) NNM_CASE(31) NNM_CASE(32)
#undef NNM_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep_fp32(const SweepArgs &a, int d, bool collect, cudaStream_t s)
{
    return d <= 16 ? launch_sweep_fp32_lo(a, d, collect, s) : launch_sweep_fp32_hi(a, d, collect, s);
}
#endif

}  // namespace nnm
