// rerank.cu -- K3: exact binary64 re-rank of the sweep candidates.
//
// The paper selects the P pairs with the smallest distance and sorts them ("General
// description of the algorithm for constructing the set of minimum distances").  Here
// each row's candidates from the FP32 or tensor-core sweep are re-ranked with the exact
// squared distance of Eq. (1),
//     D(i,j) = ((t_0 + t_1) + ...) + t_{d-1},  t_k = e_k*e_k,  e_k = x_ik - x_jk,
// every operation IEEE binary64 round-to-nearest without contraction, and the k
// smallest (D, j) are kept.  Completeness: a candidate value v approximates the exact
// squared distance within a proven bound; from the k-th smallest v the re-rank derives a
// threshold T such that every column of the exact top k has v <= T.  Each column range
// of the sweep kept every eligible value <= its own running bound, which is >= T,
// unless its band overflowed; a row with an overflowed range goes to the collect pass
// (every eligible column with v <= T) instead.
#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr int kFinWarps = 4;

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v)
{
    if (p) atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// Threshold T from the k-th smallest candidate value vk (see the file comment).
__device__ double threshold(const Margin &m, uint32_t i, float vk)
{
    if (!(vk < INFINITY)) return INFINITY;
    const double grow = 1.0 + 1e-12;
    if (!m.tensor) {
        // FP32 direct: |v - s| <= gamma*s + alpha, s the exact squared distance
        const double us = ((double)vk + m.alpha) / (1.0 - m.gamma) * grow;
        return (us * (1.0 + m.gamma) + m.alpha) * grow;
    }
    // tensor core (scaled units): |v - |x_hat_i - x_hat_j|^2| <= eps_i and
    // | |x_hat_i - x_hat_j| - scale*sqrt(s) | <= r_i + r_j
    const double Pi = (double)m.P[i];
    const double eps = m.gamma * (Pi + m.Pmax) * (Pi + m.Pmax) + (double)m.E[i] + m.Emax;
    const double rr = (double)m.r[i] + m.R;
    const double U = (sqrt((double)vk + eps) + rr) * grow;
    return ((U + rr) * (U + rr) + eps) * grow;
}

struct Best {
    double D;
    uint32_t j;
    int e;
};

__device__ __forceinline__ bool less_dj(double D1, uint32_t j1, double D2, uint32_t j2)
{
    return D1 < D2 || (D1 == D2 && j1 < j2);
}

__device__ __forceinline__ Best warp_min(Best b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best c;
        c.D = __shfl_xor_sync(0xffffffffu, b.D, o);
        c.j = __shfl_xor_sync(0xffffffffu, b.j, o);
        c.e = __shfl_xor_sync(0xffffffffu, b.e, o);
        if (less_dj(c.D, c.j, b.D, b.j)) b = c;
    }
    return b;
}

// Pick the k smallest (D, j) of n entries held in (wD, wj) -- consumed entries get
// D = +inf -- and write them to the row's result slots.
__device__ void select_topk(double *wD, uint32_t *wj, int n, int k, uint32_t i, uint32_t *res_j,
                           double *res_D, int *n_out)
{
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int m = 0; m < k; ++m) {
        Best b = {INFINITY, kInvalid, -1};
        for (int e = lane; e < n; e += 32)
            if (wD[e] < INFINITY && less_dj(wD[e], wj[e], b.D, b.j)) b = {wD[e], wj[e], e};
        b = warp_min(b);
        if (lane == 0) {
            res_j[(int64_t)i * k + m] = b.j;
            res_D[(int64_t)i * k + m] = b.D;
        }
        if (b.e < 0) continue;
        ++cnt;
        if (lane == 0) wD[b.e] = INFINITY;
        __syncwarp();
    }
    *n_out = cnt;
}

// FP32 direct squared distance, one FMA per feature in order (|s - exact| <= gamma32*s + alpha32).
__device__ __forceinline__ float fp32_D(const float *__restrict__ xi, const float *__restrict__ xj, int d)
{
    float s = 0.0f;
    for (int k = 0; k < d; ++k) {
        const float e = xi[k] - xj[k];
        s = fmaf(e, e, s);
    }
    return s;
}

// Exact distances of the candidates in wD (entries < inf) of one row, cheapest first:
// with refine, every candidate first gets its FP32 direct value s; from the k-th
// smallest s the FP32 bound T32 (as for the FP32 sweep) keeps only the candidates that
// can still be among the exact k nearest, and only those get the binary64 distance.
// On return wD[e] = D (binary64) or +inf.  Returns the number of binary64 evaluations.
__device__ int exact_distances(const float *xi, const float *X, int d, double *wD, const uint32_t *wj, int n, int k,
                               const Margin &m, bool refine)
{
    const int lane = threadIdx.x & 31;
    double T32 = INFINITY;
    if (refine) {
        for (int e = lane; e < n; e += 32)
            if (wD[e] < INFINITY) wD[e] = (double)fp32_D(xi, X + (int64_t)wj[e] * d, d);
        __syncwarp();
        // k-th smallest s: extracted entries are marked by w -> -1 - w and restored after
        int taken = 0;
        double vk = INFINITY;
        for (int mth = 0; mth < k; ++mth) {
            Best b = {INFINITY, kInvalid, -1};
            for (int e = lane; e < n; e += 32)
                if (wD[e] >= 0.0 && wD[e] < INFINITY && less_dj(wD[e], (uint32_t)e, b.D, b.j)) b = {wD[e], (uint32_t)e, e};
            b = warp_min(b);
            if (b.e < 0) break;
            vk = b.D;
            ++taken;
            if (lane == 0) wD[b.e] = -1.0 - wD[b.e];
            __syncwarp();
        }
        for (int e = lane; e < n; e += 32)
            if (wD[e] < 0.0) wD[e] = -1.0 - wD[e];
        __syncwarp();
        if (taken == k) {
            const double grow = 1.0 + 1e-12;
            const double us = (vk + m.alpha32) / (1.0 - m.gamma32) * grow;
            T32 = (us * (1.0 + m.gamma32) + m.alpha32) * grow;
        }
    }
    int nd = 0;
    for (int e = lane; e < n; e += 32) {
        double D = INFINITY;
        if (wD[e] < INFINITY && wD[e] <= T32) {
            D = canon_D(xi, X + (int64_t)wj[e] * d, d);
            ++nd;
        }
        wD[e] = D;
    }
    __syncwarp();
    return __reduce_add_sync(0xffffffffu, nd);
}

__global__ void __launch_bounds__(kFinWarps * 32) k_finalize(const FinalizeArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_ent = a.splits * kListC;
    double *wD = reinterpret_cast<double *>(smem) + (size_t)warp * n_ent;
    float *wv = reinterpret_cast<float *>(reinterpret_cast<double *>(smem) + (size_t)kFinWarps * n_ent) +
                (size_t)warp * n_ent;
    uint32_t *wj = reinterpret_cast<uint32_t *>(reinterpret_cast<float *>(reinterpret_cast<double *>(smem) +
                                                                          (size_t)kFinWarps * n_ent) +
                                                (size_t)kFinWarps * n_ent) +
                   (size_t)warp * n_ent;
    const int64_t q = (int64_t)blockIdx.x * kFinWarps + warp;
    if (q >= a.nslots) return;
    const uint32_t ipos = a.rows ? a.rows[q] : (uint32_t)q;
    const uint32_t i = a.pos2row[ipos];
    const float *vin = a.in_v + q * n_ent;
    const uint32_t *jin = a.in_j + q * n_ent;
    for (int e = lane; e < n_ent; e += 32) {
        const uint32_t j = jin[e];   // a position; from here on original row indices
        const float v = vin[e];
        wv[e] = v;
        wj[e] = j != kInvalid ? a.pos2row[j] : kInvalid;
        wD[e] = j != kInvalid ? (double)v : INFINITY;
    }
    const bool ovf = lane < a.splits && a.in_ovf[q * a.splits + lane];
    __syncwarp();
    // k-th smallest value over all records (extraction on a scratch copy)
    int taken = 0;
    double vk = INFINITY;
    for (int m = 0; m < a.k; ++m) {
        Best b = {INFINITY, kInvalid, -1};
        for (int e = lane; e < n_ent; e += 32)
            if (wD[e] < INFINITY && less_dj(wD[e], (uint32_t)e, b.D, b.j)) b = {wD[e], (uint32_t)e, e};
        b = warp_min(b);
        if (b.e < 0) break;
        vk = b.D;
        ++taken;
        if (lane == 0) wD[b.e] = INFINITY;
        __syncwarp();
    }
    // a bounded row needs only columns with D <= B: their candidate values are at most
    // the threshold of the value B (in candidate units)
    const double B = a.row_B ? a.row_B[i] : INFINITY;
    double T = threshold(a.m, i, taken < a.k ? INFINITY : (float)vk);
    if (B < INFINITY) T = fmin(T, threshold(a.m, i, __double2float_ru(B / a.m.inv_scale2)));
    const bool any_ovf = __any_sync(0xffffffffu, ovf);
    if (lane == 0) {
        a.ovf_flag[q] = any_ovf ? 1 : 0;
        if (any_ovf) a.ovf_thr[q] = __double2float_ru(T);
    }
    if (any_ovf) return;
    const float *xi = a.X + (int64_t)i * a.d;
    for (int e = lane; e < n_ent; e += 32) wD[e] = (wj[e] != kInvalid && (double)wv[e] <= T) ? 0.0 : INFINITY;
    __syncwarp();
    const int nc = exact_distances(xi, a.X, a.d, wD, wj, n_ent, a.k, a.m, a.m.tensor != 0);
    if (B < INFINITY) {
        for (int e = lane; e < n_ent; e += 32)
            if (wD[e] > B) wD[e] = INFINITY;
        __syncwarp();
    }
    double emax_abs = 0.0, emax_rel = 0.0;
    for (int e = lane; e < n_ent; e += 32) {
        if (wD[e] < INFINITY) {
            const double err = fabs((double)wv[e] * a.m.inv_scale2 - wD[e]);
            emax_abs = fmax(emax_abs, err);
            if (wD[e] > 0.0) emax_rel = fmax(emax_rel, err / wD[e]);
        }
    }
    int n_out;
    select_topk(wD, wj, n_ent, a.k, i, a.res_j, a.res_D, &n_out);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        emax_abs = fmax(emax_abs, __shfl_xor_sync(0xffffffffu, emax_abs, o));
        emax_rel = fmax(emax_rel, __shfl_xor_sync(0xffffffffu, emax_rel, o));
    }
    if (lane == 0) {
        if (a.res_n) a.res_n[i] = (uint8_t)n_out;
        // fewer than k results from an unbounded row means every eligible column was
        // among the candidates
        if (a.res_exh) a.res_exh[i] = (uint8_t)(n_out < a.k && !(B < INFINITY));
        atomic_max_nonneg(a.st_max_abs, emax_abs);
        atomic_max_nonneg(a.st_max_rel, emax_rel);
        if (a.st_pairs) atomicAdd(a.st_pairs, (unsigned long long)nc);
        if (a.st_max_cand) atomicMax(a.st_max_cand, (unsigned long long)nc);
    }
}

__global__ void __launch_bounds__(kFinWarps * 32) k_collect_rerank(const CollectRerankArgs a)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kFinWarps + warp;
    if (p >= a.n) return;
    const uint32_t i = a.pos2row[a.rows[p]];
    const uint32_t cnt = a.coll_cnt[p];
    const bool heavy = (int64_t)cnt > a.cap;
    if (lane == 0) a.heavy_flag[a.heavy_base + p] = heavy ? 1 : 0;
    if (heavy) {
        // too many for this pass's capacity: the count is exact, the host re-runs the
        // row with room for all of them
        if (lane == 0) {
            atomicExch(a.retry_flag, 1);
            atomicMax(a.heavy_max, (unsigned long long)cnt);
        }
        return;
    }
    const float *xi = a.X + (int64_t)i * a.d;
    double *wD = a.scratch_D + p * a.cap;
    uint32_t *wj = const_cast<uint32_t *>(a.coll_j) + p * a.cap;
    for (uint32_t e = lane; e < cnt; e += 32) {
        wj[e] = a.pos2row[wj[e]];   // positions -> original row indices
        wD[e] = 0.0;
    }
    __syncwarp();
    __threadfence_block();
    const int nd = exact_distances(xi, a.X, a.d, wD, wj, (int)cnt, a.k, a.m, true);
    const double B = a.row_B ? a.row_B[i] : INFINITY;
    if (B < INFINITY)
        for (uint32_t e = lane; e < cnt; e += 32)
            if (wD[e] > B) wD[e] = INFINITY;
    __threadfence_block();
    int n_out;
    select_topk(wD, wj, (int)cnt, a.k, i, a.res_j, a.res_D, &n_out);
    if (lane == 0) {
        if (a.res_n) a.res_n[i] = (uint8_t)n_out;
        if (a.res_exh) a.res_exh[i] = (uint8_t)((int)cnt < a.k && !(B < INFINITY));
        if (a.st_pairs) atomicAdd(a.st_pairs, (unsigned long long)nd);
        if (a.st_max_cand) atomicMax(a.st_max_cand, (unsigned long long)cnt);
    }
}

}  // namespace

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s)
{
    if (a.nslots <= 0) return cudaSuccess;
    const size_t smem = (size_t)kFinWarps * a.splits * kListC * (8 + 4 + 4);   // <= 160 KB
    cudaError_t e = cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((a.nslots + kFinWarps - 1) / kFinWarps);
    k_finalize<<<blocks, kFinWarps * 32, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_collect_rerank(const CollectRerankArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((a.n + kFinWarps - 1) / kFinWarps);
    k_collect_rerank<<<blocks, kFinWarps * 32, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnm
