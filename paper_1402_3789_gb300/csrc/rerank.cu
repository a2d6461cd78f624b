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
// threshold T such that every column of the exact top k has v <= T (in FP32 rounded
// upwards: the sweeps' own bound of select.cuh, which dominates the binary64 bound of
// the error analysis; a larger T only keeps more).  Each column range
// of the sweep kept every eligible value <= its own running bound, which is >= T,
// unless its band overflowed; a row with an overflowed range goes to the collect pass
// (every eligible column with v <= T) instead.
#include "nnm_internal.cuh"
#include "select.cuh"

namespace nnm {

namespace {

constexpr int kFinWarps = 4;

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v)
{
    if (p) atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// Selections compare keys as integers: the bits of a non-negative double (or float)
// order like the value, and the FP64 pipe, slow on this GPU, is kept for the distances.
constexpr long long kInfD = 0x7FF0000000000000LL;   // bits of +inf (double)
constexpr long long kInfF = 0x7F800000LL;           // bits of +inf (float)
constexpr long long kNone = kInfF + 1;              // a float-key slot without a candidate
constexpr long long kTaken = 1LL << 62;             // mark of an extracted float key

__device__ __forceinline__ long long dkey(double x) { return __double_as_longlong(x); }

struct Best {
    long long key;
    uint32_t j;
    int e;
};

__device__ __forceinline__ bool less_kj(long long k1, uint32_t j1, long long k2, uint32_t j2)
{
    return k1 < k2 || (k1 == k2 && j1 < j2);
}

__device__ __forceinline__ Best warp_min(Best b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best c;
        c.key = __shfl_xor_sync(0xffffffffu, b.key, o);
        c.j = __shfl_xor_sync(0xffffffffu, b.j, o);
        c.e = __shfl_xor_sync(0xffffffffu, b.e, o);
        if (less_kj(c.key, c.j, b.key, b.j)) b = c;
    }
    return b;
}

// k-th smallest of n float keys held as integers in kk (entries >= lim are ignored;
// ties by position).  Extracted entries are marked and restored afterwards.  Returns
// the value (+inf if fewer than k) and the number found.
__device__ float kth_float(long long *kk, int n, int k, int *found)
{
    const int lane = threadIdx.x & 31;
    int taken = 0;
    long long vk = kInfF;
    for (int m = 0; m < k; ++m) {
        Best b = {kInfF, kInvalid, -1};
        for (int e = lane; e < n; e += 32)
            if (kk[e] < kInfF && less_kj(kk[e], (uint32_t)e, b.key, b.j)) b = {kk[e], (uint32_t)e, e};
        b = warp_min(b);
        if (b.e < 0) break;
        vk = b.key;
        ++taken;
        if (lane == 0) kk[b.e] |= kTaken;
        __syncwarp();
    }
    for (int e = lane; e < n; e += 32) kk[e] &= ~kTaken;
    __syncwarp();
    *found = taken;
    return __int_as_float((int)vk);
}

// Pick the k smallest (D, j) of n entries held in (wD, wj) -- consumed entries get
// D = +inf -- and write them to the row's result slots.
__device__ void select_topk(double *wD, uint32_t *wj, int n, int k, int stride, uint32_t i, uint32_t *res_j,
                           double *res_D, int *n_out)
{
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    for (int m = 0; m < k; ++m) {
        Best b = {kInfD, kInvalid, -1};
        for (int e = lane; e < n; e += 32) {
            const long long kd = dkey(wD[e]);
            if (kd < kInfD && less_kj(kd, wj[e], b.key, b.j)) b = {kd, wj[e], e};
        }
        b = warp_min(b);
        if (lane == 0) {
            res_j[(int64_t)i * stride + m] = b.j;
            res_D[(int64_t)i * stride + m] = __longlong_as_double(b.key);
        }
        if (b.e < 0) continue;
        ++cnt;
        if (lane == 0) wD[b.e] = INFINITY;
        __syncwarp();
    }
    *n_out = cnt;
}

// FP32 direct value of D, features in order, as the FP32 sweep computes it: one FMA per
// feature for the squared Euclidean distance, a sum of |e| for Manhattan, a running
// max of |e| for Chebyshev (|s - exact| <= gamma32*s + alpha32 in every case).
__device__ __forceinline__ float fp32_D(const float *__restrict__ xi, const float *__restrict__ xj, int d, int metric)
{
    float s = 0.0f;
    if (metric == 1) {
        for (int k = 0; k < d; ++k) s += fabsf(xi[k] - xj[k]);
    } else if (metric == 2) {
        for (int k = 0; k < d; ++k) s = fmaxf(s, fabsf(xi[k] - xj[k]));
    } else {
        for (int k = 0; k < d; ++k) {
            const float e = xi[k] - xj[k];
            s = fmaf(e, e, s);
        }
    }
    return s;
}

// Per-warp shared scratch of exact_distances: the products of up to 32 candidates
// (row stride d rounded up to odd: no bank conflicts) and their column / entry indices.
__host__ __device__ inline int ed_stride(int d) { return d | 1; }
__host__ __device__ inline size_t ed_scratch_bytes(int d) { return (size_t)32 * ed_stride(d) * 8 + 64 * 4; }

// Exact distances of the candidates in wD (entries 0, others +inf) of one row, cheapest
// first: with refine, every candidate first gets its FP32 direct value s; from the k-th
// smallest s the FP32 bound T32 (as for the FP32 sweep, rounded up) keeps only the
// candidates that can still be among the exact k nearest, and only those get the
// binary64 distance.  The binary64 work is canon_D's, operation for operation and in the
// same order, with the lanes kept busy: for the marked entries of each run of 32, the
// products (or absolute differences) of all (candidate, feature) pairs are spread over
// the lanes, then one lane per candidate sums (or takes the max of) them in feature
// order.  On return wD[e] = D (binary64) or +inf.  Returns the number of binary64
// evaluations.
__device__ int exact_distances(const float *xi, const float *X, int d, double *wD, const uint32_t *wj, int n, int k,
                               const SelConst &sc, int metric, bool refine, uint8_t *scratch)
{
    const int lane = threadIdx.x & 31;
    long long *kk = reinterpret_cast<long long *>(wD);
    if (refine) {
        // float keys of s in place of the marks (+inf keys for non-candidates)
        for (int e = lane; e < n; e += 32)
            kk[e] = kk[e] < kInfD ? (long long)__float_as_int(fp32_D(xi, X + (int64_t)wj[e] * d, d, metric)) : kNone;
        __syncwarp();
        int taken = 0;
        const float vk = kth_float(kk, n, k, &taken);
        const float t32 = taken == k ? __fadd_ru(__fmul_ru(__fadd_ru(vk, sc.c0_32), sc.c1_32), sc.c0_32) : INFINITY;
        const long long lim = (long long)__float_as_int(t32);   // +inf: every candidate
        for (int e = lane; e < n; e += 32) kk[e] = kk[e] <= lim ? 0LL : kInfD;   // back to marks
        __syncwarp();
    }
    const int stride = ed_stride(d);
    double *tsm = reinterpret_cast<double *>(scratch);
    uint32_t *cj = reinterpret_cast<uint32_t *>(scratch + (size_t)32 * stride * 8);   // [32] columns, [32] entries
    int nd = 0;
    for (int base = 0; base < n; base += 32) {
        const int e = base + lane;
        const bool mk = e < n && kk[e] == 0LL;
        const unsigned int bm = __ballot_sync(0xffffffffu, mk);
        const int nb = __popc(bm);
        if (mk) {
            const int slot = __popc(bm & ((1u << lane) - 1u));
            cj[slot] = wj[e];
            cj[32 + slot] = (uint32_t)e;
        } else if (e < n) {
            wD[e] = INFINITY;
        }
        __syncwarp();
        // (candidate c, feature f) of the lane's pairs q = lane, lane + 32, ...: stepped
        // rather than divided (d is a run-time value)
        int c = 0, f = lane;
        while (f >= d) {
            f -= d;
            ++c;
        }
        for (int q = lane; q < nb * d; q += 32) {
            const double ev = __dsub_rn((double)xi[f], (double)X[(int64_t)cj[c] * d + f]);
            tsm[c * stride + f] = metric == 0 ? __dmul_rn(ev, ev) : fabs(ev);
            f += 32;
            while (f >= d) {
                f -= d;
                ++c;
            }
        }
        __syncwarp();
        if (lane < nb) {
            const double *t = tsm + lane * stride;
            double D = t[0];
            for (int f = 1; f < d; ++f) D = metric == 2 ? fmax(D, t[f]) : __dadd_rn(D, t[f]);
            wD[cj[32 + lane]] = D;
        }
        nd += nb;
        __syncwarp();
    }
    return nd;
}

__global__ void __launch_bounds__(kFinWarps * 32) k_finalize(const FinalizeArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_ent = a.splits * kListC;
    double *wD = reinterpret_cast<double *>(smem) + (size_t)warp * n_ent;
    float *wv = reinterpret_cast<float *>(reinterpret_cast<double *>(smem) + (size_t)kFinWarps * n_ent) +
                (size_t)warp * n_ent;
    uint32_t *wj_all = reinterpret_cast<uint32_t *>(reinterpret_cast<float *>(reinterpret_cast<double *>(smem) +
                                                                              (size_t)kFinWarps * n_ent) +
                                                    (size_t)kFinWarps * n_ent);
    uint32_t *wj = wj_all + (size_t)warp * n_ent;
    const int64_t q = (int64_t)blockIdx.x * kFinWarps + warp;
    if (q >= a.nslots) return;
    const uint32_t ipos = a.rows ? a.rows[q] : (uint32_t)q;
    const uint32_t i = a.pos2row[ipos];
    const float *vin = a.in_v + q * n_ent;
    const uint32_t *jin = a.in_j + q * n_ent;
    long long *kk = reinterpret_cast<long long *>(wD);
    for (int e = lane; e < n_ent; e += 32) {
        const uint32_t j = jin[e];   // a position; from here on original row indices
        const float v = vin[e];
        wv[e] = v;
        wj[e] = j != kInvalid ? a.pos2row[j] : kInvalid;
        // candidate values are >= 0 except the tensor path's small negative rounding:
        // the key is clamped at +0 (a larger k-th value only keeps more)
        kk[e] = j != kInvalid ? (long long)__float_as_int(v > 0.0f ? v : 0.0f) : kNone;
    }
    const bool ovf = lane < a.splits && a.in_ovf[q * a.splits + lane];
    __syncwarp();
    // k-th smallest value over all records
    int taken = 0;
    const float vk = kth_float(kk, n_ent, a.k, &taken);
    // a bounded row needs only columns with D <= B: their candidate values are at most
    // the threshold of the value B (in candidate units)
    const double B = a.row_B ? a.row_B[i] : INFINITY;
    const RowConst rc = make_rowconst(a.sc, a.m, i);
    float T = sel_threshold(a.sc, rc, taken < a.k ? INFINITY : vk);
    if (B < INFINITY) T = fminf(T, sel_threshold(a.sc, rc, __double2float_ru(B / a.m.inv_scale2)));
    const bool any_ovf = __any_sync(0xffffffffu, ovf);
    if (lane == 0) {
        a.ovf_flag[q] = any_ovf ? 1 : 0;
        if (any_ovf) a.ovf_thr[q] = T;
    }
    if (any_ovf) return;
    const float *xi = a.X + (int64_t)i * a.d;
    const float Tf = T;
    for (int e = lane; e < n_ent; e += 32) wD[e] = (wj[e] != kInvalid && wv[e] <= Tf) ? 0.0 : INFINITY;
    __syncwarp();
    uint8_t *scratch = reinterpret_cast<uint8_t *>(wj_all + (size_t)kFinWarps * n_ent) + (size_t)warp * ed_scratch_bytes(a.d);
    const int nc = exact_distances(xi, a.X, a.d, wD, wj, n_ent, a.k, a.sc, a.m.metric, a.m.tensor != 0, scratch);
    if (B < INFINITY) {
        const long long kb = dkey(B);
        for (int e = lane; e < n_ent; e += 32)
            if (dkey(wD[e]) > kb) wD[e] = INFINITY;
        __syncwarp();
    }
    double emax_abs = 0.0;
    float emax_rel = 0.0f;
    for (int e = lane; e < n_ent; e += 32) {
        const long long kd = dkey(wD[e]);
        if (kd < kInfD) {
            const double err = fabs((double)wv[e] * a.m.inv_scale2 - wD[e]);
            emax_abs = fmax(emax_abs, err);
            if (kd > 0) emax_rel = fmaxf(emax_rel, (float)err / (float)wD[e]);
        }
    }
    int n_out;
    select_topk(wD, wj, n_ent, a.k, a.res_stride, i, a.res_j, a.res_D, &n_out);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        emax_abs = fmax(emax_abs, __shfl_xor_sync(0xffffffffu, emax_abs, o));
        emax_rel = fmaxf(emax_rel, __shfl_xor_sync(0xffffffffu, emax_rel, o));
    }
    if (lane == 0) {
        if (a.res_n) a.res_n[i] = (uint8_t)n_out;
        // fewer than k results: every eligible column (unbounded row), or every eligible
        // column with D <= B (bounded row), is among them
        if (a.res_exh) a.res_exh[i] = n_out == a.k ? kCacheFull : (B < INFINITY ? kCacheBounded : kCacheAll);
        atomic_max_nonneg(a.st_max_abs, emax_abs);
        atomic_max_nonneg(a.st_max_rel, (double)emax_rel);
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
    extern __shared__ __align__(16) uint8_t cr_smem[];
    uint8_t *scratch = cr_smem + (size_t)warp * ed_scratch_bytes(a.d);
    const int nd = exact_distances(xi, a.X, a.d, wD, wj, (int)cnt, a.k, a.sc, a.m.metric, true, scratch);
    const double B = a.row_B ? a.row_B[i] : INFINITY;
    if (B < INFINITY)
        for (uint32_t e = lane; e < cnt; e += 32)
            if (dkey(wD[e]) > dkey(B)) wD[e] = INFINITY;
    __threadfence_block();
    int n_out;
    select_topk(wD, wj, (int)cnt, a.k, a.res_stride, i, a.res_j, a.res_D, &n_out);
    if (lane == 0) {
        if (a.res_n) a.res_n[i] = (uint8_t)n_out;
        if (a.res_exh) a.res_exh[i] = n_out == a.k ? kCacheFull : (B < INFINITY ? kCacheBounded : kCacheAll);
        if (a.st_pairs) atomicAdd(a.st_pairs, (unsigned long long)nd);
        if (a.st_max_cand) atomicMax(a.st_max_cand, (unsigned long long)cnt);
    }
}

}  // namespace

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t s)
{
    if (a.nslots <= 0) return cudaSuccess;
    const size_t smem = (size_t)kFinWarps * a.splits * kListC * (8 + 4 + 4) +   // <= 160 KB
                        (size_t)kFinWarps * ed_scratch_bytes(a.d);             // <= 35 KB
    cudaError_t e = set_max_dynamic_smem(k_finalize);
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
    k_collect_rerank<<<blocks, kFinWarps * 32, (size_t)kFinWarps * ed_scratch_bytes(a.d), s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnm
