// prep.cu -- K0: checks and operand preparation for the candidate sweeps.
//
// The paper's main module checks the data array and fills auxiliary working fields
// ("Objectives of the main module"); here that is: reject non-finite values, build the
// padded FP32 copy for the direct-difference sweep, and, for the tensor-core sweeps,
// the centred, scaled, rounded operands with the per-row bounds that make the later
// exact re-rank provably complete.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nnm_internal.cuh"

namespace nnm {

__global__ void k_check_finite(const float *__restrict__ X, int64_t n, int *flag)
{
    int bad = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(X[q]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_check_finite(const float *X, int64_t n, int *flag, cudaStream_t s)
{
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_check_finite<<<blocks, 256, 0, s>>>(X, n, flag);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Spatial order of the rows.  The sweeps read operands in an order where rows that are
// close in space are close in memory, so that a row tile meets its near neighbours in
// its first column tiles and far tiles can be bounded as a whole.
//   - Landmarks: L rows taken at regular strides; every row joins the group of its
//     nearest landmark.
//   - Groups are ordered along a greedy nearest-neighbour chain through S <= 1024 coarse
//     landmarks (also regular strides): a landmark follows the chain rank of its nearest
//     coarse landmark, then its distance to it.
//   - Within a group rows follow their distance to the landmark, then their index.
//   - Rows much farther from their landmark than is typical (squared distance above 9
//     times the median) are isolated points: they go, in the same order, after all
//     other rows, so that they do not widen the tiles of the dense groups.
// The order only affects speed: every decision uses original indices and the exact
// binary64 distance.
// ---------------------------------------------------------------------------------
constexpr int kLandChunk = 128;
constexpr int kMaxLandmarks = 1024;

// Order of the coarse landmarks: a greedy nearest-neighbour chain (start at landmark 0,
// always step to the nearest unvisited one).  One CTA; landmark m is row m*N/L.
__global__ void __launch_bounds__(kMaxLandmarks) k_landmark_chain(const float *__restrict__ X, int64_t N, int d,
                                                                  int L, uint32_t *__restrict__ rank)
{
    extern __shared__ float lmk[];   // [L][d]
    __shared__ float wbest[kMaxLandmarks / 32];
    __shared__ int warg[kMaxLandmarks / 32];
    __shared__ int cur_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int q = t; q < L * d; q += blockDim.x) lmk[q] = X[((int64_t)(q / d) * N / L) * d + q % d];
    bool visited = t >= L;
    if (t == 0) cur_s = 0;
    __syncthreads();
    for (int step = 0; step < L; ++step) {
        const int cur = cur_s;
        if (t == cur) {
            rank[cur] = (uint32_t)step;
            visited = true;
        }
        float v = INFINITY;
        if (!visited) {
            float acc = 0.0f;
            for (int k = 0; k < d; ++k) {
                const float e = lmk[t * d + k] - lmk[cur * d + k];
                acc = fmaf(e, e, acc);
            }
            v = acc;
        }
        int arg = t;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ov < v || (ov == v && oa < arg)) {
                v = ov;
                arg = oa;
            }
        }
        if (lane == 0) {
            wbest[w] = v;
            warg[w] = arg;
        }
        __syncthreads();
        if (t == 0) {
            float bv = INFINITY;
            int ba = 0;
            for (int q = 0; q < (int)(blockDim.x / 32); ++q)
                if (wbest[q] < bv || (wbest[q] == bv && warg[q] < ba)) {
                    bv = wbest[q];
                    ba = warg[q];
                }
            cur_s = ba;
        }
        __syncthreads();
    }
}

cudaError_t launch_landmark_chain(const float *X, int64_t N, int d, int64_t L, uint32_t *rank, cudaStream_t s)
{
    const size_t smem = (size_t)L * d * sizeof(float);
    cudaError_t e = set_max_dynamic_smem(k_landmark_chain);
    if (e != cudaSuccess) return e;
    k_landmark_chain<<<1, kMaxLandmarks, smem, s>>>(X, N, d, (int)L, rank);
    count_launches(1);
    return cudaGetLastError();
}

// For each query q < Q (row q*N/Q of X) the nearest of the R reference rows (row r*N/R)
// by FP32 squared distance (first one on ties): index and value.  Features are summed in
// order with one FMA each; DP = d rounded up to 4 (the padding adds 0 * 0, which changes
// no sum).  Each thread takes two queries, so every float4 of a reference row read from
// shared memory feeds eight FMAs.
template <int DP, int DC = DP>   // DP: padded width (float4 loads), DC: features summed (DC <= DP)
__global__ void __launch_bounds__(256) k_nearest_ref(const float *__restrict__ X, int64_t N, int d, int64_t Q,
                                                     int64_t R, uint32_t *__restrict__ arg_out,
                                                     float *__restrict__ dist_out)
{
    __shared__ __align__(16) float lm[kLandChunk * DP];
    __shared__ int64_t lrow[kLandChunk];   // the chunk's landmark rows
    const int64_t qa = (int64_t)blockIdx.x * 512 + threadIdx.x, qb = qa + 256;
    const int64_t ra = qa < Q ? qa * N / Q : 0, rb = qb < Q ? qb * N / Q : 0;
    float xa[DP], xb[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
        xa[k] = k < d ? X[ra * d + k] : 0.0f;
        xb[k] = k < d ? X[rb * d + k] : 0.0f;
    }
    float besta = INFINITY, bestb = INFINITY;
    int64_t arga = 0, argb = 0;
    for (int64_t m0 = 0; m0 < R; m0 += kLandChunk) {
        __syncthreads();
        if (threadIdx.x < kLandChunk) lrow[threadIdx.x] = (m0 + threadIdx.x) * N / R;   // one division per landmark
        __syncthreads();
        for (int t = threadIdx.x; t < kLandChunk * DP; t += blockDim.x) {
            const int64_t m = m0 + t / DP;
            const int k = t % DP;
            lm[t] = (m < R && k < d) ? X[lrow[t / DP] * d + k] : 0.0f;
        }
        __syncthreads();
        const int cnt = (int)(R - m0 < kLandChunk ? R - m0 : kLandChunk);
        for (int m = 0; m < cnt; ++m) {
            const float4 *l4 = reinterpret_cast<const float4 *>(lm + m * DP);
            float acca = 0.0f, accb = 0.0f;
#pragma unroll
            for (int k4 = 0; k4 < DP / 4; ++k4) {
                const float4 v = l4[k4];
                const float l[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (4 * k4 + j >= DC) continue;   // zero padding: would add +0 exactly
                    const float ea = xa[4 * k4 + j] - l[j], eb = xb[4 * k4 + j] - l[j];
                    acca = fmaf(ea, ea, acca);
                    accb = fmaf(eb, eb, accb);
                }
            }
            if (acca < besta) {
                besta = acca;
                arga = m0 + m;
            }
            if (accb < bestb) {
                bestb = accb;
                argb = m0 + m;
            }
        }
    }
    if (qa < Q) {
        arg_out[qa] = (uint32_t)arga;
        dist_out[qa] = besta;
    }
    if (qb < Q) {
        arg_out[qb] = (uint32_t)argb;
        dist_out[qb] = bestb;
    }
}

cudaError_t launch_nearest_ref(const float *X, int64_t N, int d, int64_t Q, int64_t R, uint32_t *arg, float *dist,
                               cudaStream_t s)
{
    const unsigned blocks = (unsigned)((Q + 511) / 512);
    switch ((d + 3) / 4) {
    case 1: k_nearest_ref<4><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist); break;
    case 2: k_nearest_ref<8><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist); break;
    case 3: k_nearest_ref<12><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist); break;
    case 4: k_nearest_ref<16><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist); break;
    case 5: k_nearest_ref<20><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist); break;
    case 6: k_nearest_ref<24><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist); break;
    case 7:
        if (d == 25) k_nearest_ref<28, 25><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist);   // the paper's width
        else k_nearest_ref<28><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist);
        break;
    default: k_nearest_ref<32><<<blocks, 256, 0, s>>>(X, N, d, Q, R, arg, dist); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

// Histogram of the squared distances to the landmarks by their top 12 bits (exponent and
// three mantissa bits), for the median.
constexpr int kHistBins = 4096;

__global__ void __launch_bounds__(256) k_dist_hist(const float *__restrict__ dist, int64_t n,
                                                   unsigned int *__restrict__ hist)
{
    __shared__ unsigned int h[kHistBins];
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[__float_as_uint(dist[q]) >> 20], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < kHistBins; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Isolation threshold: 9 times the upper edge of the median's bin.
__global__ void k_dist_tau(const unsigned int *__restrict__ hist, int64_t n, float *__restrict__ tau)
{
    if (threadIdx.x != 0) return;
    unsigned long long run = 0;
    int b = 0;
    for (; b < kHistBins; ++b) {
        run += hist[b];
        if (2 * run >= (unsigned long long)n) break;
    }
    const float edge = b + 1 < 2040 ? __uint_as_float((unsigned int)(b + 1) << 20) : INFINITY;
    *tau = 9.0f * edge;
}

// Sort keys of the landmarks: (chain rank of the nearest coarse landmark, distance).
__global__ void k_landmark_keys(const uint32_t *__restrict__ arg, const float *__restrict__ dist, int64_t L,
                                const uint32_t *__restrict__ crank, nnm_edge *__restrict__ keys)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    nnm_edge e;
    e.a = (uint32_t)m;
    e.b = 0u;
    e.D = (double)crank[arg[m]] * 4294967296.0 + (double)__float_as_uint(dist[m]);   // exact: < 2^53
    keys[m] = e;
}

// Sort keys of the rows: (instance, isolated, rank of the landmark group, distance), the
// distance by its top 24 bits (an order-preserving truncation), in one exact double:
// instance < 2^16, 1 + 12 bits, 24 bits.
__global__ void k_row_keys(const uint32_t *__restrict__ arg, const float *__restrict__ dist, int64_t N,
                           const uint32_t *__restrict__ lrank, const uint32_t *__restrict__ inst,
                           const float *__restrict__ tau, nnm_edge *__restrict__ keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float v = dist[i];
    const double far = v > *tau ? 4096.0 : 0.0;   // above every group rank (< 4096)
    const double b = inst ? (double)inst[i] * 8192.0 : 0.0;
    nnm_edge e;
    e.a = (uint32_t)i;
    e.b = 0u;
    e.D = (b + far + (double)lrank[arg[i]]) * 16777216.0 + (double)(__float_as_uint(v) >> 8);   // exact: < 2^53
    keys[i] = e;
}

__global__ void k_instance_ids(const int64_t *__restrict__ off, int64_t B, int64_t N, uint32_t *__restrict__ inst)
{
    const int64_t b = blockIdx.x;
    if (b >= B) return;
    for (int64_t p = off[b] + threadIdx.x; p < off[b + 1] && p < N; p += blockDim.x) inst[p] = (uint32_t)b;
}

cudaError_t launch_instance_ids(const int64_t *off, int64_t B, int64_t N, uint32_t *inst, cudaStream_t s)
{
    k_instance_ids<<<(unsigned)B, 256, 0, s>>>(off, B, N, inst);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_spatial_keys(const uint32_t *larg, const float *ldist, int64_t L, const uint32_t *crank,
                                const uint32_t *rarg, const float *rdist, int64_t N, const uint32_t *lrank,
                                const uint32_t *inst, unsigned int *hist, float *tau, nnm_edge *lkeys,
                                nnm_edge *rkeys, int which, cudaStream_t s)
{
    if (which == 0) {
        k_landmark_keys<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(larg, ldist, L, crank, lkeys);
        count_launches(1);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(hist, 0, kHistBins * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    int blocks = (int)((N + 255) / 256);
    if (blocks > 152 * 4) blocks = 152 * 4;
    k_dist_hist<<<blocks, 256, 0, s>>>(rdist, N, hist);
    k_dist_tau<<<1, 32, 0, s>>>(hist, N, tau);
    k_row_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(rarg, rdist, N, lrank, inst, tau, rkeys);
    count_launches(3);
    return cudaGetLastError();
}

__global__ void k_order_from_keys(const nnm_edge *__restrict__ keys, int64_t N, uint32_t *pos2row,
                                  uint32_t *row2pos, uint32_t *group)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const uint32_t i = keys[p].a;
    pos2row[p] = i;
    row2pos[i] = (uint32_t)p;
    if (group) group[p] = (uint32_t)(keys[p].D * 0x1p-24);   // the row key's high part: instance, isolated, group
}

cudaError_t launch_order_from_keys(const nnm_edge *keys, int64_t N, uint32_t *pos2row, uint32_t *row2pos,
                                   uint32_t *group, cudaStream_t s)
{
    k_order_from_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(keys, N, pos2row, row2pos, group);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_gather_u32(const uint32_t *__restrict__ in, const uint32_t *__restrict__ map, int64_t n,
                             uint32_t *__restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = map[in[q]];
}

cudaError_t launch_gather_u32(const uint32_t *in, const uint32_t *map, int64_t n, uint32_t *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_gather_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, map, n, out);
    count_launches(1);
    return cudaGetLastError();
}

// Ordered compaction (per-block counts, one prefix over the blocks, ordered scatter).
constexpr int kCompactThreads = 1024;

int64_t compact_blocks(int64_t n) { return (n + kCompactThreads - 1) / kCompactThreads; }

__global__ void __launch_bounds__(kCompactThreads) k_cmp_count(const uint8_t *__restrict__ flag, int64_t n,
                                                               uint32_t *__restrict__ block_cnt)
{
    const int64_t q = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
    const int c = __syncthreads_count(q < n && flag[q] != 0);
    if (threadIdx.x == 0) block_cnt[blockIdx.x] = (uint32_t)c;
}

// exclusive prefix over nb block counts, one block of 1024 threads in chunks of 1024
__global__ void __launch_bounds__(kCompactThreads) k_cmp_prefix(uint32_t *__restrict__ block_cnt, int64_t nb,
                                                                uint32_t *__restrict__ count)
{
    __shared__ uint32_t ws[kCompactThreads / 32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += kCompactThreads) {
        const int64_t b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? block_cnt[b] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        if (w == 0) {
            const uint32_t t = ws[lane];
            uint32_t z = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            ws[lane] = z - t;
        }
        __syncthreads();
        const uint32_t c0 = carry;
        if (b < nb) block_cnt[b] = c0 + ws[w] + x - v;
        __syncthreads();
        if (threadIdx.x == kCompactThreads - 1) carry = c0 + ws[w] + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

__global__ void __launch_bounds__(kCompactThreads) k_cmp_scatter(const uint8_t *__restrict__ flag, int64_t n,
                                                                 const uint32_t *__restrict__ rows,
                                                                 const float *__restrict__ vals,
                                                                 const uint32_t *__restrict__ block_cnt,
                                                                 uint32_t *__restrict__ out_rows,
                                                                 float *__restrict__ out_vals)
{
    __shared__ uint32_t ws[kCompactThreads / 32];
    const int64_t q = (int64_t)blockIdx.x * kCompactThreads + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool f = q < n && flag[q] != 0;
    const uint32_t bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) ws[w] = __popc(bal);
    __syncthreads();
    if (w == 0) {
        const uint32_t v = ws[lane];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        ws[lane] = x - v;
    }
    __syncthreads();
    if (f) {
        const uint32_t r = block_cnt[blockIdx.x] + ws[w] + __popc(bal & ((1u << lane) - 1u));
        out_rows[r] = rows ? rows[q] : (uint32_t)q;
        if (vals) out_vals[r] = vals[q];
    }
}

cudaError_t launch_compact(const uint8_t *flag, int64_t n, const uint32_t *rows, const float *vals, uint32_t *block_cnt,
                           uint32_t *out_rows, float *out_vals, uint32_t *count, cudaStream_t s)
{
    if (n <= 0) return cudaMemsetAsync(count, 0, sizeof(uint32_t), s);
    const int64_t nb = compact_blocks(n);
    k_cmp_count<<<(unsigned)nb, kCompactThreads, 0, s>>>(flag, n, block_cnt);
    k_cmp_prefix<<<1, kCompactThreads, 0, s>>>(block_cnt, nb, count);
    k_cmp_scatter<<<(unsigned)nb, kCompactThreads, 0, s>>>(flag, n, rows, vals, block_cnt, out_rows, out_vals);
    count_launches(3);
    return cudaGetLastError();
}

__global__ void k_gather_f32(const uint32_t *__restrict__ in, const float *__restrict__ map, int64_t n,
                             float *__restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = map[in[q]];
}

cudaError_t launch_gather_f32(const uint32_t *in, const float *map, int64_t n, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_gather_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, map, n, out);
    count_launches(1);
    return cudaGetLastError();
}

// One block per column tile.  The tile's positions split where their landmark group
// first changes (part 0: the first group, part 1: the rest, possibly empty): two
// bounding spheres, each the centroid (mean) of y = (x - mu_f) * scale_f over its part
// and the largest distance to it, enlarged by sphere_slack (radius -1: empty part).
// A tile that straddles two groups is then bounded by two tight spheres, not one wide one.
__global__ void __launch_bounds__(128) k_tile_spheres(const float *__restrict__ X, int64_t N, int d,
                                                      const uint32_t *__restrict__ pos2row,
                                                      const uint32_t *__restrict__ group,
                                                      const float *__restrict__ mu_f, float scale_f, int tile_w,
                                                      float *__restrict__ tile_c, float *__restrict__ tile_rho,
                                                      const float *__restrict__ land_d2, float land_slack,
                                                      float *__restrict__ lup, float *__restrict__ tile_lmin)
{
    __shared__ float csum[2][32];
    __shared__ unsigned int rbits[2], ybits;
    __shared__ int cnt[2];
    const int64_t p0 = (int64_t)blockIdx.x * tile_w;
    const int64_t p = p0 + threadIdx.x;
    const bool valid = threadIdx.x < tile_w && p < N;
    const int h = (valid && group && group[p] != group[p0]) ? 1 : 0;
    if (threadIdx.x < 64) (&csum[0][0])[threadIdx.x] = 0.0f;
    if (threadIdx.x == 0) {
        rbits[0] = rbits[1] = 0u;
        ybits = 0u;
        cnt[0] = cnt[1] = 0;
    }
    __syncthreads();
    float y[32];
    float ny = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        y[k] = 0.0f;
        if (valid && k < d) {
            const float x = X[(int64_t)pos2row[p] * d + k];
            y[k] = (x - (mu_f ? mu_f[k] : 0.0f)) * scale_f;
            ny = fmaf(y[k], y[k], ny);
            atomicAdd(&csum[h][k], y[k]);
        }
    }
    if (valid) {
        atomicAdd(&cnt[h], 1);
        atomicMax(&ybits, __float_as_uint(sqrtf(ny)));
    }
    // Landmark distances in y units.  a = sqrtf(FP32 squared distance) is within 2^-20 of
    // the exact x distance to the row's landmark, and the FP32 nearest-landmark search
    // compared every landmark, so a also bounds the distance to any landmark from below
    // within the same factor; scale_f is a power of two, and land_slack covers the
    // rounding of y = (x - mu) * scale.  Up: |y - y_l| <= lup; down: every landmark is at
    // least lo away.
    __shared__ unsigned int lmin_bits;
    if (threadIdx.x == 0) lmin_bits = 0x7F800000u;   // +inf
    __syncthreads();
    if (land_d2 && valid) {
        const float a = sqrtf(land_d2[pos2row[p]]) * scale_f;
        lup[p] = __fadd_ru(__fmul_ru(a, 1.0f + 0x1p-12f), land_slack);
        const float lo = fmaxf(__fsub_rd(__fmul_rd(a, 1.0f - 0x1p-12f), land_slack), 0.0f);
        atomicMin(&lmin_bits, __float_as_uint(lo));   // non-negative floats order as their bits
    }
    __syncthreads();
    float dd = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        if (k < d) {
            const float e = y[k] - csum[h][k] / (float)(cnt[h] > 0 ? cnt[h] : 1);
            dd = fmaf(e, e, dd);
        }
    }
    if (valid) atomicMax(&rbits[h], __float_as_uint(sqrtf(dd)));
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * d; q += blockDim.x) {
        const int hh = q / d, k = q - hh * d;
        tile_c[((int64_t)blockIdx.x * 2 + hh) * d + k] = csum[hh][k] / (float)(cnt[hh] > 0 ? cnt[hh] : 1);
    }
    if (threadIdx.x < 2)
        tile_rho[blockIdx.x * 2 + threadIdx.x] =
            cnt[threadIdx.x] > 0 ? sphere_slack(__uint_as_float(rbits[threadIdx.x]), __uint_as_float(ybits)) : -1.0f;
    if (land_d2 && threadIdx.x == 0) tile_lmin[blockIdx.x] = __uint_as_float(lmin_bits);
}

cudaError_t launch_tile_spheres(const float *X, int64_t N, int d, const uint32_t *pos2row, const uint32_t *group,
                                const float *mu_f, float scale_f, int tile_w, float *tile_c, float *tile_rho,
                                const float *land_d2, float land_slack, float *lup, float *tile_lmin, cudaStream_t s)
{
    const int64_t nt = (N + tile_w - 1) / tile_w;
    k_tile_spheres<<<(unsigned)nt, 128, 0, s>>>(X, N, d, pos2row, group, mu_f, scale_f, tile_w, tile_c, tile_rho,
                                                 land_d2, land_slack, lup, tile_lmin);
    count_launches(1);
    return cudaGetLastError();
}

// One block of 64 threads per block of 32 tiles (thread = one of the tiles' two
// spheres): centre = mean of the non-empty sphere centres, radius = the largest
// |c - centre| + rho over them, enlarged by sphere_slack: a sphere holding all of them.
__global__ void __launch_bounds__(64) k_block_spheres(const float *__restrict__ tile_c,
                                                     const float *__restrict__ tile_rho, int64_t ntiles, int d,
                                                     float *__restrict__ blk_c, float *__restrict__ blk_rho,
                                                     const float *__restrict__ tile_lmin,
                                                     float *__restrict__ blk_lmin)
{
    __shared__ float csum[32];
    __shared__ unsigned int rbits, ybits, lbits;
    __shared__ int cnt;
    const int64_t sp = (int64_t)blockIdx.x * 64 + threadIdx.x;   // sphere index: tile * 2 + part
    const bool valid = sp < ntiles * 2 && tile_rho[sp] >= 0.0f;
    if (threadIdx.x < 32) csum[threadIdx.x] = 0.0f;
    if (threadIdx.x == 0) {
        rbits = 0u;
        ybits = 0u;
        lbits = 0x7F800000u;
        cnt = 0;
    }
    __syncthreads();
    if (tile_lmin && (sp & 1) == 0 && sp < ntiles * 2) atomicMin(&lbits, __float_as_uint(tile_lmin[sp >> 1]));
    float c[32];
    float nc = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        c[k] = (valid && k < d) ? tile_c[sp * d + k] : 0.0f;
        nc = fmaf(c[k], c[k], nc);
        if (valid && k < d) atomicAdd(&csum[k], c[k]);
    }
    const float rho = valid ? tile_rho[sp] : 0.0f;
    if (valid) {
        atomicAdd(&cnt, 1);
        atomicMax(&ybits, __float_as_uint(__fadd_ru(sqrtf(nc), rho)));
    }
    __syncthreads();
    if (valid) {
        float dd = 0.0f;
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (k < d) {
                const float e = c[k] - csum[k] / (float)cnt;
                dd = fmaf(e, e, dd);
            }
        atomicMax(&rbits, __float_as_uint(__fadd_ru(sqrtf(dd), rho)));
    }
    __syncthreads();
    if (threadIdx.x < d) blk_c[(int64_t)blockIdx.x * d + threadIdx.x] = csum[threadIdx.x] / (float)(cnt > 0 ? cnt : 1);
    if (threadIdx.x == 0) blk_rho[blockIdx.x] = cnt > 0 ? sphere_slack(__uint_as_float(rbits), __uint_as_float(ybits)) : -1.0f;
    if (tile_lmin && threadIdx.x == 0) blk_lmin[blockIdx.x] = __uint_as_float(lbits);
}

cudaError_t launch_block_spheres(const float *tile_c, const float *tile_rho, int64_t ntiles, int d, float *blk_c,
                                 float *blk_rho, const float *tile_lmin, float *blk_lmin, cudaStream_t s)
{
    const int64_t nb = (ntiles + 31) / 32;
    k_block_spheres<<<(unsigned)nb, 64, 0, s>>>(tile_c, tile_rho, ntiles, d, blk_c, blk_rho, tile_lmin, blk_lmin);
    count_launches(1);
    return cudaGetLastError();
}

// Padded FP32 copy in position order: positions [N, Npad) get a large value in every
// feature so that their candidate values are large; they are excluded by index anyway.
__global__ void k_pad_fp32(const float *__restrict__ X, int64_t N, int d, int dp, int64_t Npad,
                           const uint32_t *__restrict__ pos2row, float *__restrict__ Xs)
{
    int64_t total = Npad * dp;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = q / dp;
        int k = (int)(q - p * dp);
        float v = 0.0f;
        if (p >= N) v = k < d ? 1.0e18f : 0.0f;
        else if (k < d) v = X[(int64_t)pos2row[p] * d + k];
        Xs[q] = v;
    }
}

cudaError_t launch_pad_fp32(const float *X, int64_t N, int d, int dp, int64_t Npad, const uint32_t *pos2row,
                            float *Xs, cudaStream_t s)
{
    int64_t total = Npad * dp;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_pad_fp32<<<blocks, 256, 0, s>>>(X, N, d, dp, Npad, pos2row, Xs);
    count_launches(1);
    return cudaGetLastError();
}

// Column means: block b sums rows [b*chunk, (b+1)*chunk) in a fixed order, the final
// kernel adds the block sums in block order: the result does not depend on timing.
int mean_blocks(int64_t N)
{
    int64_t b = (N + 2047) / 2048;
    if (b > 1024) b = 1024;
    return (int)(b < 1 ? 1 : b);
}

__global__ void __launch_bounds__(256) k_mean_partial(const float *__restrict__ X, int64_t N, int d,
                                                      double *__restrict__ partial)
{
    __shared__ double red[256];
    int64_t chunk = (N + gridDim.x - 1) / gridDim.x;
    int64_t lo = (int64_t)blockIdx.x * chunk;
    int64_t hi = lo + chunk < N ? lo + chunk : N;
    for (int k = 0; k < d; ++k) {
        double acc = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += 256) acc += (double)X[i * d + k];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * d + k] = red[0];
        __syncthreads();
    }
}

__global__ void k_mean_final(const double *__restrict__ partial, int blocks, int d, int64_t N,
                             double *__restrict__ mu)
{
    int k = threadIdx.x;
    if (k >= d) return;
    double acc = 0.0;
    for (int b = 0; b < blocks; ++b) acc += partial[(int64_t)b * d + k];
    mu[k] = acc / (double)N;
}

cudaError_t launch_mean(const float *X, int64_t N, int d, double *partial, int blocks, double *mu,
                        cudaStream_t s)
{
    k_mean_partial<<<blocks, 256, 0, s>>>(X, N, d, partial);
    count_launches(1);
    k_mean_final<<<1, 32, 0, s>>>(partial, blocks, d, N, mu);
    count_launches(1);
    return cudaGetLastError();
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v)
{
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_max_sqnorm(const float *__restrict__ X, int64_t N, int d, const double *__restrict__ mu,
                             unsigned long long *out)
{
    double best = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        double s2 = 0.0;
        for (int k = 0; k < d; ++k) {
            double e = (double)X[i * d + k] - mu[k];
            s2 += e * e;
        }
        best = fmax(best, s2);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, best);
}

cudaError_t launch_max_sqnorm(const float *X, int64_t N, int d, const double *mu,
                              unsigned long long *out_bits, cudaStream_t s)
{
    int blocks = (int)((N + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_max_sqnorm<<<blocks, 256, 0, s>>>(X, N, d, mu, out_bits);
    count_launches(1);
    return cudaGetLastError();
}

// Round a binary64 value to the 16-bit operand format (round to nearest even) and
// return it both as bits and as its exact binary64 value.
__device__ __forceinline__ uint16_t round16(double v, int fp16, double *exact)
{
    if (fp16) {
        __half h = __double2half(v);
        *exact = (double)__half2float(h);
        return __half_as_ushort(h);
    }
    __nv_bfloat16 h = __double2bfloat16(v);
    *exact = (double)__bfloat162float(h);
    return __bfloat16_as_ushort(h);
}

// Tensor-core operands.  With y = (x - mu) * scale (scale a power of two) and x_hat
// its 16-bit approximation, the accumulator of the row operand A_i against the column
// operand B_j is |x_hat_i - x_hat_j|^2 (+ a bounded term for the split form):
//   one term  : x_hat = round16(y);  A = [x_hat, 1,1,1, a],  B = [-2 x_hat, a, 1,1,1]
//   split (3) : x_hat = hi + lo, hi = bf16(y), lo = bf16(y - hi);
//               A = [hi, hi, lo, 1,1,1, a],  B = [-2 hi, -2 lo, -2 hi, a, 1,1,1]
//               so A.B = |x_hat_i|^2 + |x_hat_j|^2 - 2 x_hat_i.x_hat_j + 2 lo_i.lo_j
// where a = (a1, a2, a3) splits the binary64 norm |x_hat|^2 into three 16-bit values.
// Per row: r = |x_hat - y| (rounding radius, rounded up); P bounds the terms' size
// (|x_hat| for one term, |hi| + |lo| for the split form); E = the norm split's residual
// plus, for the split form, |lo|^2 (2 lo_i.lo_j <= |lo_i|^2 + |lo_j|^2).  These bound
// the candidate error in the re-rank's completeness test.
constexpr int kOpThreads = 64;   // positions per block (a multiple of 8: whole core-matrix groups)

// One thread per position; the row's 16-bit values are assembled in shared memory and the
// block writes its positions' region of XA / XB with 16-byte stores.  Layout (core-matrix
// interleaved): element (position p, K index k) sits at
//     (((p / 8) * (kpad / 8) + k / 8) * 8 + p % 8) * 8 + k % 8,
// 8-position groups of kpad/8 core matrices (8 rows x 16 bytes), so the positions of one
// block (a multiple of 8) own one contiguous region.
__global__ void __launch_bounds__(kOpThreads) k_tc_operands(const float *__restrict__ X, int64_t N, int d,
                                                            const double *__restrict__ mu, double scale, int fp16,
                                                            int terms, int kpad, int64_t Npad,
                                                            const uint32_t *__restrict__ pos2row,
                                                            uint16_t *__restrict__ XA, uint16_t *__restrict__ XB,
                                                            float *__restrict__ r_out, float *__restrict__ P_out,
                                                            float *__restrict__ E_out, unsigned long long *max_bits)
{
    extern __shared__ __align__(16) uint16_t op_sm[];   // [2][kOpThreads][kpad]
    uint16_t *sa = op_sm + (size_t)threadIdx.x * kpad;
    uint16_t *sb = op_sm + (size_t)(kOpThreads + threadIdx.x) * kpad;
    const int64_t p = (int64_t)blockIdx.x * kOpThreads + threadIdx.x;   // position (< Npad)
    const uint16_t one = fp16 ? (uint16_t)0x3C00 : (uint16_t)0x3F80;
    const int D = terms * d;   // product columns
    float rf = 0.0f, Pf = 0.0f, Ef = 0.0f;
    if (p >= N) {
        // padding column: a huge accumulator; padding row: zeros (never read back)
        const uint16_t big = fp16 ? (uint16_t)0x7800 /* 32768 */ : (uint16_t)0x7180 /* 2^100 */;
        for (int k = 0; k < kpad; ++k) {
            sa[k] = 0;
            sb[k] = (k >= D && k < D + 3) ? big : (uint16_t)0;
        }
    } else {
        const int64_t i = pos2row[p];
        double rr = 0.0, n = 0.0, ynorm2 = 0.0, hn = 0.0, ln = 0.0;
        for (int k = 0; k < d; ++k) {
            const double y = ((double)X[i * d + k] - mu[k]) * scale;
            double h, l = 0.0, t;
            const uint16_t hb = round16(y, fp16, &h);
            uint16_t lb = 0;
            if (terms == 3) lb = round16(y - h, fp16, &l);
            const double xh = h + l;   // exact: both are 16-bit values of nearby binades
            rr += (xh - y) * (xh - y);
            n += xh * xh;
            ynorm2 += y * y;
            hn += h * h;
            ln += l * l;
            // -2 * v is exact in either format (sign flip, exponent + 1)
            const uint16_t hb2 = round16(-2.0 * h, fp16, &t);
            if (terms == 1) {
                sa[k] = hb;
                sb[k] = hb2;
            } else {
                const uint16_t lb2 = round16(-2.0 * l, fp16, &t);
                sa[k] = hb;
                sa[d + k] = hb;
                sa[2 * d + k] = lb;
                sb[k] = hb2;
                sb[d + k] = lb2;
                sb[2 * d + k] = hb2;
            }
        }
        double a1, a2, a3;
        const uint16_t b1 = round16(n, fp16, &a1);
        const double rem = n - a1;
        const uint16_t b2 = round16(rem, fp16, &a2);
        const double rem2 = rem - a2;
        const uint16_t b3 = round16(rem2, fp16, &a3);
        double E = fabs(rem2 - a3) + ln;
        for (int k = D; k < kpad; ++k) {
            uint16_t va = 0, vb = 0;
            if (k < D + 3) {
                va = one;
                vb = k == D ? b1 : (k == D + 1 ? b2 : b3);
            } else if (k < D + 6) {
                va = k == D + 3 ? b1 : (k == D + 4 ? b2 : b3);
                vb = one;
            }
            sa[k] = va;
            sb[k] = vb;
        }
        // rounding radius: |x_hat - y| plus the binary64 error of (x - mu) * scale, both
        // enlarged by a relative 1e-12 for the roundings of these bound computations
        const double r = (sqrt(rr) + sqrt(ynorm2) * 0x1p-52) * (1.0 + 1e-12) + 1e-300;
        const double P = (terms == 1 ? sqrt(n) : sqrt(hn) + sqrt(ln)) * (1.0 + 1e-12);
        E = E * (1.0 + 1e-12);
        rf = __double2float_ru(r);
        Pf = __double2float_ru(P);
        Ef = __double2float_ru(E);
        r_out[i] = rf;
        P_out[i] = Pf;
        E_out[i] = Ef;
    }
    // maxima: one atomic per warp (non-negative floats order as their bits)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rf = fmaxf(rf, __shfl_xor_sync(0xffffffffu, rf, o));
        Pf = fmaxf(Pf, __shfl_xor_sync(0xffffffffu, Pf, o));
        Ef = fmaxf(Ef, __shfl_xor_sync(0xffffffffu, Ef, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&max_bits[0], (double)rf);
        atomic_max_nonneg(&max_bits[1], (double)Pf);
        atomic_max_nonneg(&max_bits[2], (double)Ef);
    }
    __syncthreads();
    // copy-out: uint4 u of the block's region is row (u / (8 cpr)) * 8 + u % 8 of the
    // block, chunk (u / 8) % cpr
    const int cpr = kpad >> 3;
    const int nu = kOpThreads * cpr;
    uint4 *ga = reinterpret_cast<uint4 *>(XA) + (int64_t)blockIdx.x * nu;
    uint4 *gb = reinterpret_cast<uint4 *>(XB) + (int64_t)blockIdx.x * nu;
    for (int u = threadIdx.x; u < nu; u += kOpThreads) {
        const int gl = u / (cpr * 8), rem = u - gl * cpr * 8, c = rem >> 3, row = gl * 8 + (rem & 7);
        ga[u] = *reinterpret_cast<const uint4 *>(op_sm + (size_t)row * kpad + c * 8);
        gb[u] = *reinterpret_cast<const uint4 *>(op_sm + (size_t)(kOpThreads + row) * kpad + c * 8);
    }
}

cudaError_t launch_tc_operands(const float *X, int64_t N, int d, const double *mu, double scale, int fp16, int terms,
                               int kpad, int64_t Npad, const uint32_t *pos2row, uint16_t *XA, uint16_t *XB, float *r,
                               float *P, float *E, unsigned long long *max_bits, cudaStream_t s)
{
    if (Npad % kOpThreads != 0 || kpad % 16 != 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * kOpThreads * kpad * sizeof(uint16_t);   // <= 28 KB (kpad <= 112)
    const unsigned blocks = (unsigned)(Npad / kOpThreads);
    k_tc_operands<<<blocks, kOpThreads, smem, s>>>(X, N, d, mu, scale, fp16, terms, kpad, Npad, pos2row, XA, XB, r, P,
                                                   E, max_bits);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnm
