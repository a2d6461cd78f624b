// literal.cu -- the restrictions in the paper's all-pairs reading (nnm_restrictions
// semantics = 1): the gates act on every pair in key order, as in the paper's batched
// procedure over the P minimal pairs ("General description of the algorithm for
// constructing the set of minimum distances"; gates of "Problem settings").
//
// Two facts make it data-parallel between sequential walks:
//   - sizes only grow, so a pair that a gate blocks stays blocked, and a blocked pair
//     changes nothing.  Hence at any moment the next join is the smallest-key pair that
//     crosses two clusters and passes every gate now; a pair that fails at the start of
//     a batch fails at its own turn too and can be left out of the batch;
//   - a batch is the set of such pairs with key in (L, tau]: complete for that range, it
//     is walked in key order (restrict.cu, persist mode) and the next batch starts above
//     tau.  This is the paper's "P smallest pairs above the last one" with the pairs that
//     cannot join removed first.
// Batches are cut by value: one pass histograms the FP32 direct values of the eligible
// pairs by exponent, a second histograms the chosen octave by its top 12 mantissa bits,
// a third emits the pairs up to the cut value E (the same FP32 arithmetic in every pass,
// so the count is exact).  With |s - D| bounded by the FP32 margin, every pair with
// D <= tau = lo(E) has s <= E; binary64 D (canon_D) then keeps the pairs with
// L < D <= tau exactly.
//
// KL4 (joins touching a cluster below KL4 first) takes two phases.  Phase 1 joins only
// pairs touching a cluster below KL4 and passes over the others; phase 2 walks the
// passed-over pairs in key order.  A pair was passed over iff, at its turn in phase 1,
// it crossed two clusters that both had reached KL4 rows.  With t_i the key of the
// phase-1 join that brought row i's cluster to KL4 rows (computed by k_lit_reach), that
// is: key > max(t_i, t_j) and the pair still crossed then.  Pairs that no longer crossed
// are inside one cluster in phase 2 as well, so phase 2 takes every pair with
// key > max(t_i, t_j) and lets the walk skip the ones already joined.
#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr int kLT = 64;          // rows / columns per pair tile
constexpr int kLThreads = 256;   // 16 x 16 threads, 4 x 4 pairs each
constexpr int kFineBins = 4096;  // top 12 mantissa bits within one octave

__device__ __forceinline__ float hi_bound(float s, float c0, float c1)
{
    return __fadd_ru(__fmul_ru(__fadd_ru(s, c0), c1), c0);
}

// one pass over the pairs (i < j) of tile (blockIdx.y, blockIdx.x), blockIdx.x >= blockIdx.y
template <int METRIC, int MODE>
__global__ void __launch_bounds__(kLThreads) k_lit_pass(const LitArgs a)
{
    if (blockIdx.x < blockIdx.y) return;
    __shared__ float xr[kLT][33], xc[kLT][33];
    __shared__ uint32_t rc[kLT], cc[kLT], rs[kLT], cs[kLT];
    __shared__ double rt[kLT], ct[kLT];
    __shared__ uint32_t hist[MODE == 0 ? 256 : (MODE == 1 ? kFineBins : 1)];
    const int64_t i0 = (int64_t)blockIdx.y * kLT, j0 = (int64_t)blockIdx.x * kLT;
    const int t = threadIdx.x;
    for (int q = t; q < kLT * 32; q += kLThreads) {
        const int r = q >> 5, k = q & 31;
        const int64_t i = i0 + r, j = j0 + r;
        xr[r][k] = (i < a.N && k < a.d) ? a.X[i * a.d + k] : 0.0f;
        xc[r][k] = (j < a.N && k < a.d) ? a.X[j * a.d + k] : 0.0f;
    }
    if (t < kLT) {
        const int64_t i = i0 + t, j = j0 + t;
        rc[t] = i < a.N ? a.comp[i] : kInvalid;
        cc[t] = j < a.N ? a.comp[j] : kInvalid;
        rs[t] = i < a.N ? a.csize[i] : 0u;
        cs[t] = j < a.N ? a.csize[j] : 0u;
        rt[t] = (i < a.N && a.phase == 2) ? a.tD[i] : -1.0;
        ct[t] = (j < a.N && a.phase == 2) ? a.tD[j] : -1.0;
    }
    if (MODE == 0)
        for (int q = t; q < 256; q += kLThreads) hist[q] = 0u;
    if (MODE == 1)
        for (int q = t; q < kFineBins; q += kLThreads) hist[q] = 0u;
    __syncthreads();
    const int ty = t >> 4, tx = t & 15;
    float s[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) s[u][v] = 0.0f;
    for (int k = 0; k < a.d; ++k) {
        float xi[4], xj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xi[u] = xr[ty * 4 + u][k];
#pragma unroll
        for (int v = 0; v < 4; ++v) xj[v] = xc[tx * 4 + v][k];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float e = xi[u] - xj[v];
                if (METRIC == 1) s[u][v] += fabsf(e);
                else if (METRIC == 2) s[u][v] = fmaxf(s[u][v], fabsf(e));
                else s[u][v] = fmaf(e, e, s[u][v]);
            }
    }
    const float c0 = a.c0, c1 = a.c1, c1inv = a.c1inv;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = ty * 4 + u;
        const int64_t i = i0 + r;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int cidx = tx * 4 + v;
            const int64_t j = j0 + cidx;
            if (j <= i || j >= a.N) continue;
            if (rc[r] == cc[cidx]) continue;                                   // one cluster
            const uint32_t si = rs[r], sj = cs[cidx];
            if (a.kl2 > 0 && ((int64_t)si > a.kl2 || (int64_t)sj > a.kl2)) continue;
            if (a.kl3 > 0 && (int64_t)si + sj > a.kl3) continue;
            if (a.phase == 1 && a.kl4 > 0 && (int64_t)si >= a.kl4 && (int64_t)sj >= a.kl4) continue;
            const float sv = s[u][v];
            const float hi = hi_bound(sv, c0, c1);                             // D <= hi
            const float lo = __fsub_rd(__fmul_rd(__fsub_rd(sv, c0), c1inv), c0);   // D >= lo
            if (lo > a.cap2f) continue;                                        // beyond the cap
            if (a.have_last && (double)hi < a.last_D) continue;                // at or below the last batch
            if (a.phase == 2 && (double)hi < fmax(rt[r], ct[cidx])) continue;  // not passed over in phase 1
            const uint32_t bits = __float_as_uint(sv);
            if (MODE == 0) {
                atomicAdd(&hist[bits >> 23], 1u);
            } else if (MODE == 1) {
                if ((bits >> 23) == a.octave) atomicAdd(&hist[(bits >> 11) & (kFineBins - 1)], 1u);
            } else {
                if (sv <= a.cut) {
                    const unsigned long long q = atomicAdd(a.n_emit, 1ull);
                    if ((int64_t)q < a.emit_cap) {
                        nnm_edge ed;
                        ed.a = (uint32_t)i;
                        ed.b = (uint32_t)j;
                        ed.D = 0.0;
                        a.emit[q] = ed;
                    }
                }
            }
        }
    }
    if (MODE == 2) return;
    __syncthreads();
    const int nb = MODE == 0 ? 256 : kFineBins;
    for (int q = t; q < nb; q += kLThreads)
        if (hist[q]) atomicAdd(&a.hist[q], (unsigned long long)hist[q]);
}

// Exact binary64 D of the emitted pairs; a pair is kept iff L < key (D > L_D after the
// first batch), D <= tau, D <= the cap, and in phase 2 key > max(t_a, t_b).
__global__ void k_lit_exact(const LitArgs a)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.n_emitted) return;
    nnm_edge e = a.emit[q];
    const double D = canon_D(a.X + (int64_t)e.a * a.d, a.X + (int64_t)e.b * a.d, a.d, a.metric);
    if (a.have_last && !(D > a.last_D)) return;
    if (!(D <= a.tau_D) || !(D <= a.cap2)) return;
    if (a.phase == 2) {
        const unsigned long long ab = ((unsigned long long)e.a << 32) | e.b;
        for (int side = 0; side < 2; ++side) {
            const uint32_t r = side ? e.b : e.a;
            const double tD = a.tD[r];
            const unsigned long long tab = a.tab[r];
            if (!(tD < D || (tD == D && tab < ab))) return;   // the pair's key must exceed t_r
        }
    }
    e.D = D;
    const unsigned long long o = atomicAdd(a.n_kept, 1ull);
    a.kept[o] = e;
}

__device__ __forceinline__ uint32_t lit_find(uint32_t *par, uint32_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

__global__ void k_lit_flatten(const LitArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    uint32_t x = (uint32_t)i;
    for (int guard = 0; guard < (1 << 26); ++guard) {
        const uint32_t p = a.uf_parent[x];
        if (p == x) break;
        x = p;
    }
    a.comp[i] = x;
    a.csize[i] = a.uf_size[x];
}

__global__ void k_lit_init(const LitArgs a, double t0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    a.uf_parent[i] = (uint32_t)i;
    a.uf_size[i] = 1u;
    a.tD[i] = t0;
    a.tab[i] = 0ull;
}

// t_i: replay of the phase-1 joins (key order) with row lists per cluster; when a join
// makes a cluster of >= KL4 rows, the rows of each side that was below KL4 get the join's
// key.  One thread: the joins are at most N - 1 and each row is labelled once.
__global__ void k_lit_reach(const LitArgs a, const nnm_merge *merges, int64_t n1)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t *par = a.w0, *sz = a.w1, *head = a.w2, *nxt = a.w3, *tail = a.w4;
    for (int64_t i = 0; i < a.N; ++i) {
        par[i] = (uint32_t)i;
        sz[i] = 1u;
        head[i] = (uint32_t)i;
        tail[i] = (uint32_t)i;
        nxt[i] = kInvalid;
        // with KL4 <= 1 every cluster has reached KL4 from the start
        a.tD[i] = a.kl4 <= 1 ? -1.0 : INFINITY;
        a.tab[i] = a.kl4 <= 1 ? 0ull : ~0ull;
    }
    for (int64_t q = 0; q < n1; ++q) {
        const nnm_merge m = merges[q];
        uint32_t x = lit_find(par, m.a), y = lit_find(par, m.b);
        if (x == y) continue;
        const uint32_t sx = sz[x], sy = sz[y];
        if ((int64_t)sx + sy >= a.kl4) {
            for (int side = 0; side < 2; ++side) {
                const uint32_t r = side ? y : x;
                if ((int64_t)(side ? sy : sx) >= a.kl4) continue;
                for (uint32_t v = head[r]; v != kInvalid; v = nxt[v]) {
                    a.tD[v] = m.D;
                    a.tab[v] = ((unsigned long long)m.a << 32) | m.b;
                }
            }
        }
        if (sx < sy) {
            const uint32_t t = x;
            x = y;
            y = t;
        }
        par[y] = x;
        sz[x] = sx + sy;
        nxt[tail[x]] = head[y];
        tail[x] = tail[y];
    }
}

template <int METRIC>
cudaError_t lit_pass_m(const LitArgs &a, int mode, cudaStream_t s)
{
    const unsigned nt = (unsigned)((a.N + kLT - 1) / kLT);
    dim3 grid(nt, nt);
    if (mode == 0) k_lit_pass<METRIC, 0><<<grid, kLThreads, 0, s>>>(a);
    else if (mode == 1) k_lit_pass<METRIC, 1><<<grid, kLThreads, 0, s>>>(a);
    else k_lit_pass<METRIC, 2><<<grid, kLThreads, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int literal_fine_bins() { return kFineBins; }

cudaError_t launch_lit_pass(const LitArgs &a, int mode, cudaStream_t s)
{
    if (a.N > 65535LL * kLT) return cudaErrorInvalidValue;
    if (a.metric == 1) return lit_pass_m<1>(a, mode, s);
    if (a.metric == 2) return lit_pass_m<2>(a, mode, s);
    return lit_pass_m<0>(a, mode, s);
}

cudaError_t launch_lit_exact(const LitArgs &a, cudaStream_t s)
{
    if (a.n_emitted <= 0) return cudaSuccess;
    k_lit_exact<<<(unsigned)((a.n_emitted + 255) / 256), 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lit_flatten(const LitArgs &a, cudaStream_t s)
{
    k_lit_flatten<<<(unsigned)((a.N + 255) / 256), 256, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lit_init(const LitArgs &a, double t0, cudaStream_t s)
{
    k_lit_init<<<(unsigned)((a.N + 255) / 256), 256, 0, s>>>(a, t0);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_lit_reach(const LitArgs &a, const nnm_merge *merges, int64_t n1, cudaStream_t s)
{
    k_lit_reach<<<1, 32, 0, s>>>(a, merges, n1);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnm
