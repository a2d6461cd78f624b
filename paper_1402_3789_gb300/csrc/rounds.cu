// rounds.cu -- K4/K5: merge rounds on the device.
//
// The paper joins clusters along minimal pairs, skipping pairs that already lie
// inside one cluster ("General description of the algorithm for constructing the set
// of minimum distances").  On the GPU the same tree (the unique minimum spanning tree
// under key order) is grown in rounds: every component finds its smallest outgoing
// pair (key order), every component hooks onto the component at the other end (of a
// mutual pair, the smaller id stays root), and pointer jumping flattens the hooks.
// Each selected pair is a tree edge by the cut property; each is emitted once.
//
// Each row's exact k nearest neighbours (cache) answer most rows' "nearest neighbour
// outside my component" without a sweep: the first cached neighbour outside the
// component is the answer, because all columns outside the cache are farther.  A row
// whose whole cache lies inside its component only bounds its answer from below (by
// its last cached key); it is rescanned only if that bound is below its component's
// best resolved key.
//
// A rescan only has to find outgoing pairs that could still be the component's
// minimum, so it is bounded by an exact D that some outgoing pair of the component
// already has: the best resolved one, or one found by the flagged rows themselves
// among their neighbours in the spatial order of the operands.  A bounded rescan
// caches the k nearest eligible columns with D <= bound; when fewer than k exist, every
// other eligible column has D > bound, which is the row's new lower bound.
#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ unsigned long long pack_ab(uint32_t i, uint32_t j)
{
    const uint32_t a = i < j ? i : j, b = i < j ? j : i;
    return ((unsigned long long)a << 32) | b;
}

__device__ __forceinline__ bool key_less(unsigned long long d1, unsigned long long ab1, unsigned long long d2,
                                         unsigned long long ab2)
{
    return d1 < d2 || (d1 == d2 && ab1 < ab2);
}

inline unsigned grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b < 1 ? 1 : b);
}

__global__ void k_round_init(RoundState st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.N) return;
    st.comp[i] = (uint32_t)i;
    st.parent[i] = (uint32_t)i;
    st.frozen[i] = 0;
    st.row_B[i] = INFINITY;
}

// Per row: the key of its nearest neighbour outside its component, from the cache.
__global__ void k_resolve(RoundState st, const uint32_t *__restrict__ rows, int64_t nrows)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nrows) return;
    const uint32_t i = rows ? rows[q] : (uint32_t)q;
    const uint32_t c = st.comp[i];
    if (st.frozen[c]) {
        st.row_state[i] = 0;
        return;
    }
    const int n = st.cache_n[i];
    const uint32_t *cj = st.cache_j + (int64_t)i * st.k;
    const double *cD = st.cache_D + (int64_t)i * st.k;
    for (int m = 0; m < n; ++m) {
        const uint32_t j = cj[m];
        if (st.comp[j] != c) {
            st.row_D[i] = (unsigned long long)__double_as_longlong(cD[m]);
            st.row_ab[i] = pack_ab(i, j);
            st.row_state[i] = 1;
            return;
        }
    }
    const uint8_t cs = st.cache_exh[i];
    if (cs == kCacheAll || (n == 0 && cs == kCacheFull)) {
        st.row_state[i] = 0;   // every eligible column was cached: none is outside
        return;
    }
    if (cs == kCacheBounded) {
        // bounded scan: every column not cached has D > row_B
        const double B = st.row_B[i];
        if (!(B < INFINITY)) {
            st.row_state[i] = 0;
            return;
        }
        st.row_D[i] = (unsigned long long)__double_as_longlong(B);
        st.row_ab[i] = kMaxKey;
        st.row_state[i] = 2;
        return;
    }
    // lower bound: every column not cached has a larger key than the last cached one
    st.row_D[i] = (unsigned long long)__double_as_longlong(cD[n - 1]);
    st.row_ab[i] = pack_ab(i, cj[n - 1]);
    st.row_state[i] = 2;
}

__global__ void k_best_reset(RoundState st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.N) return;
    st.best_D[i] = kMaxKey;
    st.best_ab[i] = kMaxKey;
    st.comp_bound[i] = (unsigned long long)__double_as_longlong(INFINITY);
}

__global__ void k_best_d(RoundState st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.N || st.row_state[i] != 1) return;
    atomicMin(&st.best_D[st.comp[i]], st.row_D[i]);
    // the same pair leaves the other endpoint's component too: its D bounds that
    // component's minimum from above
    const unsigned long long ab = st.row_ab[i];
    const uint32_t lo = (uint32_t)(ab >> 32), hi = (uint32_t)ab;
    const uint32_t j = lo == (uint32_t)i ? hi : lo;
    atomicMin(&st.comp_bound[st.comp[j]], st.row_D[i]);
}

__global__ void k_best_ab(RoundState st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.N || st.row_state[i] != 1) return;
    const uint32_t c = st.comp[i];
    if (st.row_D[i] == st.best_D[c]) atomicMin(&st.best_ab[c], st.row_ab[i]);
}

constexpr int kNeighbourSearch = 16;   // positions searched on each side

__global__ void k_flag(RoundState st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.N) return;
    uint8_t f = 0;
    const uint32_t p = st.row2pos[i];
    bool done = false;   // the row's instance is one component already
    if (st.inst_edges) {
        const uint32_t b = st.inst_pos[i];
        done = (int64_t)st.inst_edges[b] + 1 == st.inst_off[b + 1] - st.inst_off[b];
    }
    if (st.row_state[i] == 2 && !done) {
        const uint32_t c = st.comp[i];
        f = key_less(st.row_D[i], st.row_ab[i], st.best_D[c], st.best_ab[c]);
        if (f) {
            // the nearest positions outside the component on either side give outgoing
            // pairs, whose exact D bound the component's minimum from above
            const float *xi = st.X + i * st.d;
            for (int side = -1; side <= 1; side += 2) {
                for (int s = 1; s <= kNeighbourSearch; ++s) {
                    const int64_t q = (int64_t)p + side * s;
                    if (q < 0 || q >= st.N) break;
                    if (st.inst_pos && st.inst_pos[q] != st.inst_pos[p]) break;   // another instance
                    const uint32_t j = st.pos2row[q];
                    if (st.comp[j] == c) continue;
                    const double D = canon_D(xi, st.X + (int64_t)j * st.d, st.d, st.metric);
                    atomicMin(&st.comp_bound[c], (unsigned long long)__double_as_longlong(D));
                    break;
                }
            }
        }
    }
    st.flag_pos[p] = f;
}

// A flagged row whose lower bound already exceeds a known outgoing D of its component
// cannot hold the component's minimum: it is not rescanned.
__global__ void k_flag_filter(RoundState st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.N) return;
    const uint32_t p = st.row2pos[i];
    if (!st.flag_pos[p]) return;
    const double lb = __longlong_as_double((long long)st.row_D[i]);
    const double B = __longlong_as_double((long long)st.comp_bound[st.comp[i]]);
    if (lb > B) st.flag_pos[p] = 0;
}

// Rescan rows in increasing position (so that a row tile of a rescan is spatially
// coherent): per-block counts, a prefix over blocks, then an ordered scatter.
constexpr int kCompact = 1024;

__global__ void __launch_bounds__(kCompact) k_compact_count(RoundState st)
{
    const int64_t p = (int64_t)blockIdx.x * kCompact + threadIdx.x;
    const int f = p < st.N ? st.flag_pos[p] : 0;
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) st.block_cnt[blockIdx.x] = (uint32_t)c;
}

__global__ void k_compact_prefix(RoundState st, int64_t nb)
{
    if (threadIdx.x != 0) return;
    uint32_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const uint32_t v = st.block_cnt[b];
        st.block_cnt[b] = run;
        run += v;
    }
    st.counters[0] = run;
}

__global__ void __launch_bounds__(kCompact) k_compact_scatter(RoundState st)
{
    __shared__ uint32_t ws[kCompact / 32];
    const int64_t p = (int64_t)blockIdx.x * kCompact + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t f = p < st.N ? st.flag_pos[p] : 0u;
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
        const uint32_t r = st.block_cnt[blockIdx.x] + ws[w] + __popc(bal & ((1u << lane) - 1u));
        const uint32_t i = st.pos2row[p];
        st.list_pos[r] = (uint32_t)p;
        st.list[r] = i;
        // the rescan bound: the smaller of the best resolved D and the neighbour bound
        const uint32_t c = st.comp[i];
        const unsigned long long bd = st.best_D[c];
        double B = bd == kMaxKey ? INFINITY : __longlong_as_double((long long)bd);
        B = fmin(B, __longlong_as_double((long long)st.comp_bound[c]));
        st.row_B[i] = B * st.overscan;
    }
}

// Hook every component root onto the component at the far end of its best pair.
__global__ void k_hook(RoundState st)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st.N || st.comp[c] != (uint32_t)c) return;   // roots only
    st.parent[c] = (uint32_t)c;
    if (st.frozen[c] || st.best_D[c] == kMaxKey) return;
    const double D = __longlong_as_double((long long)st.best_D[c]);
    if (D > st.cap2) {
        st.frozen[c] = 1;   // nothing within the cap leaves this component
        return;
    }
    const uint32_t a = (uint32_t)(st.best_ab[c] >> 32), b = (uint32_t)(st.best_ab[c] & 0xFFFFFFFFu);
    const uint32_t other = st.comp[a] == (uint32_t)c ? b : a;
    const uint32_t c2 = st.comp[other];
    const bool mutual = st.best_D[c2] == st.best_D[c] && st.best_ab[c2] == st.best_ab[c];
    if (mutual && (uint32_t)c < c2) return;   // the smaller id of a mutual pair stays root
    st.parent[c] = c2;
    if (st.inst_edges) atomicAdd(&st.inst_edges[st.inst_pos[a]], 1u);
    const uint32_t e = atomicAdd(st.n_edges, 1u);
    nnm_edge ed;
    ed.a = a;
    ed.b = b;
    ed.D = D;
    st.edges[e] = ed;
    atomicAdd(&st.counters[1], 1u);
}

__global__ void k_jump(RoundState st)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st.N || st.comp[c] != (uint32_t)c) return;
    const uint32_t p = st.parent[c];
    const uint32_t pp = st.parent[p];
    if (pp != p) {
        st.parent[c] = pp;
        st.counters[2] = 1u;
    }
}

__global__ void k_relabel(RoundState st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.N) return;
    st.comp[i] = st.parent[st.comp[i]];
}

// One warp per column tile: the component of each position, and the tile's common one.
__global__ void k_position_comps(const RoundState st, int tile_w, uint32_t *__restrict__ comp_pos,
                                 uint32_t *__restrict__ tile_comp, int64_t ntiles)
{
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (int q = lane; q < tile_w; q += 32) {
        const int64_t p = t * tile_w + q;
        if (p >= st.N) break;
        const uint32_t c = st.comp[st.pos2row[p]];
        comp_pos[p] = c;
        lo = min(lo, c);
        hi = max(hi, c);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) tile_comp[t] = lo == hi ? lo : kInvalid;
}

}  // namespace

cudaError_t launch_position_comps(const RoundState &st, int tile_w, uint32_t *comp_pos, uint32_t *tile_comp,
                                  cudaStream_t s)
{
    const int64_t ntiles = (st.N + tile_w - 1) / tile_w;
    k_position_comps<<<(unsigned)((ntiles * 32 + kThreads - 1) / kThreads), kThreads, 0, s>>>(st, tile_w, comp_pos,
                                                                                                tile_comp, ntiles);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_round_init(RoundState &st, cudaStream_t s)
{
    k_round_init<<<grid_for(st.N), kThreads, 0, s>>>(st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_resolve(RoundState &st, const uint32_t *rows, int64_t nrows, cudaStream_t s)
{
    if (nrows <= 0) return cudaSuccess;
    k_resolve<<<grid_for(nrows), kThreads, 0, s>>>(st, rows, nrows);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_component_min(RoundState &st, cudaStream_t s)
{
    k_best_reset<<<grid_for(st.N), kThreads, 0, s>>>(st);
    count_launches(1);
    k_best_d<<<grid_for(st.N), kThreads, 0, s>>>(st);
    count_launches(1);
    k_best_ab<<<grid_for(st.N), kThreads, 0, s>>>(st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_flag_rescans(RoundState &st, cudaStream_t s)
{
    k_flag<<<grid_for(st.N), kThreads, 0, s>>>(st);
    k_flag_filter<<<grid_for(st.N), kThreads, 0, s>>>(st);
    const int64_t nb = (st.N + kCompact - 1) / kCompact;
    k_compact_count<<<(unsigned)nb, kCompact, 0, s>>>(st);
    k_compact_prefix<<<1, 32, 0, s>>>(st, nb);
    k_compact_scatter<<<(unsigned)nb, kCompact, 0, s>>>(st);
    count_launches(5);
    return cudaGetLastError();
}

cudaError_t launch_hook(RoundState &st, cudaStream_t s)
{
    k_hook<<<grid_for(st.N), kThreads, 0, s>>>(st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_jump(RoundState &st, cudaStream_t s)
{
    k_jump<<<grid_for(st.N), kThreads, 0, s>>>(st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_relabel(RoundState &st, cudaStream_t s)
{
    k_relabel<<<grid_for(st.N), kThreads, 0, s>>>(st);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnm
