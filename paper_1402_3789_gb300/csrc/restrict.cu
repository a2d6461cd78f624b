// restrict.cu -- K7 restriction walk and K8 labels.
//
// The restrictions of "Problem statement" and "Problem settings" (maximum joining
// distance, KL1..KL4) act on the merge sequence.  With only the cap and KL1 the accepted
// joins are a prefix and dendro.cu computes them in parallel; when KL2, KL3 or KL4 is
// set (gates that read cluster sizes) the tree edges are walked in key order
// (in a batched context: each instance's edges, one CTA per instance, in parallel)
// with a union-find that tracks cluster sizes and the cluster count.  The walk is
// sequential by definition (each decision reads sizes that earlier joins changed), so
// it runs in one CTA over chunks of 2048 edges:
//   1. all threads find the current global roots of the chunk's endpoints,
//   2. the distinct roots get local ids (shared-memory hash), with their sizes,
//   3. one thread walks the chunk in order on the local union-find in shared memory,
//      applying the gates, and records each decision,
//   4. all threads write the joins back to the global union-find and emit the
//      accepted merges (and, with KL4, the deferred edges) in order.
// KL4 runs the walk twice: the first walk joins only pairs that touch a cluster smaller
// than KL4 and defers the others; the second walks the deferred edges in key order.
//
// Labels: the union-find after the walk is the final partition; labels are numbered by
// each cluster's smallest row index (a prefix sum over "row is its cluster's smallest").
#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr int kWalkThreads = 1024;
constexpr int kChunk = 2048;
constexpr int kLocal = 2 * kChunk;
constexpr int kHash = 2 * kLocal;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

struct WalkShared {
    uint32_t ra[kChunk], rb[kChunk];          // global roots of the endpoints
    uint16_t la[kChunk], lb[kChunk];          // local ids
    uint32_t hkey[kHash];
    uint16_t hval[kHash];
    uint32_t glob[kLocal];                    // local id -> global root
    uint16_t lpar[kLocal];                    // local union-find
    uint32_t lsize[kLocal];
    uint32_t newsize[kChunk];
    uint8_t dec[kChunk];                      // 0 none, 1 joined, 2 deferred
    uint32_t scan1[kChunk], scan2[kChunk];
    uint32_t wsum1[32], wsum2[32];
    uint32_t nloc;
    int stop;
    int64_t joined;                           // joins so far
};

__device__ __forceinline__ uint32_t gfind(uint32_t *par, uint32_t x)
{
    for (int guard = 0; guard < (1 << 26); ++guard) {
        uint32_t p = par[x];
        if (p == x) return x;
        uint32_t pp = par[p];
        if (pp != p) par[x] = pp;   // halving: only ever shortens paths
        x = pp;
    }
    return x;
}

__device__ __forceinline__ uint32_t lfind(uint16_t *par, uint32_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Exclusive block scan of two flag arrays over n <= kChunk entries (2 per thread).
__device__ void scan2_block(WalkShared &S, int n, uint32_t *tot1, uint32_t *tot2)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t a0 = 0, a1 = 0, b0 = 0, b1 = 0;
    const int e0 = 2 * t, e1 = 2 * t + 1;
    if (e0 < n) {
        a0 = S.dec[e0] == 1;
        b0 = S.dec[e0] == 2;
    }
    if (e1 < n) {
        a1 = S.dec[e1] == 1;
        b1 = S.dec[e1] == 2;
    }
    uint32_t sa = a0 + a1, sb = b0 + b1;
    uint32_t ia = sa, ib = sb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t xa = __shfl_up_sync(0xffffffffu, ia, o), xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += xa;
            ib += xb;
        }
    }
    if (lane == 31) {
        S.wsum1[w] = ia;
        S.wsum2[w] = ib;
    }
    __syncthreads();
    if (w == 0) {
        uint32_t va = S.wsum1[lane], vb = S.wsum2[lane];
        uint32_t xa = va, xb = vb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
            if (lane >= o) {
                xa += ya;
                xb += yb;
            }
        }
        S.wsum1[lane] = xa - va;   // exclusive warp offsets
        S.wsum2[lane] = xb - vb;
        if (lane == 31) {
            *tot1 = xa;
            *tot2 = xb;
        }
    }
    __syncthreads();
    const uint32_t ea = S.wsum1[w] + ia - sa, eb = S.wsum2[w] + ib - sb;
    if (e0 < n) {
        S.scan1[e0] = ea;
        S.scan2[e0] = eb;
    }
    if (e1 < n) {
        S.scan1[e1] = ea + a0;
        S.scan2[e1] = eb + b0;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kWalkThreads, 1) k_restrict(const RestrictArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    WalkShared &S = *reinterpret_cast<WalkShared *>(smem);
    __shared__ uint32_t tot1, tot2;
    __shared__ int64_t m_adm, n_def, n_out;
    const int t = threadIdx.x;
    // this walk's rows and edges: everything, or (batched) instance blockIdx.x
    const bool batched = a.n_inst > 1;
    const int64_t rlo = batched ? a.inst_off[blockIdx.x] : 0, rhi = batched ? a.inst_off[blockIdx.x + 1] : a.N;
    const int64_t elo = batched ? a.ebeg[blockIdx.x] : 0, ehi = batched ? a.eend[blockIdx.x] : a.m;
    const int64_t nrows = rhi - rlo;
    const nnm_edge *edges = a.edges + elo;
    nnm_merge *merges = batched ? a.merges_tmp + elo : a.merges;
    uint32_t *deferred = a.deferred + elo;

    if (!a.persist) {
        for (int64_t i = rlo + t; i < rhi; i += kWalkThreads) {
            a.uf_parent[i] = (uint32_t)i;
            a.uf_size[i] = 1u;
        }
    }
    if (t == 0) {
        // admissible prefix: the edges are key-sorted, so D <= cap^2 is a prefix
        int64_t lo = 0, hi = ehi - elo;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (edges[mid].D <= a.cap2) lo = mid + 1;
            else hi = mid;
        }
        m_adm = lo;
        n_def = 0;
        n_out = a.persist ? (int64_t)*a.n_merges : 0;
        S.stop = a.persist ? *a.stop_io : 0;
        S.joined = a.persist ? (int64_t)*a.joined_io : 0;
    }
    __syncthreads();

    const int walks = (a.kl4 > 0 && !a.persist) ? 2 : 1;
    for (int walk = 0; walk < walks && !S.stop; ++walk) {
        const bool defer_pass = a.kl4 > 0 && walk == 0 && !a.persist;
        const bool skip_big = a.persist && a.lit_phase == 1 && a.kl4 > 0;
        const int64_t total = walk == 0 ? m_adm : n_def;
        for (int64_t c0 = 0; c0 < total && !S.stop; c0 += kChunk) {
            const int n = (int)(total - c0 < kChunk ? total - c0 : kChunk);
            // 1. global roots
            for (int e = t; e < n; e += kWalkThreads) {
                const int64_t ei = walk == 0 ? c0 + e : (int64_t)deferred[c0 + e];
                const nnm_edge ed = edges[ei];
                S.ra[e] = gfind(a.uf_parent, ed.a);
                S.rb[e] = gfind(a.uf_parent, ed.b);
            }
            for (int h = t; h < kHash; h += kWalkThreads) S.hkey[h] = kEmpty;
            if (t == 0) S.nloc = 0;
            __syncthreads();
            // 2. local ids: insert keys, then number the occupied slots, then look up
            for (int q = t; q < 2 * n; q += kWalkThreads) {
                const uint32_t r = q < n ? S.ra[q] : S.rb[q - n];
                uint32_t h = hash32(r) & (kHash - 1);
                for (;;) {
                    const uint32_t prev = atomicCAS(&S.hkey[h], kEmpty, r);
                    if (prev == kEmpty || prev == r) break;
                    h = (h + 1) & (kHash - 1);
                }
            }
            __syncthreads();
            for (int h = t; h < kHash; h += kWalkThreads) {
                if (S.hkey[h] != kEmpty) {
                    const uint32_t id = atomicAdd(&S.nloc, 1u);
                    S.hval[h] = (uint16_t)id;
                    S.glob[id] = S.hkey[h];
                    S.lpar[id] = (uint16_t)id;
                    S.lsize[id] = a.uf_size[S.hkey[h]];
                }
            }
            __syncthreads();
            for (int q = t; q < 2 * n; q += kWalkThreads) {
                const uint32_t r = q < n ? S.ra[q] : S.rb[q - n];
                uint32_t h = hash32(r) & (kHash - 1);
                while (S.hkey[h] != r) h = (h + 1) & (kHash - 1);
                if (q < n) S.la[q] = S.hval[h];
                else S.lb[q - n] = S.hval[h];
            }
            __syncthreads();
            // 3. the sequential walk
            if (t == 0) {
                int64_t joined = S.joined;
                for (int e = 0; e < n; ++e) {
                    S.dec[e] = 0;
                    if (S.stop) continue;
                    const uint32_t x = lfind(S.lpar, S.la[e]), y = lfind(S.lpar, S.lb[e]);
                    if (x == y) continue;
                    const uint32_t sx = S.lsize[x], sy = S.lsize[y];
                    if ((defer_pass || skip_big) && sx >= (uint64_t)a.kl4 && sy >= (uint64_t)a.kl4) {
                        S.dec[e] = skip_big ? 0 : 2;
                        continue;
                    }
                    if (a.kl2 > 0 && (sx > (uint64_t)a.kl2 || sy > (uint64_t)a.kl2)) continue;
                    if (a.kl3 > 0 && (uint64_t)sx + sy > (uint64_t)a.kl3) continue;
                    if (a.kl1 > 0 && nrows - joined <= a.kl1) {
                        S.stop = 1;
                        continue;
                    }
                    uint32_t big = x, small = y;
                    if (sx < sy) {
                        big = y;
                        small = x;
                    }
                    S.lpar[small] = (uint16_t)big;
                    S.lsize[big] = sx + sy;
                    S.newsize[e] = sx + sy;
                    S.dec[e] = 1;
                    ++joined;
                }
                S.joined = joined;
            }
            __syncthreads();
            // 4. write back
            for (uint32_t l = t; l < S.nloc; l += kWalkThreads) {
                uint32_t r = l;
                while (S.lpar[r] != r) r = S.lpar[r];
                if (r != l) a.uf_parent[S.glob[l]] = S.glob[r];
                else a.uf_size[S.glob[l]] = S.lsize[l];
            }
            scan2_block(S, n, &tot1, &tot2);
            for (int e = t; e < n; e += kWalkThreads) {
                const int64_t ei = walk == 0 ? c0 + e : (int64_t)deferred[c0 + e];
                if (S.dec[e] == 1) {
                    const nnm_edge ed = edges[ei];
                    nnm_merge mg;
                    mg.a = ed.a;
                    mg.b = ed.b;
                    mg.D = ed.D;
                    mg.dist = a.metric == 0 ? sqrt(ed.D) : ed.D;
                    mg.new_size = S.newsize[e];
                    merges[n_out + S.scan1[e]] = mg;
                } else if (S.dec[e] == 2) {
                    deferred[n_def + S.scan2[e]] = (uint32_t)ei;
                }
            }
            __syncthreads();
            if (t == 0) {
                n_out += tot1;
                if (walk == 0) n_def += tot2;
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        if (batched) a.inst_nm[blockIdx.x] = (unsigned long long)n_out;
        else *a.n_merges = (unsigned long long)n_out;
        if (a.persist) {
            *a.joined_io = (long long)S.joined;
            *a.stop_io = S.stop;
        }
    }
}

// Batched walks: exclusive prefix of the per-instance merge counts (one thread), then
// one block per instance copies its merges into place.
__global__ void k_merge_offsets(unsigned long long *nm, int64_t n_inst, unsigned long long *total)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long run = 0;
    for (int64_t b = 0; b < n_inst; ++b) {
        const unsigned long long v = nm[b];
        nm[b] = run;
        run += v;
    }
    nm[n_inst] = run;
    *total = run;
}

__global__ void k_merge_pack(const RestrictArgs a)
{
    const int64_t b = blockIdx.x;
    const unsigned long long o = a.inst_nm[b], n = a.inst_nm[b + 1] - o;
    for (unsigned long long q = threadIdx.x; q < n; q += blockDim.x) a.merges[o + q] = a.merges_tmp[a.ebeg[b] + q];
}

__global__ void k_edge_ranges(const nnm_edge *__restrict__ e, int64_t m, const uint32_t *__restrict__ inst,
                              int64_t *__restrict__ ebeg, int64_t *__restrict__ eend)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t b = inst[e[i].a];
    if (i == 0 || inst[e[i - 1].a] != b) ebeg[b] = i;
    if (i == m - 1 || inst[e[i + 1].a] != b) eend[b] = i + 1;
}

constexpr int kLabThreads = 256;

__global__ void k_lab_roots(LabelArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    a.minm[i] = kEmpty;
}

__global__ void k_lab_min(LabelArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const uint32_t r = gfind(a.uf_parent, (uint32_t)i);
    atomicMin(&a.minm[r], (uint32_t)i);
}

// flag[i] = 1 iff row i is its cluster's smallest member; block-local exclusive scan
__global__ void k_lab_flag_scan(LabelArgs a)
{
    __shared__ uint32_t ws[kLabThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t f = 0;
    if (i < a.N) f = a.minm[gfind(a.uf_parent, (uint32_t)i)] == (uint32_t)i;
    uint32_t x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t v = lane < kLabThreads / 32 ? ws[lane] : 0, s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kLabThreads / 32) ws[lane] = s - v;
        if (lane == kLabThreads / 32 - 1) a.block_sums[blockIdx.x] = s;
    }
    __syncthreads();
    if (i < a.N) a.flag[i] = ws[w] + x - f;
}

__global__ void k_lab_block_prefix(LabelArgs a, int64_t nblocks)
{
    if (threadIdx.x != 0) return;
    uint64_t run = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        const uint32_t v = a.block_sums[b];
        a.block_sums[b] = (uint32_t)run;
        run += v;
    }
    *a.K = run;
}

__global__ void k_lab_write(LabelArgs a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const uint32_t m = a.minm[gfind(a.uf_parent, (uint32_t)i)];
    a.labels[i] = (int32_t)(a.flag[m] + a.block_sums[m / kLabThreads]);
}

}  // namespace

cudaError_t launch_restrict(const RestrictArgs &a, cudaStream_t s)
{
    const size_t smem = sizeof(WalkShared);
    cudaError_t e = cudaFuncSetAttribute(k_restrict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const bool batched = a.n_inst > 1;
    k_restrict<<<batched ? (unsigned)a.n_inst : 1u, kWalkThreads, smem, s>>>(a);
    count_launches(1);
    if (batched) {
        k_merge_offsets<<<1, 32, 0, s>>>(a.inst_nm, a.n_inst, a.n_merges);
        k_merge_pack<<<(unsigned)a.n_inst, 256, 0, s>>>(a);
        count_launches(2);
    }
    return cudaGetLastError();
}

cudaError_t launch_edge_ranges(const nnm_edge *edges, int64_t m, const uint32_t *inst_of_row, int64_t n_inst,
                               int64_t *ebeg, int64_t *eend, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(ebeg, 0, (size_t)n_inst * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(eend, 0, (size_t)n_inst * sizeof(int64_t), s);
    if (e != cudaSuccess || m <= 0) return e;
    k_edge_ranges<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(edges, m, inst_of_row, ebeg, eend);
    count_launches(1);
    return cudaGetLastError();
}

int64_t labels_scratch_blocks(int64_t N) { return (N + kLabThreads - 1) / kLabThreads; }

cudaError_t launch_labels(const LabelArgs &a, cudaStream_t s)
{
    const int64_t nb = labels_scratch_blocks(a.N);
    k_lab_roots<<<(unsigned)nb, kLabThreads, 0, s>>>(a);
    count_launches(1);
    k_lab_min<<<(unsigned)nb, kLabThreads, 0, s>>>(a);
    count_launches(1);
    k_lab_flag_scan<<<(unsigned)nb, kLabThreads, 0, s>>>(a);
    count_launches(1);
    k_lab_block_prefix<<<1, 32, 0, s>>>(a, nb);
    count_launches(1);
    k_lab_write<<<(unsigned)nb, kLabThreads, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace nnm
