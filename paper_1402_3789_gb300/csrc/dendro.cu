// dendro.cu -- the restriction step when no gate reads cluster sizes (only the maximum
// joining distance and KL1 of "Problem statement" / "Problem settings", or none).
//
// Without KL2, KL3 and KL4 every admissible tree edge joins two different clusters, so
// the accepted joins of an instance are a prefix of its key-ordered tree edges: those
// with D within the cap, at most (rows - KL1) of them.  The decision is a parallel cut.
// What remains sequential in the walk is each join's new size: the number of rows in
// the cluster it creates, i.e. the rows connected to the edge through edges of smaller
// key.  Here all new sizes come out of O(log m) data-parallel levels instead:
//
// Invariant: the accepted edges (ranks 0..M-1) are split into ranges of 2h ranks; every
// endpoint of an edge carries the label (a representative row) and the size of its
// cluster under the edges ranked before its range.  One level turns ranges of 2h into
// ranges of h: in each range the low half's edges are joined on those labels (a
// concurrent union-find over (range, label) keys in a hash table), and the high half's
// endpoints take the label and the summed size of their component.  Starting from one
// range (labels = rows, sizes 1) and ending at ranges of one edge, every endpoint holds
// its cluster just before the edge, and the new size is the sum of the two.
// Work O(m log m), every step a flat kernel; each level's hash table holds at most 2M
// keys at load <= 1/2.
//
// The final clusters (for the labels) come from one concurrent union-find over the
// accepted edges.
#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr unsigned long long kEmptyKey = ~0ULL;
constexpr int kThreads = 256;
constexpr int kUnionGuard = 1 << 22;   // retries of one union (far above what contention allows)

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

// Root of x with path halving.  Parents only ever point at ancestors (links go from a
// larger root to a smaller index), so concurrent halving and linking stay consistent;
// loads bypass L1, which other SMs' links do not update.
__device__ __forceinline__ uint32_t cfind(uint32_t *par, uint32_t x)
{
    for (;;) {
        const uint32_t p = __ldcg(par + x);
        if (p == x) return x;
        const uint32_t pp = __ldcg(par + p);
        if (pp != p) par[x] = pp;
        x = pp;
    }
}

// Join the sets of x and y: the larger root is linked under the smaller one.
__device__ bool cunion(uint32_t *par, uint32_t x, uint32_t y)
{
    for (int guard = 0; guard < kUnionGuard; ++guard) {
        x = cfind(par, x);
        y = cfind(par, y);
        if (x == y) return true;
        const uint32_t hi = x > y ? x : y, lo = x > y ? y : x;
        if (atomicCAS(par + hi, hi, lo) == hi) return true;
    }
    return false;
}

__global__ void k_cut_count(const CutArgs a)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.n_inst) return;
    const bool batched = a.n_inst > 1;
    const int64_t lo = batched ? a.ebeg[b] : 0, hi = batched ? a.eend[b] : a.m;
    const int64_t nrows = batched ? a.inst_off[b + 1] - a.inst_off[b] : a.N;
    // the edges are key-ordered within the instance: D <= cap is a prefix
    int64_t l = lo, h = hi;
    while (l < h) {
        const int64_t mid = (l + h) >> 1;
        if (a.edges[mid].D <= a.cap2) l = mid + 1;
        else h = mid;
    }
    int64_t acc = l - lo;
    if (a.kl1 > 0) {
        const int64_t room = nrows > a.kl1 ? nrows - a.kl1 : 0;   // joins until KL1 clusters remain
        if (acc > room) acc = room;
    }
    a.cnt[b] = (unsigned long long)acc;
}

// exclusive prefix of the per-instance counts (one thread; instances number in the
// thousands at most)
__global__ void k_cut_offsets(const CutArgs a)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long run = 0;
    for (int64_t b = 0; b < a.n_inst; ++b) {
        const unsigned long long v = a.cnt[b];
        a.cnt[b] = run;
        run += v;
    }
    a.cnt[a.n_inst] = run;
    *a.n_merges = run;
}

// accepted edges in (instance, key) order -> merges (new sizes later) and the level
// state: labels = the endpoints, sizes 1
__global__ void k_cut_gather(const CutArgs a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.m) return;
    const nnm_edge ed = a.edges[p];
    const int64_t b = a.n_inst > 1 ? (int64_t)a.inst_of_row[ed.a] : 0;
    const int64_t q = p - (a.n_inst > 1 ? a.ebeg[b] : 0);
    const unsigned long long off = a.cnt[b];
    if (q >= (int64_t)(a.cnt[b + 1] - off)) return;
    const int64_t j = (int64_t)off + q;
    nnm_merge mg;
    mg.a = ed.a;
    mg.b = ed.b;
    mg.D = ed.D;
    mg.dist = a.metric == 0 ? sqrt(ed.D) : ed.D;
    mg.new_size = 0;
    a.merges[j] = mg;
    a.lab[2 * j] = ed.a;
    a.lab[2 * j + 1] = ed.b;
    a.w[2 * j] = 1u;
    a.w[2 * j + 1] = 1u;
}

// One level with ranges of h2 ranks.  A range whose high half is empty (the last one)
// takes no part.
__device__ __forceinline__ bool has_high_half(int64_t j, int64_t h2, int64_t M)
{
    return (j / h2) * h2 + h2 / 2 < M;
}

__global__ void k_lv_insert(const CutArgs a, int64_t M, int64_t h2)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * M) return;
    const int64_t j = q >> 1;
    if (!has_high_half(j, h2, M)) return;
    const uint32_t lab = a.lab[q];
    const unsigned long long key = ((unsigned long long)(j / h2) << 32) | lab;
    const uint64_t mask = (uint64_t)a.H - 1;
    uint64_t hs = mix64(key) & mask;
    // at most 2M keys in 4M or more slots: an empty slot or the key is always found
    for (int64_t probe = 0; probe < a.H; ++probe) {
        const unsigned long long prev = atomicCAS(a.hkey + hs, kEmptyKey, key);
        if (prev == kEmptyKey) {
            a.hpar[hs] = (uint32_t)hs;
            a.hw[hs] = a.w[q];
            a.hlab[hs] = lab;
            break;
        }
        if (prev == key) break;
        hs = (hs + 1) & mask;
    }
    a.slot[q] = (uint32_t)hs;
}

__global__ void k_lv_union(const CutArgs a, int64_t M, int64_t h2)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M || !has_high_half(j, h2, M)) return;
    if (j - (j / h2) * h2 >= h2 / 2) return;   // high half: no join at this level
    if (!cunion(a.hpar, a.slot[2 * j], a.slot[2 * j + 1])) atomicExch(a.err_flag, 1);
}

__global__ void k_lv_sum(const CutArgs a)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.H || a.hkey[s] == kEmptyKey) return;
    atomicAdd(a.hsum + cfind(a.hpar, (uint32_t)s), a.hw[s]);
}

__global__ void k_lv_relabel(const CutArgs a, int64_t M, int64_t h2)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    if (j - (j / h2) * h2 < h2 / 2) return;   // low half: labels stay
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const uint32_t r = cfind(a.hpar, a.slot[2 * j + side]);
        a.lab[2 * j + side] = a.hlab[r];
        a.w[2 * j + side] = a.hsum[r];
    }
}

__global__ void k_cut_sizes(const CutArgs a, int64_t M)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    a.merges[j].new_size = (int64_t)a.w[2 * j] + a.w[2 * j + 1];
}

__global__ void k_uf_init(uint32_t *par, int64_t N)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) par[i] = (uint32_t)i;
}

__global__ void k_uf_merges(const CutArgs a, int64_t M)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    if (!cunion(a.uf_parent, (uint32_t)a.merges[j].a, (uint32_t)a.merges[j].b)) atomicExch(a.err_flag, 1);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// ---------------------------------------------------------------------------------
// KL2 / KL3 without KL4 (one instance): most decisions without the walk.  With the
// unrestricted process's cluster sizes s_a, s_b just before each admissible edge (the
// cut's levels above, KL1 left out), an edge with s_a + s_b <= KL3 and s_a, s_b <= KL2 is
// joined whatever the restricted sizes are (they are no larger), and so is every edge
// below it in the merge tree (their sizes are smaller): these "safe" edges are joined,
// with new size s_a + s_b.  Everything above an unsafe edge is unsafe, so an unsafe
// edge's clusters are made only of edges below it: the union-find with every safe edge
// applied serves all unsafe edges, which the walk then decides in key order.  KL1 only
// cuts the accepted sequence after N - KL1 joins.
// ---------------------------------------------------------------------------------
__global__ void k_fw_mark(const FastWalkArgs f)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= f.M) return;
    const int64_t sa = f.w[2 * j], sb = f.w[2 * j + 1];
    const bool safe = (f.kl3 <= 0 || sa + sb <= f.kl3) && (f.kl2 <= 0 || (sa <= f.kl2 && sb <= f.kl2));
    f.dec[j] = safe ? 1 : 0;
    f.unsafe[j] = safe ? 0 : 1;
}

__global__ void k_fw_union_safe(const FastWalkArgs f)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= f.M || !f.dec[j]) return;
    if (!cunion(f.uf_parent, f.cand[j].a, f.cand[j].b)) atomicExch(f.err_flag, 1);
}

__global__ void k_fw_sizes(const FastWalkArgs f)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.N) return;
    atomicAdd(f.uf_size + cfind(f.uf_parent, (uint32_t)i), 1u);
}

__global__ void k_fw_gather_unsafe(const FastWalkArgs f, int64_t n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const nnm_merge m = f.cand[f.pos[t]];
    nnm_edge e;
    e.a = m.a;
    e.b = m.b;
    e.D = m.D;
    f.unsafe_edges[t] = e;
}

// an accepted unsafe edge back at its place among the admissible edges (keys are unique)
__global__ void k_fw_place(const FastWalkArgs f, int64_t n)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const nnm_merge m = f.walk_out[t];
    const long long dm = __double_as_longlong(m.D);
    int64_t lo = 0, hi = f.M;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const nnm_merge c = f.cand[mid];
        const long long dc = __double_as_longlong(c.D);
        const bool less = dc < dm || (dc == dm && (c.a < m.a || (c.a == m.a && c.b < m.b)));
        if (less) lo = mid + 1;
        else hi = mid;
    }
    if (lo < f.M && f.cand[lo].a == m.a && f.cand[lo].b == m.b) {
        f.dec[lo] = 1;
        f.cand[lo].new_size = m.new_size;
    } else {
        atomicExch(f.err_flag, 1);
    }
}

__global__ void k_fw_emit(const FastWalkArgs f, int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) f.merges[k] = f.cand[f.pos[k]];
}

}  // namespace

cudaError_t launch_fast_walk_steps(const FastWalkArgs &f, int step, int64_t n, cudaStream_t s)
{
    switch (step) {
    case 0:
        if (f.M > 0) k_fw_mark<<<blocks_for(f.M), kThreads, 0, s>>>(f);
        break;
    case 1:
        k_uf_init<<<blocks_for(f.N), kThreads, 0, s>>>(f.uf_parent, f.N);
        if (f.M > 0) k_fw_union_safe<<<blocks_for(f.M), kThreads, 0, s>>>(f);
        if (cudaMemsetAsync(f.uf_size, 0, (size_t)f.N * sizeof(uint32_t), s) != cudaSuccess) return cudaGetLastError();
        k_fw_sizes<<<blocks_for(f.N), kThreads, 0, s>>>(f);
        count_launches(1);
        break;
    case 2:
        if (n > 0) k_fw_gather_unsafe<<<blocks_for(n), kThreads, 0, s>>>(f, n);
        break;
    case 3:
        if (n > 0) k_fw_place<<<blocks_for(n), kThreads, 0, s>>>(f, n);
        break;
    case 4:
        if (n > 0) k_fw_emit<<<blocks_for(n), kThreads, 0, s>>>(f, n);
        break;
    case 5:
        // the final partition: the emitted joins only (KL1 may have cut the sequence)
        k_uf_init<<<blocks_for(f.N), kThreads, 0, s>>>(f.uf_parent, f.N);
        if (n > 0) {
            CutArgs a{};
            a.merges = f.merges;
            a.uf_parent = f.uf_parent;
            a.err_flag = f.err_flag;
            k_uf_merges<<<blocks_for(n), kThreads, 0, s>>>(a, n);
            count_launches(1);
        }
        break;
    default:
        return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

namespace {
}  // namespace

int64_t cut_hash_slots(int64_t m)
{
    int64_t H = 1024;
    while (H < 4 * m) H <<= 1;
    return H;
}

cudaError_t launch_restrict_cut(const CutArgs &a, int64_t *n_merges_host, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    k_cut_count<<<blocks_for(a.n_inst), kThreads, 0, s>>>(a);
    k_cut_offsets<<<1, 32, 0, s>>>(a);
    count_launches(2);
    if (a.m > 0) {
        k_cut_gather<<<blocks_for(a.m), kThreads, 0, s>>>(a);
        count_launches(1);
    }
    unsigned long long Mh = 0;
    e = cudaMemcpyAsync(&Mh, a.n_merges, sizeof Mh, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const int64_t M = (int64_t)Mh;
    *n_merges_host = M;
    int64_t h2 = 2;
    while (h2 < M) h2 <<= 1;   // one range holds every rank
    for (; M > 1 && h2 >= 2; h2 >>= 1) {
        e = cudaMemsetAsync(a.hkey, 0xFF, (size_t)a.H * sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.hsum, 0, (size_t)a.H * sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        k_lv_insert<<<blocks_for(2 * M), kThreads, 0, s>>>(a, M, h2);
        k_lv_union<<<blocks_for(M), kThreads, 0, s>>>(a, M, h2);
        k_lv_sum<<<blocks_for(a.H), kThreads, 0, s>>>(a);
        k_lv_relabel<<<blocks_for(M), kThreads, 0, s>>>(a, M, h2);
        count_launches(4);
    }
    k_uf_init<<<blocks_for(a.N), kThreads, 0, s>>>(a.uf_parent, a.N);
    count_launches(1);
    if (M > 0) {
        k_cut_sizes<<<blocks_for(M), kThreads, 0, s>>>(a, M);
        k_uf_merges<<<blocks_for(M), kThreads, 0, s>>>(a, M);
        count_launches(2);
    }
    return cudaGetLastError();
}

}  // namespace nnm
