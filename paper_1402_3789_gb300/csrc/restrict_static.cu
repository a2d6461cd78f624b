// restrict_static.cu -- nnm_restrict_static: the restriction walk and labels on a given
// merge tree, with every scratch buffer in one fixed device array instead of memory
// obtained from cudaMalloc.
//
// Some callers cannot allocate device memory at call time: applications whose device
// memory is owned by a pool or arena that must not see foreign cudaMalloc/cudaFree
// calls (those synchronise the device and fragment the pool), and services that fix
// their memory budget when they start.  This entry point serves them: the caller passes
// the tree, the restrictions and the output buffers; the walk's union-find, deferral
// list, label scratch and counters live in g_static_scratch below.
//
// Consequences of the fixed array:
//   - every GPU that loads this library holds it (kStaticBytes) until the process exits;
//   - N is limited to NNM_STATIC_MAX_ROWS rows; larger N is rejected before any launch;
//   - all calls share it: calls whose work overlaps on the GPU (different streams, or
//     different host threads without ordering) race and corrupt each other's results;
//     calls ordered on one stream are safe, each starts from its own initialisation;
//   - the first call on a device looks up the array's device address (once per device,
//     with that device current); make that first call before any stream capture;
//   - the caller's tree is checked on the device (endpoints below N, key order) before
//     the walk indexes the union-find with its endpoints; a bad tree gives NNM_EINVAL.
#include <mutex>

#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr int64_t kStaticMaxRows = NNM_STATIC_MAX_ROWS;
constexpr int64_t kStaticBlocks = (kStaticMaxRows + 255) / 256;
// layout (uint32 words): uf_parent, uf_size, deferred, minm, flag [kStaticMaxRows each],
// block_sums [kStaticBlocks], then two 64-bit counters (n_merges, K) and the tree-check
// word (bit 0: an endpoint >= N, bit 1: a == b or a > b, bit 2: D not finite and >= 0,
// bit 3: keys not strictly increasing), padded to 8 bytes
constexpr int64_t kCounterWord = 5 * kStaticMaxRows + kStaticBlocks;
constexpr int64_t kWords = kCounterWord + 6;
constexpr size_t kStaticBytes = (size_t)kWords * 4;
static_assert(kCounterWord % 2 == 0, "64-bit counters stay aligned");
static_assert(kStaticBytes < (size_t)24 << 20, "the fixed scratch array stays modest (~21 MB)");

static __device__ __align__(256) uint32_t g_static_scratch[kWords];

// The caller's tree is checked before the walk reads the union-find at its endpoints:
// every endpoint below N, a < b, D finite and non-negative, and keys (D, a, b) strictly
// increasing along the array (a tree grouped by instance, as a batched context returns
// it, is not in key order across groups and fails here).  Violations set bits of *err.
__global__ void k_check_tree(const nnm_edge *__restrict__ e, int64_t m, int64_t N, uint32_t *err)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    const nnm_edge x = e[q];
    uint32_t bits = 0;
    if ((int64_t)x.a >= N || (int64_t)x.b >= N) bits |= 1u;
    if (x.a >= x.b) bits |= 2u;
    if (!(x.D >= 0.0 && x.D < INFINITY)) bits |= 4u;
    if (q + 1 < m) {
        const nnm_edge y = e[q + 1];
        const bool inc = x.D < y.D || (x.D == y.D && (x.a < y.a || (x.a == y.a && x.b < y.b)));
        if (!inc) bits |= 8u;
    }
    if (bits) atomicOr(err, bits);
}

// Device address of g_static_scratch per device (host code may not use the symbol's
// host-side stand-in as a pointer).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_addr[kMaxDevices] = {};

cudaError_t scratch_address(uint32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace nnm

using namespace nnm;

extern "C" nnm_status nnm_restrict_static(const nnm_edge *tree_dev, int64_t n_edges, int64_t N,
                                          nnm_metric metric, const nnm_restrictions *restrictions,
                                          nnm_merge *merges_dev, int64_t *n_merges_host, int32_t *labels_dev,
                                          int64_t *n_clusters_host, void *cuda_stream)
{
    if (!tree_dev || !merges_dev || !n_merges_host || !labels_dev || !n_clusters_host) return NNM_EINVAL;
    if (N < 2 || n_edges < 0 || n_edges > N - 1) return NNM_EINVAL;
    if (metric != NNM_EUCLIDEAN && metric != NNM_MANHATTAN && metric != NNM_CHEBYSHEV) return NNM_EINVAL;
    if (N > kStaticMaxRows) return NNM_EUNSUPPORTED;   // beyond the fixed scratch array
    nnm_restrictions r{};
    if (restrictions) r = *restrictions;
    if (r.semantics == 1) return NNM_EUNSUPPORTED;
    if (r.semantics != 0) return NNM_EINVAL;
    if (isnan(r.max_join_dist) || r.kl1_stop_clusters < 0 || r.kl2_max_pre_size < 0 || r.kl3_max_size < 0 ||
        r.kl4_min_size < 0)
        return NNM_EINVAL;
    if (r.kl2_max_pre_size > 0 && r.kl3_max_size > 0 && r.kl3_max_size <= r.kl2_max_pre_size) return NNM_EINVAL;

    uint32_t *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return NNM_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(base + kCounterWord);
    uint32_t *check = base + kCounterWord + 4;
    // the counters and the check word are the only state read before being written
    if (cudaMemsetAsync(counters, 0, 6 * sizeof(uint32_t), s) != cudaSuccess) return NNM_ECUDA;
    if (n_edges > 0) {
        k_check_tree<<<(unsigned)((n_edges + 255) / 256), 256, 0, s>>>(tree_dev, n_edges, N, check);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return NNM_ECUDA;
        uint32_t bad = 0;
        if (cudaMemcpyAsync(&bad, check, sizeof bad, cudaMemcpyDeviceToHost, s) != cudaSuccess) return NNM_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return NNM_ECUDA;
        if (bad) return NNM_EINVAL;   // nothing was walked; the array holds no result
    }

    RestrictArgs ra{};
    ra.edges = tree_dev;
    ra.m = n_edges;
    ra.N = N;
    // the cap in D units, as nnm_cluster: squared for the squared Euclidean D
    ra.cap2 = (r.max_join_dist > 0.0 && isfinite(r.max_join_dist))
                  ? (metric == NNM_EUCLIDEAN ? r.max_join_dist * r.max_join_dist : r.max_join_dist)
                  : INFINITY;
    ra.metric = (int)metric;
    ra.kl1 = r.kl1_stop_clusters;
    ra.kl2 = r.kl2_max_pre_size;
    ra.kl3 = r.kl3_max_size;
    ra.kl4 = r.kl4_min_size;
    ra.uf_parent = base;
    ra.uf_size = base + kStaticMaxRows;
    ra.deferred = base + 2 * kStaticMaxRows;
    ra.merges = merges_dev;
    ra.n_merges = &counters[0];
    if (launch_restrict(ra, s) != cudaSuccess) return NNM_ECUDA;

    LabelArgs la{};
    la.N = N;
    la.uf_parent = base;
    la.minm = base + 3 * kStaticMaxRows;
    la.flag = base + 4 * kStaticMaxRows;
    la.block_sums = base + 5 * kStaticMaxRows;
    la.labels = labels_dev;
    la.K = &counters[1];
    if (launch_labels(la, s) != cudaSuccess) return NNM_ECUDA;

    unsigned long long h[2] = {0, 0};
    if (cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return NNM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return NNM_ECUDA;
    *n_merges_host = (int64_t)h[0];
    *n_clusters_host = (int64_t)h[1];
    return NNM_OK;
}
