// sort.cu -- K6: device merge sort of the merge-tree edges by key (D, a, b).
//
// The paper sorts the selected minimal pairs by distance before joining clusters
// ("General description of the algorithm for constructing the set of minimum
// distances"); the restriction walk needs the whole tree in that order.  Blocks first
// sort runs of 2048 edges in shared memory (bitonic network), then merge passes double
// the run length; each thread places 8 outputs after a merge-path binary search.
#include "nnm_internal.cuh"

namespace nnm {

namespace {

constexpr int kSortThreads = 256;
constexpr int kRun = 2048;
constexpr int kPer = 8;

// Key order (D, a, b); D >= 0 compares as its bit pattern (an integer compare: the FP64
// pipe is narrow).  With a major key per row (the instance of a batched context), edges
// are first ordered by the major key of their endpoint a.
__device__ __forceinline__ bool edge_less(const nnm_edge &x, const nnm_edge &y, const uint32_t *major)
{
    if (major) {
        const uint32_t mx = x.a == 0xFFFFFFFFu ? 0xFFFFFFFFu : major[x.a];
        const uint32_t my = y.a == 0xFFFFFFFFu ? 0xFFFFFFFFu : major[y.a];
        if (mx != my) return mx < my;
    }
    const long long dx = __double_as_longlong(x.D), dy = __double_as_longlong(y.D);
    if (dx != dy) return dx < dy;
    if (x.a != y.a) return x.a < y.a;
    return x.b < y.b;
}

__device__ __forceinline__ nnm_edge max_edge()
{
    nnm_edge e;
    e.a = 0xFFFFFFFFu;
    e.b = 0xFFFFFFFFu;
    e.D = INFINITY;
    return e;
}

__global__ void __launch_bounds__(kSortThreads) k_block_sort(nnm_edge *e, int64_t m, const uint32_t *major)
{
    __shared__ nnm_edge s[kRun];
    const int64_t base = (int64_t)blockIdx.x * kRun;
    for (int q = threadIdx.x; q < kRun; q += kSortThreads) s[q] = base + q < m ? e[base + q] : max_edge();
    __syncthreads();
    for (int k = 2; k <= kRun; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int q = threadIdx.x; q < kRun; q += kSortThreads) {
                const int p = q ^ j;
                if (p > q) {
                    const bool up = (q & k) == 0;
                    nnm_edge x = s[q], y = s[p];
                    if (edge_less(y, x, major) == up) {
                        s[q] = y;
                        s[p] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int q = threadIdx.x; q < kRun; q += kSortThreads)
        if (base + q < m) e[base + q] = s[q];
}

// Merge adjacent sorted runs of length w from src into dst.
__global__ void __launch_bounds__(kSortThreads) k_merge_pass(const nnm_edge *__restrict__ src,
                                                             nnm_edge *__restrict__ dst, int64_t m, int64_t w,
                                                             const uint32_t *major)
{
    const int64_t p0 = ((int64_t)blockIdx.x * kSortThreads + threadIdx.x) * kPer;
    if (p0 >= m) return;
    const int64_t pair = p0 / (2 * w);
    const int64_t a0 = pair * 2 * w;
    const int64_t lenA = (a0 + w < m ? w : m - a0);
    const int64_t b0 = a0 + lenA;
    const int64_t lenB = b0 + w < m ? w : (m > b0 ? m - b0 : 0);
    const nnm_edge *A = src + a0;
    const nnm_edge *B = src + b0;
    const int64_t o = p0 - a0;
    int64_t lo = o - lenB > 0 ? o - lenB : 0, hi = o < lenA ? o : lenA;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (edge_less(B[o - mid - 1], A[mid], major)) hi = mid;
        else lo = mid + 1;
    }
    int64_t i = lo, j = o - lo;
    for (int t = 0; t < kPer && p0 + t < m && p0 + t < a0 + lenA + lenB; ++t) {
        nnm_edge x;
        if (j >= lenB || (i < lenA && edge_less(A[i], B[j], major))) x = A[i++];
        else x = B[j++];
        dst[p0 + t] = x;
    }
}

}  // namespace

cudaError_t launch_sort_edges(nnm_edge *e, nnm_edge *tmp, int64_t m, cudaStream_t s, nnm_edge **sorted_out,
                              const uint32_t *major)
{
    *sorted_out = e;
    if (m <= 1) return cudaSuccess;
    const unsigned blocks = (unsigned)((m + kRun - 1) / kRun);
    k_block_sort<<<blocks, kSortThreads, 0, s>>>(e, m, major);
    count_launches(1);
    nnm_edge *src = e, *dst = tmp;
    for (int64_t w = kRun; w < m; w *= 2) {
        const int64_t threads = (m + kPer - 1) / kPer;
        k_merge_pass<<<(unsigned)((threads + kSortThreads - 1) / kSortThreads), kSortThreads, 0, s>>>(src, dst, m, w,
                                                                                                     major);
        count_launches(1);
        nnm_edge *t = src;
        src = dst;
        dst = t;
    }
    *sorted_out = src;
    return cudaGetLastError();
}

}  // namespace nnm
