// peaks.cu -- measured arithmetic peaks for the roofline denominators of the FP32 direct
// sweep (FP32 FMA pipe) and of the binary64 re-rank (FP64 pipe).  Not part of the
// method: a separate small library (libnnm_peaks.so) that bench.py calls before its
// timed region.
//
// Each thread runs kChains independent FMA chains (enough to cover the pipe latency)
// for `iters` rounds; every SM gets `blocks_per_sm` blocks of 256 threads.  Flops =
// 2 per FMA.  The result of every chain is folded into one store per thread behind a
// data-dependent test, so the compiler keeps every FMA.  Timed with CUDA events on one
// stream after one warm-up launch.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(T *out, int iters, T b, T c)
{
    T acc[kChains];
#pragma unroll
    for (int q = 0; q < kChains; ++q) acc[q] = (T)(threadIdx.x + q) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int q = 0; q < kChains; ++q) acc[q] = fma(acc[q], b, c);
        }
    }
    T s = 0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += acc[q];
    if (s == (T)-1.2345) out[blockIdx.x * kThreads + threadIdx.x] = s;   // never true; keeps the chains
}

template <typename T>
int measure(int blocks_per_sm, int iters, double *tflops, double *ms_out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * blocks_per_sm;
    T *out = nullptr;
    if (cudaMalloc((void **)&out, (size_t)blocks * kThreads * sizeof(T)) != cudaSuccess) return 2;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreate(&s);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b slightly below 1 and c small keep the values finite and normal
    k_fma_chain<T><<<blocks, kThreads, 0, s>>>(out, iters / 4 + 1, (T)0.999999, (T)1e-7);
    cudaEventRecord(e0, s);
    k_fma_chain<T><<<blocks, kThreads, 0, s>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(out);
    if (e != cudaSuccess) return 3;
    const double fmas = (double)blocks * kThreads * iters * 16.0 * kChains;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
    *ms_out = ms;
    return 0;
}

}  // namespace

extern "C" {

// FP32 FMA throughput of the whole GPU in TFLOP/s (2 flops per FMA); 0 on success.
int nnm_peak_fp32(int blocks_per_sm, int iters, double *tflops, double *ms)
{
    if (blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || !tflops || !ms) return 1;
    return measure<float>(blocks_per_sm, iters, tflops, ms);
}

// FP64 FMA throughput of the whole GPU in TFLOP/s (2 flops per FMA); 0 on success.
int nnm_peak_fp64(int blocks_per_sm, int iters, double *tflops, double *ms)
{
    if (blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || !tflops || !ms) return 1;
    return measure<double>(blocks_per_sm, iters, tflops, ms);
}

}  // extern "C"
