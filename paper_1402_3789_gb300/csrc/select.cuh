// select.cuh -- per-row candidate selection shared by the two sweep kernels.
//
// The re-rank needs, for each row, every column whose candidate value v is at most
// T(v_k), where v_k is the k-th smallest value and T the proven error bound around it
// (see rerank.cu).  A sweep therefore keeps, per row and column range:
//   - the KC smallest values seen so far, sorted, in registers (KC >= k), and
//   - a "band" of up to CB further values that are still <= T(current KC-th), in
//     shared memory (CB is chosen per kernel: narrow for FP32, wide for 16-bit).
// The fast-path threshold of the row is T(current KC-th value): it only falls, so a
// value above it can never be needed.  When the band is full it is compacted against
// the current threshold; if it is still full the row is flagged (the re-rank then sends
// it to the collect pass).  All bounds here are computed in FP32 rounded upwards, and
// enlarged by 2^-20, so that they dominate the binary64 bound of the re-rank.
#pragma once

#include "nnm_internal.cuh"

namespace nnm {

constexpr int kTop = 16;                    // register slots per row in the output record
constexpr int kBandMax = kListC - kTop;     // band slots per row in the output record

// Per-row constants (tensor path): eps = gamma (P_i + Pmax)^2 + E_i + Emax, rr = r_i + R.
struct RowConst {
    float eps, rr;
};

__device__ __forceinline__ RowConst make_rowconst(const SelConst &c, const Margin &m, uint32_t i)
{
    RowConst rc{0.f, 0.f};
    if (c.tensor) {
        const float p = __fadd_ru(m.P[i], c.Pmax);
        rc.eps = __fadd_ru(__fadd_ru(__fmul_ru(c.gamma, __fmul_ru(p, p)), m.E[i]), c.Emax);
        rc.rr = __fadd_ru(m.r[i], c.R);
    }
    return rc;
}

// Upper bound on T(vk) of the re-rank (same formula, FP32 rounded up, enlarged).
__device__ __forceinline__ float sel_threshold(const SelConst &c, const RowConst &rc, float vk)
{
    if (!(vk < INFINITY)) return INFINITY;
    const float g = 1.0f + 0x1p-20f;
    if (!c.tensor) return __fadd_ru(__fmul_ru(__fadd_ru(vk, c.c0), c.c1), c.c0);
    const float s = __fsqrt_ru(fmaxf(__fadd_ru(vk, rc.eps), 0.0f));
    const float U = __fmul_ru(__fadd_ru(s, rc.rr), g);
    const float W = __fadd_ru(U, rc.rr);
    return __fmul_ru(__fadd_ru(__fmul_ru(W, W), rc.eps), g);
}

// Append (v, j) to a row's band (entry m at bv[m * stride]); when it is full, first
// drop the entries above thr.  Returns the new count, or -1 if it is still full.
static __device__ __noinline__ int band_push(float v, uint32_t j, int bcnt, int cap, float thr, float *bv, uint32_t *bj,
                                             int stride)
{
    if (bcnt == cap) {
        int w = 0;
        for (int m = 0; m < cap; ++m) {
            const float x = bv[m * stride];
            if (x <= thr) {
                bv[w * stride] = x;
                bj[w * stride] = bj[m * stride];
                ++w;
            }
        }
        bcnt = w;
        if (bcnt == cap) return -1;
    }
    bv[bcnt * stride] = v;
    bj[bcnt * stride] = j;
    return bcnt + 1;
}

// Threshold shared by the column ranges (CTAs) of one row: any range's bound T is a
// valid bound for every range (the final T uses the k-th smallest over all ranges, which
// is no larger), so each range may prune at the smallest one published.  Stored as the
// bits of a non-negative float (unsigned order = float order); all ones = none yet.
__device__ __forceinline__ float shared_thr_exchange(unsigned int *slot_bits, float own)
{
    if (own >= 0.0f && own < INFINITY) atomicMin(slot_bits, __float_as_uint(own));
    const unsigned int g = *reinterpret_cast<volatile unsigned int *>(slot_bits);
    return g == 0xFFFFFFFFu ? INFINITY : __uint_as_float(g);
}

template <int KC, int CB>
struct RowSel {
    static_assert(CB <= kBandMax, "band larger than the output record");
    float tv[KC];
    uint32_t tj[KC];
    float thr;   // values above thr are never needed
    float ext;   // bound learnt from the row's other column ranges
    int bcnt;
    int bovf;

    __device__ __forceinline__ void init(bool valid)
    {
#pragma unroll
        for (int m = 0; m < KC; ++m) {
            tv[m] = INFINITY;
            tj[m] = kInvalid;
        }
        thr = valid ? INFINITY : -INFINITY;
        ext = INFINITY;
        bcnt = 0;
        bovf = 0;
    }

    // tighten with a bound from another column range of the same row
    __device__ __forceinline__ void bound(float g)
    {
        ext = fminf(ext, g);
        thr = fminf(thr, ext);
    }

    // v <= thr and column j eligible.
    __device__ __forceinline__ void insert(float v, uint32_t j, const SelConst &c, const RowConst &rc, float *bv,
                                           uint32_t *bj, int stride)
    {
        if (v < tv[KC - 1]) {
            // bubble (v, j) into place; what the bubble carries out of the end is the
            // entry that leaves the list (with ties that need not be the old last one)
#pragma unroll
            for (int m = 0; m < KC; ++m) {
                const bool sw = v < tv[m];
                const float x = sw ? tv[m] : v;
                const uint32_t y = sw ? tj[m] : j;
                tv[m] = sw ? v : tv[m];
                tj[m] = sw ? j : tj[m];
                v = x;
                j = y;
            }
            thr = fminf(sel_threshold(c, rc, tv[KC - 1]), ext);
            if (j != kInvalid && v <= thr) push(v, j, bv, bj, stride);
        } else {
            push(v, j, bv, bj, stride);
        }
    }

    __device__ __forceinline__ void push(float v, uint32_t j, float *bv, uint32_t *bj, int stride)
    {
        const int r = band_push(v, j, bcnt, CB, thr, bv, bj, stride);
        if (r < 0) {
            bovf = 1;
            thr = -INFINITY;   // flagged: nothing more is needed from this sweep
        } else {
            bcnt = r;
        }
    }

    // Output record: kTop top slots (KC used), kBandMax band slots (CB used); overflow
    // flag separately.
    __device__ __forceinline__ void write(float *ov, uint32_t *oj, uint8_t *oflag, const float *bv, const uint32_t *bj,
                                          int stride)
    {
#pragma unroll
        for (int m = 0; m < kTop; ++m) {
            ov[m] = m < KC ? tv[m < KC ? m : 0] : INFINITY;
            oj[m] = m < KC ? tj[m < KC ? m : 0] : kInvalid;
        }
        for (int m = 0; m < kBandMax; ++m) {
            const bool ok = m < bcnt && !bovf;
            ov[kTop + m] = ok ? bv[m * stride] : INFINITY;
            oj[kTop + m] = ok ? bj[m * stride] : kInvalid;
        }
        *oflag = (uint8_t)bovf;
    }
};

}  // namespace nnm
