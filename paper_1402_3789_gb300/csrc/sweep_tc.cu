// sweep_tc.cu -- K2: all-pairs candidate sweep on the 5th-generation tensor cores.
//
// Candidate values c~(i,j) = |x_hat_i - x_hat_j|^2 come out of one tcgen05 MMA chain
// per tile: the row operand A_i = [x_hat_i, 1,1,1, a_i] and column operand
// B_j = [-2 x_hat_j, a_j, 1,1,1] (prepared by k_tc_operands, K padded to kpad) give
// |x_hat_i|^2 + |x_hat_j|^2 - 2 x_hat_i.x_hat_j directly in the FP32 accumulator, so
// the epilogue is a compare against the row's threshold (a 3-input min over 32
// values, then the rare slow path) -- distances and minimum selection fused, the
// paper's second and third parallel items.
//
// CTA = 256 rows (two M=128 MMAs sharing each B tile) x one column range, 384 threads:
//   warps 0-7  epilogue, one row per thread (TMEM lane quadrant = warp % 4, half = warp / 4)
//   warp 8     MMA issuer (one elected thread); also allocates / frees TMEM
//   warp 9     producer: 1-D bulk copies (cp.async.bulk) of 128-column B tiles into an
//              S-stage shared-memory ring; the operand is stored in HBM already in the
//              core-matrix layout the MMA reads, so each tile is one contiguous copy.
//   warps 10-11 planners: bound tests that decide the column tiles, each for half of the
//              column blocks, ahead of the producer through shared-memory queues.
// TMEM: 512 columns = 2 accumulator buffers x 2 row halves x 128 columns (fp32).
// Every wait is bounded (global timer); on time-out the CTA raises the error flag,
// drains its own copies and MMAs with bounded waits, frees TMEM and exits.
#include "select.cuh"

namespace nnm {

namespace {

constexpr int kEpiWarps = 8;
constexpr int kThreadsTc = (kEpiWarps + 4) * 32;
constexpr int kMmaWarp = 8;
constexpr int kProdWarp = 9;
constexpr int kPlanWarp = 10;     // planners: warps 10 and 11
constexpr int kPlanners = 2;
constexpr int kPlanQ = 1024;      // planned tiles: two queues of kPlanQh, one per planner
constexpr int kPlanQh = kPlanQ / kPlanners;
constexpr int kBN = 128;          // columns per B tile
constexpr int kBlkTiles = 32;     // tiles per column block (one bounding sphere per block)
constexpr int kMaxStages = 8;
constexpr int kMaxKSteps = 6;     // K steps of 16 per tile: kpad <= 96 (split BF16 at d <= 30)
constexpr int kBandWide = 64;   // band slots per row for one-term BF16 (a wide band)
constexpr int kInfoQ = kMaxStages + 2;   // tile records in flight: the ring's stages plus the two TMEM buffers
// Waits for work (stages, accumulators, plan entries, thresholds) give up after the
// caller's limit (SweepArgs::wait_ns, 2 s by default).  The drain waits at the end --
// copies and MMAs this CTA issued, which must land before its shared memory and TMEM
// are released -- keep their own fixed bound, so a short limit never cuts them.
constexpr uint64_t kDrainNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase parity by the whole warp: every lane polls and the warp
// decides together, so that no lane waits alone while the others stall at the next
// warp-wide operation (a lone waiting lane cost about a thousand cycles per wait).  Every
// lane observes the completed phase itself (acquire).  Returns false if the wait gave up
// (time-out, or another role of this CTA already aborted).
__device__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, volatile int *abort_flag, uint64_t wait_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        if (it == 0) t0 = global_ns();
        if ((it & 15) == 15) {
            const int give_up = __shfl_sync(0xffffffffu, (int)(*abort_flag != 0 || global_ns() - t0 > wait_ns), 0);
            if (give_up) return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, no swizzle (canonical core-matrix layout):
// start >> 4 | LBO (K-direction core-matrix stride) >> 4 << 16 | SBO (8-row-group
// stride) >> 4 << 32 | version 1 << 46 | layout SWIZZLE_NONE (0) << 61.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A/B = F16 (0) or BF16 (1), both K-major,
// N = 128, M = 128.
__device__ __forceinline__ uint32_t instr_desc(int fp16)
{
    const uint32_t fmt = fp16 ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The MMAs of one tile: KS steps of K = 16 into the two row halves' accumulators
// (columns d0 and d0 + kBN), each chain starting with accumulate = 0.  KS is a template
// argument so that the issuing thread runs straight-line code (a runtime bound on an
// unrolled loop cost about sixty cycles per step slot, issued or not).
template <int KS>
__device__ __forceinline__ void mma_tile(uint32_t d0, uint64_t a0, uint64_t a1, uint64_t b0, uint32_t idesc);

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

template <int KS>
__device__ __forceinline__ void mma_tile(uint32_t d0, uint64_t a0, uint64_t a1, uint64_t b0, uint32_t idesc)
{
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) mma_f16(d0, a0 + 16u * kk, b0 + 16u * kk, idesc, kk > 0 ? 1u : 0u);
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) mma_f16(d0 + kBN, a1 + 16u * kk, b0 + 16u * kk, idesc, kk > 0 ? 1u : 0u);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

// Wait for this thread's tcgen05.ld results.  The 32 registers are tied to the wait as
// read-write operands so that no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
          "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]),
          "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]),
          "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
        :
        : "memory");
}

// w[q] for a q known only at run time, without local memory: a five-level selection
// by the bits of q (31 selects).
__device__ __forceinline__ uint32_t pick32(const uint32_t (&w)[32], int q)
{
    uint32_t a[16], b[8], c[4], d[2];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = (q & 1) ? w[2 * i + 1] : w[2 * i];
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = (q & 2) ? a[2 * i + 1] : a[2 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = (q & 4) ? b[2 * i + 1] : b[2 * i];
#pragma unroll
    for (int i = 0; i < 2; ++i) d[i] = (q & 8) ? c[2 * i + 1] : c[2 * i];
    return (q & 16) ? d[1] : d[0];
}

// Order-only barrier for 32 more registers after a wait (asm volatile keeps the order).
__device__ __forceinline__ void reg_fence(uint32_t (&v)[32])
{
    asm volatile(""
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                   "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]),
                   "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}


struct __align__(8) TcShared {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
    // Record of the q-th staged tile at q % kInfoQ, written by the producer and read by
    // the MMA warp and the epilogue: the producer is at most kStages tiles ahead of the
    // MMAs and those at most two ahead of the epilogue, so a record is read before it is
    // written again.
    int info_tile[kInfoQ];              // column tile (-1: end of the sequence)
    unsigned int info_mask[kInfoQ];     // epilogue warps that need the tile
    uint32_t info_comp[kInfoQ];         // masked sweeps: the tile's component (kInvalid: mixed)
    float warp_thr[kEpiWarps];   // largest row threshold of each epilogue warp
    float cR[2][32];             // row tile spheres (part 0: the first landmark group of the
    unsigned int rho_bits[2];    // tile's rows, part 1: the rest): centres, radii,
    unsigned int ymax_bits;      // largest |y| (float bits) and row counts
    int nvalid[2];
    unsigned int warps_in[2];    // epilogue warps holding rows of each part (bit masks)
    int npub;                    // epilogue warps that have published a threshold
    int plan_ct[kPlanQ];         // planned column tiles (-1: end), a ring of kPlanQh per planner ...
    unsigned int plan_mask[kPlanQ];   // ... with the epilogue warps that need them
    uint32_t plan_comp[kPlanQ];       // ... and, in masked sweeps, the tile's component
    int plan_head[kPlanners], plan_tail[kPlanners];
    unsigned int lup_bits[2];    // largest landmark distance bound of each row part    // entries written by the planner / taken by the producer
    unsigned int cmin, cmax;     // smallest and largest component among the tile's rows
};
constexpr int kShBytes = 16384;
static_assert(sizeof(TcShared) <= kShBytes, "shared control block");

// Shared-memory stages of the B ring that fit next to the other regions.
__host__ __device__ inline int tc_stages(int kpad, int band)
{
    const size_t fixed = (size_t)kRowTile * kpad * 2 + kShBytes + (size_t)band * kRowTile * 8 +
                         1024;
    const size_t per = (size_t)kBN * kpad * 2;
    int s = (int)((225 * 1024 - fixed) / per);
    return s > kMaxStages ? kMaxStages : s;
}

template <int KC, int CB, bool COLLECT>
__global__ void __launch_bounds__(kThreadsTc, 1) k_sweep_tc(const SweepArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const int kpad = a.kpad;
    const int kStages = tc_stages(kpad, CB);
    const uint32_t a_bytes = (uint32_t)kRowTile * kpad * 2;
    const uint32_t b_bytes = (uint32_t)kBN * kpad * 2;
    uint8_t *sA = smem_raw;
    uint8_t *sB = smem_raw + a_bytes;
    TcShared *sh = reinterpret_cast<TcShared *>(sB + (size_t)kStages * b_bytes);
    float *band_v = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(sh) + kShBytes);   // [CB][256]
    uint32_t *band_j = reinterpret_cast<uint32_t *>(band_v + CB * kRowTile);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    const int64_t slot0 = (int64_t)blockIdx.x * kRowTile;
    // The column tiles this row tile may meet: all of them, or in a batched context the
    // tiles of its rows' instances, [rtb, rte).  They are taken in blocks of kBlkTiles
    // consecutive tiles (a block has a bounding sphere of its own), blocks in cyclic order
    // starting at this row tile's own block (near neighbours first, so thresholds fall
    // early); split s takes the s-th range of that order.
    const int ntile_all = (int)((a.N + kBN - 1) / kBN);
    const int64_t p_first = a.rows ? a.rows[slot0] : slot0;
    int rtb = 0, rte = ntile_all;
    if (a.inst_pos) {
        const int64_t last = (slot0 + kRowTile < a.nslots ? slot0 + kRowTile : a.nslots) - 1;
        const int64_t p_last = a.rows ? a.rows[last] : last;
        rtb = (int)(a.inst_off[a.inst_pos[p_first]] / kBN);
        rte = (int)((a.inst_off[a.inst_pos[p_last] + 1] + kBN - 1) / kBN);
    }
    const int rbb = rtb / kBlkTiles;
    const int nblk_all = (rte + kBlkTiles - 1) / kBlkTiles - rbb;   // blocks of the range
    const int tile0 = (int)(p_first / kBN);
    const int bps = (nblk_all + a.splits - 1) / a.splits;
    const int b_begin = split * bps;
    const int b_end = b_begin + bps < nblk_all ? b_begin + bps : nblk_all;
    const int nblk = b_end > b_begin ? b_end - b_begin : 0;
    const int bstart = (tile0 / kBlkTiles - rbb + b_begin) % nblk_all;
    auto blk_at = [&](int u) -> int { return rbb + (bstart + u >= nblk_all ? bstart + u - nblk_all : bstart + u); };
    // tiles of block cb inside the range
    auto blk_tiles = [&](int cb) -> int {
        const int lo = cb * kBlkTiles > rtb ? cb * kBlkTiles : rtb;
        const int hi = cb * kBlkTiles + kBlkTiles < rte ? cb * kBlkTiles + kBlkTiles : rte;
        return hi > lo ? hi - lo : 0;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->tfull[b], 2);   // the MMA completion and the tile number
            mbar_init(&sh->tempty[b], kEpiWarps);
        }
        mbar_init(&sh->drain, 1);
        sh->abort_flag = 0;
        for (int w = 0; w < kEpiWarps; ++w) sh->warp_thr[w] = INFINITY;
        for (int k = 0; k < 32; ++k) sh->cR[0][k] = sh->cR[1][k] = 0.0f;
        sh->rho_bits[0] = sh->rho_bits[1] = 0u;
        sh->lup_bits[0] = sh->lup_bits[1] = 0u;
        sh->ymax_bits = 0u;
        sh->nvalid[0] = sh->nvalid[1] = 0;
        sh->warps_in[0] = sh->warps_in[1] = 0u;
        sh->npub = 0;
        for (int p = 0; p < kPlanners; ++p) sh->plan_head[p] = sh->plan_tail[p] = 0;
        sh->cmin = 0xFFFFFFFFu;
        sh->cmax = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32(&sh->tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }

    __syncthreads();
    // Row operand tile: 256 rows gathered (a row list, or consecutive rows) into the
    // interleaved layout by the epilogue threads; with pruning, also the bounding sphere
    // of the tile's rows (centre = mean of y, radius = largest distance to it).
    int myrow_slot = -1;
    uint32_t myrow = 0, mycomp = 0;
    int part = 0;   // sphere part of this thread's row
    float yv[32];
    if (warp < kEpiWarps) {
        const int r = (warp >> 2) * 128 + (warp & 3) * 32 + lane;   // row within the tile
        const int64_t slot = slot0 + r;
        const int chunks = kpad >> 3;
        uint4 *dst = reinterpret_cast<uint4 *>(sA);
        if (slot < a.nslots) {
            myrow_slot = r;
            myrow = a.rows ? a.rows[slot] : (uint32_t)slot;   // position
            mycomp = a.comp ? a.comp_pos[myrow] : 0u;
            if (a.comp) {
                atomicMin(&sh->cmin, mycomp);
                atomicMax(&sh->cmax, mycomp);
            }
            const uint4 *src = reinterpret_cast<const uint4 *>(a.XA);
            for (int c = 0; c < chunks; ++c)
                dst[((r >> 3) * chunks + c) * 8 + (r & 7)] = src[(((int64_t)myrow >> 3) * chunks + c) * 8 + (myrow & 7)];
        } else {
            for (int c = 0; c < chunks; ++c) dst[((r >> 3) * chunks + c) * 8 + (r & 7)] = make_uint4(0, 0, 0, 0);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (a.prune && myrow_slot >= 0) {
            const uint32_t g0 = a.group[a.rows ? a.rows[slot0] : (uint32_t)slot0];
            part = a.group[myrow] != g0 ? 1 : 0;
            const float *xr = a.X + (int64_t)a.pos2row[myrow] * a.d;
            float ny = 0.0f;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                yv[k] = 0.0f;
                if (k < a.d) {
                    yv[k] = (xr[k] - (a.mu_f ? a.mu_f[k] : 0.0f)) * a.scale_f;
                    ny = fmaf(yv[k], yv[k], ny);
                    atomicAdd(&sh->cR[part][k], yv[k]);
                }
            }
            atomicAdd(&sh->nvalid[part], 1);
            atomicMax(&sh->ymax_bits, __float_as_uint(sqrtf(ny)));
            if (a.lup) atomicMax(&sh->lup_bits[part], __float_as_uint(a.lup[myrow]));
        }
        const unsigned int in0 = __ballot_sync(0xffffffffu, myrow_slot >= 0 && part == 0);
        const unsigned int in1 = __ballot_sync(0xffffffffu, myrow_slot >= 0 && part == 1);
        if (lane == 0) {
            if (in0) atomicOr(&sh->warps_in[0], 1u << warp);
            if (in1) atomicOr(&sh->warps_in[1], 1u << warp);
        }
    }
    __syncthreads();
    if (a.prune && warp < kEpiWarps && myrow_slot >= 0) {
        float dd = 0.0f;
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (k < a.d) {
                const float e = yv[k] - sh->cR[part][k] / (float)sh->nvalid[part];
                dd = fmaf(e, e, dd);
            }
        atomicMax(&sh->rho_bits[part], __float_as_uint(sqrtf(dd)));
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (a.prune && threadIdx.x < 64 && (threadIdx.x & 31) < a.d) {
        const int h = threadIdx.x >> 5;
        sh->cR[h][threadIdx.x & 31] /= (float)(sh->nvalid[h] > 0 ? sh->nvalid[h] : 1);
    }
    __syncthreads();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort_flag = &sh->abort_flag;
    const uint64_t wait_ns = a.wait_ns;

    if (warp == kProdWarp) {
        // Producer: takes the planned tiles from the planners' queues (whichever has one,
        // alternating when both do) and stages each into the B ring with the epilogue warps
        // that need it.  A planner ends its queue with -1; when every queue has ended, -1
        // travels with the stages as the end marker.
        int issued = 0;
        int taken0 = 0, taken1 = 0;     // entries taken from each queue
        bool end0 = false, end1 = false;
        int last = 1;
        // stage one tile (or the end marker, ct < 0) into the ring
        int s = 0, qi = 0;       // ring stage and record slot of the next staged tile
        uint32_t eph = 1u;       // parity of the stage's empty phase to wait for
        auto stage = [&](int ct, unsigned int wmask, uint32_t tcomp) -> bool {
            if (issued >= kStages && !mbar_wait_warp(&sh->empty[s], eph, abort_flag, wait_ns)) return false;
            if (lane == 0) {
                ((volatile int *)sh->info_tile)[qi] = ct;
                ((volatile unsigned int *)sh->info_mask)[qi] = wmask;
                ((volatile uint32_t *)sh->info_comp)[qi] = tcomp;
                if (ct < 0) {
                    mbar_arrive(&sh->full[s]);
                } else {
                    mbar_arrive_expect_tx(&sh->full[s], b_bytes);
                    bulk_g2s(sB + (size_t)s * b_bytes, a.XB + (int64_t)ct * kBN * kpad, b_bytes, &sh->full[s]);
                }
            }
            ++issued;
            if (++s == kStages) {
                s = 0;
                eph ^= 1u;
            }
            if (++qi == kInfoQ) qi = 0;
            __syncwarp();
            return true;
        };
        bool ok = true;
        for (;;) {
            // wait for an entry in some queue, or for the end of all of them (bounded; the
            // whole warp polls and takes lane 0's reading, so that it decides as one)
            const uint64_t t0 = global_ns();
            int q = -1;
            for (uint32_t it = 0;; ++it) {
                const int h0 = __shfl_sync(0xffffffffu, ((volatile int *)sh->plan_head)[0], 0);
                const int h1 = __shfl_sync(0xffffffffu, ((volatile int *)sh->plan_head)[1], 0);
                const bool r0 = !end0 && h0 > taken0, r1 = !end1 && h1 > taken1;
                if (r0 || r1) {
                    q = (r0 && r1) ? (last ^ 1) : (r0 ? 0 : 1);
                    break;
                }
                if (end0 && end1) break;
                if (__shfl_sync(0xffffffffu, (int)(*abort_flag != 0 || global_ns() - t0 > wait_ns), 0)) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
            }
            if (!ok || q < 0) break;
            __threadfence_block();
            const int n = q == 0 ? taken0 : taken1;
            const int at = q * kPlanQh + n % kPlanQh;
            const int ct = ((volatile int *)sh->plan_ct)[at];
            const unsigned int wmask = ((volatile unsigned int *)sh->plan_mask)[at];
            const uint32_t tcomp = ((volatile uint32_t *)sh->plan_comp)[at];
            __syncwarp();
            if (lane == 0) ((volatile int *)sh->plan_tail)[q] = n + 1;
            if (q == 0) {
                ++taken0;
                end0 = ct < 0;
            } else {
                ++taken1;
                end1 = ct < 0;
            }
            last = q;
            if (ct < 0) continue;
            if (!(ok = stage(ct, wmask, tcomp))) break;
        }
        if (ok) ok = stage(-1, 0u, kInvalid);
        if (!ok) *abort_flag = 1;
        // drain: every issued copy must have landed before the CTA exits
        if (lane == 0) {
            for (int q = issued - kStages < 0 ? 0 : issued - kStages; q < issued; ++q) {
                const uint64_t t0 = global_ns();
                while (!mbar_try_wait(&sh->full[q % kStages], (q / kStages) & 1) && global_ns() - t0 < kDrainNs)
                    __nanosleep(256);
            }
        }
        __syncwarp();
    } else if (warp == kPlanWarp || warp == kPlanWarp + 1) {
        // Planners: decide which column tiles to take, ahead of the producer (at most
        // kPlanQh tiles each), so that the bound computations overlap the copies and the
        // MMAs.  Planner p takes the column blocks at odd or even places of the cyclic
        // order (a fixed split: every block is decided by exactly one planner).  A tile is
        // skipped when the lower bound of its candidate values exceeds the threshold of
        // every row that could use it (the epilogue's published maxima, possibly stale =
        // larger = safe).
        const int pl = warp - kPlanWarp;
        float rhoR[2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            rhoR[h] = sh->nvalid[h] > 0 ? sphere_slack(__uint_as_float(sh->rho_bits[h]), __uint_as_float(sh->ymax_bits))
                                        : -1.0f;
        const unsigned int win0 = sh->warps_in[0], win1 = sh->warps_in[1];
        int planned = 0;
        bool ok_all = true;
        volatile int *q_ct = (volatile int *)sh->plan_ct + pl * kPlanQh;
        volatile unsigned int *q_mask = (volatile unsigned int *)sh->plan_mask + pl * kPlanQh;
        volatile uint32_t *q_comp = (volatile uint32_t *)sh->plan_comp + pl * kPlanQh;
        // bounded wait (the whole warp polls) for room for n more entries in this queue
        auto room = [&](int n) -> bool {
            const uint64_t t0 = global_ns();
            bool ok = true;
            while (planned + n - ((volatile int *)sh->plan_tail)[pl] > kPlanQh) {
                if (*abort_flag || global_ns() - t0 > wait_ns) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
            }
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) *abort_flag = 1;
            return ok;
        };
        // append one entry (ct, wmask, tcomp), written by lane 0
        auto push = [&](int ct, unsigned int wmask, uint32_t tcomp) -> bool {
            if (!room(1)) return false;
            if (lane == 0) {
                q_ct[planned % kPlanQh] = ct;
                q_mask[planned % kPlanQh] = wmask;
                q_comp[planned % kPlanQh] = tcomp;
                __threadfence_block();
                ((volatile int *)sh->plan_head)[pl] = planned + 1;
            }
            ++planned;
            __syncwarp();
            return true;
        };
        // append the entries of the lanes with keep, in lane order, with one update of the head
        auto push_step = [&](bool keep, int ct, unsigned int wmask, uint32_t tcomp) -> bool {
            const unsigned int km = __ballot_sync(0xffffffffu, keep);
            if (!km) return true;
            const int nk = __popc(km);
            if (!room(nk)) return false;
            if (keep) {
                const int at = (planned + __popc(km & ((1u << lane) - 1u))) % kPlanQh;
                q_ct[at] = ct;
                q_mask[at] = wmask;
                q_comp[at] = tcomp;
                __threadfence_block();
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                ((volatile int *)sh->plan_head)[pl] = planned + nk;
            }
            planned += nk;
            __syncwarp();
            return true;
        };
        int range_tiles = 0;   // tiles of this split's blocks inside the range
        // A masked sweep whose rows all lie in one component skips the column tiles of
        // that component (every column there is ineligible).
        const uint32_t rcomp = (a.comp && sh->cmin == sh->cmax) ? sh->cmin : kInvalid;
        // Warps that need a sphere pair with lower bounds lb0 / lb1 for the row parts:
        // those holding rows of a part whose bound does not exceed the warp's threshold
        // (a snapshot: thresholds only fall, so a stale one only keeps more).
        auto need_mask = [&](float lb0, float lb1) -> unsigned int {
            unsigned int m = 0u;
#pragma unroll
            for (int w = 0; w < kEpiWarps; ++w) {
                const float thr = ((volatile float *)sh->warp_thr)[w];
                const bool need = (((win0 >> w) & 1u) && !(lb0 > thr)) || (((win1 >> w) & 1u) && !(lb1 > thr));
                m |= need ? (1u << w) : 0u;
            }
            return m;
        };
        // landmark bound of a column tile or block (lmin) for the two row parts
        float dmaxR[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) dmaxR[h] = (a.lup && sh->nvalid[h] > 0) ? __uint_as_float(sh->lup_bits[h]) : -1.0f;
        auto land_bounds = [&](float lmin, float &lb0, float &lb1) {
            if (!(lmin > 0.0f)) return;
            if (dmaxR[0] >= 0.0f) lb0 = fmaxf(lb0, land_lower_bound(lmin, dmaxR[0], a.d, a.lb_R2, a.lb_eps, a.lb_gamma));
            if (dmaxR[1] >= 0.0f) lb1 = fmaxf(lb1, land_lower_bound(lmin, dmaxR[1], a.d, a.lb_R2, a.lb_eps, a.lb_gamma));
        };
        auto part_bounds = [&](const float *cC, float rhoC, float &lb0, float &lb1) {
            lb0 = rhoR[0] >= 0.0f && rhoC >= 0.0f
                      ? tile_lower_bound(sh->cR[0], rhoR[0], cC, rhoC, a.d, a.lb_R2, a.lb_eps, a.lb_gamma)
                      : INFINITY;
            lb1 = rhoR[1] >= 0.0f && rhoC >= 0.0f
                      ? tile_lower_bound(sh->cR[1], rhoR[1], cC, rhoC, a.d, a.lb_R2, a.lb_eps, a.lb_gamma)
                      : INFINITY;
        };
        int first = -1;   // a tile taken before any decision
        if (a.prune) {
            // Without thresholds known at the start, one tile (this row tile's own, the
            // nearest columns) goes unconditionally and every later decision waits for the
            // thresholds the epilogue learns from it: one tile of pipeline fill per CTA.
            // The wait is bounded; on time-out the decisions only get less selective.
            if (!(COLLECT || a.row_B) && nblk > 0) {
                first = split == 0 ? tile0 : (blk_at(0) * kBlkTiles > rtb ? blk_at(0) * kBlkTiles : rtb);
                if (pl == 0) ok_all = push(first, 0xFFu, a.comp ? a.tile_comp[first] : kInvalid);
            }
            if (ok_all && nblk > 0 && lane == 0) {
                const uint64_t t0 = global_ns();
                while (((volatile int *)&sh->npub)[0] < kEpiWarps && !*abort_flag && global_ns() - t0 < wait_ns)
                    __nanosleep(64);
            }
            __syncwarp();
        }
        // Level 1: 32 blocks per step, one per lane (this planner's half of them), against
        // the blocks' spheres.  Level 2: in each block some warp needs, its tiles (one per
        // lane) against the tiles' two spheres; the tile is skipped when no warp needs it.
        for (int u0 = 0; ok_all && u0 < nblk; u0 += 32) {
            const int nb = nblk - u0 < 32 ? nblk - u0 : 32;
            bool bneed = lane < nb && (lane & 1) == pl;
            range_tiles += __reduce_add_sync(0xffffffffu, lane < nb ? blk_tiles(blk_at(u0 + lane)) : 0);
            if (bneed && a.prune) {
                const int cb = blk_at(u0 + lane);
                float lb0, lb1;
                part_bounds(a.blk_c + (int64_t)cb * a.d, a.blk_rho[cb], lb0, lb1);
                if (a.blk_lmin) land_bounds(a.blk_lmin[cb], lb0, lb1);
                bneed = need_mask(lb0, lb1) != 0u;
            }
            unsigned int bm = __ballot_sync(0xffffffffu, bneed);
            while (ok_all && bm) {
                const int q = __ffs(bm) - 1;
                bm &= bm - 1u;
                const int t0c = blk_at(u0 + q) * kBlkTiles;
                const int n = ntile_all - t0c < kBlkTiles ? ntile_all - t0c : kBlkTiles;
                unsigned int wmask = (lane < n && t0c + lane >= rtb && t0c + lane < rte) ? 0xFFu : 0u;
                uint32_t tcomp = kInvalid;
                if (wmask) {
                    const int ct = t0c + lane;
                    if (a.comp) tcomp = a.tile_comp[ct];
                    if (ct == first || (rcomp != kInvalid && tcomp == rcomp)) {
                        wmask = 0u;
                    } else if (a.prune) {
                        float lb0 = INFINITY, lb1 = INFINITY;
#pragma unroll
                        for (int hc = 0; hc < 2; ++hc) {
                            float l0, l1;
                            part_bounds(a.tile_c + ((int64_t)ct * 2 + hc) * a.d, a.tile_rho[(int64_t)ct * 2 + hc], l0, l1);
                            lb0 = fminf(lb0, l0);
                            lb1 = fminf(lb1, l1);
                        }
                        if (a.tile_lmin) land_bounds(a.tile_lmin[ct], lb0, lb1);
                        wmask = need_mask(lb0, lb1);
                    }
                }
                ok_all = push_step(wmask != 0u, t0c + lane, wmask, tcomp);
            }
        }
        if (ok_all) push(-1, 0u, kInvalid);
        const int taken = planned > 0 ? planned - 1 : 0;   // tiles, without the end marker
        if (lane == 0 && a.st_tiles) {
            // skipped = the range's tiles (counted once) less the tiles either planner took
            atomicAdd(&a.st_tiles[0], (unsigned long long)((pl == 0 ? (long long)range_tiles : 0ll) - taken));
            atomicAdd(&a.st_tiles[1], (unsigned long long)taken);
        }
    } else if (warp == kMmaWarp) {
        const uint32_t idesc = instr_desc(a.fp16);
        const uint32_t lbo = 128, sbo = (uint32_t)(kpad / 8) * 128;
        const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
        const int ksteps = kpad / 16;
        const uint64_t adesc0[2] = {smem_desc(aaddr, lbo, sbo), smem_desc(aaddr + 16u * sbo, lbo, sbo)};
        const uint64_t bdesc0 = smem_desc(baddr, lbo, sbo);
        int done = 0;
        // stage, its phase and the record slot of tile q, kept as counters (kStages is a
        // run-time value, and a division per tile is not free on this path)
        int s = 0, qi = 0;
        uint32_t sph = 0;
        for (int q = 0;; ++q) {
            const int b = q & 1;
            bool ok = mbar_wait_warp(&sh->full[s], sph, abort_flag, wait_ns);
            if (ok && q >= 2) ok = mbar_wait_warp(&sh->tempty[b], ((q >> 1) - 1) & 1, abort_flag, wait_ns);
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            // every lane observed the stage (acquire) and reads the same record word
            const int tile = ((volatile int *)sh->info_tile)[qi];
            tc_fence_after();
            if (lane == 0) {
                if (tile >= 0) {
                    // descriptors: the start-address field (bits 0-13, address >> 4) of the
                    // stage's base plus 16 per K step of 16 (256 bytes); shared addresses stay
                    // below 2^18, so the field never carries into the next one
                    const uint64_t bd0 = bdesc0 + (uint64_t)(((uint32_t)s * b_bytes) >> 4);
                    const uint32_t d0 = tmem + (uint32_t)(b * 2 * kBN);
                    switch (ksteps) {
                    case 1: mma_tile<1>(d0, adesc0[0], adesc0[1], bd0, idesc); break;
                    case 2: mma_tile<2>(d0, adesc0[0], adesc0[1], bd0, idesc); break;
                    case 3: mma_tile<3>(d0, adesc0[0], adesc0[1], bd0, idesc); break;
                    case 4: mma_tile<4>(d0, adesc0[0], adesc0[1], bd0, idesc); break;
                    case 5: mma_tile<5>(d0, adesc0[0], adesc0[1], bd0, idesc); break;
                    default: mma_tile<6>(d0, adesc0[0], adesc0[1], bd0, idesc); break;
                    }
                    mma_commit(&sh->empty[s]);
                    mma_commit(&sh->tfull[b]);
                } else {
                    mbar_arrive(&sh->tfull[b]);   // no MMA for the end marker
                }
                mbar_arrive(&sh->tfull[b]);       // passes the producer's tile record on (release)
            }
            __syncwarp();
            if (tile < 0) break;
            done = q + 1;
            if (++s == kStages) {
                s = 0;
                sph ^= 1u;
            }
            if (++qi == kInfoQ) qi = 0;
        }
        // every issued MMA completes before TMEM is freed
        if (lane == 0 && done > 0) {
            mma_commit(&sh->drain);
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait(&sh->drain, 0) && global_ns() - t0 < kDrainNs) __nanosleep(256);
        }
        __syncwarp();
    } else {
        // epilogue: one row per thread, 128 columns per tile in two halves of 64
        const int half = warp >> 2, quad = warp & 3;
        const bool valid = myrow_slot >= 0;
        const float cthr = (COLLECT && valid) ? a.thr[slot0 + myrow_slot] : -INFINITY;
        RowSel<KC, CB> sel;
        sel.init(valid);
        const RowConst rc = valid ? make_rowconst(a.sc, a.m, a.pos2row[myrow]) : RowConst{0.f, 0.f};
        float *bv = band_v + threadIdx.x;
        uint32_t *bj = band_j + threadIdx.x;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
        // A bounded row starts at the threshold of its bound; thresholds already published
        // for these rows by other column ranges apply too.  Then the warp's first
        // publication: before the first tile when the thresholds are known from the start
        // (collect pass, bounded rows), else after it.
        if (!COLLECT && valid && a.row_B) {
            const double B = a.row_B[a.pos2row[myrow]];
            if (B < INFINITY) sel.bound(sel_threshold(a.sc, rc, __double2float_ru(B / a.m.inv_scale2)));
        }
        if (!COLLECT && a.splits > 1 && valid) sel.bound(shared_thr_exchange(&a.slot_thr[slot0 + myrow_slot], INFINITY));
        // the warp's largest threshold: thresholds are non-negative floats or -inf, whose
        // bit patterns order as signed integers, so one integer max reduction gives it
        auto publish = [&]() {
            const int wt = __reduce_max_sync(0xffffffffu, __float_as_int(COLLECT ? cthr : sel.thr));
            if (lane == 0) ((volatile float *)sh->warp_thr)[warp] = __int_as_float(wt);
        };
        bool published = false;
        if (a.prune && (COLLECT || a.row_B)) {
            publish();
            __syncwarp();
            if (lane == 0) atomicAdd(&sh->npub, 1);
            published = true;
        }
        // Fast test of 32 values against the row's threshold: a 3-input integer min over the
        // FP32 bit patterns.  For non-negative values the integer order is the float order;
        // a negative value compares below every non-negative threshold, so it can only raise
        // a false alarm, which the exact walk below rejects.
        auto imin32 = [&](const uint32_t(&w)[32]) {
            int l1[11];
#pragma unroll
            for (int q = 0; q < 10; ++q) l1[q] = __vimin3_s32((int)w[3 * q], (int)w[3 * q + 1], (int)w[3 * q + 2]);
            l1[10] = min((int)w[30], (int)w[31]);
            const int l2a = __vimin3_s32(l1[0], l1[1], l1[2]), l2b = __vimin3_s32(l1[3], l1[4], l1[5]);
            const int l2c = __vimin3_s32(l1[6], l1[7], l1[8]), l2d = min(l1[9], l1[10]);
            return min(__vimin3_s32(l2a, l2b, l2c), l2d);
        };
        // The exact walk of one 32-column chunk: the columns whose value passes the
        // threshold, in order, each value taken from the registers by its column number.
        uint32_t tcomp = kInvalid;   // component of the current column tile (kInvalid: mixed)
        // the columns of this row's instance (all columns when not batched)
        int64_t ibeg = 0, iend = a.N;
        if (a.inst_pos && valid) {
            ibeg = a.inst_off[a.inst_pos[myrow]];
            iend = a.inst_off[a.inst_pos[myrow] + 1];
        }
        auto walk = [&](const uint32_t(&w)[32], int64_t jbase) {
            const float thr = COLLECT ? cthr : sel.thr;
            uint32_t mask = 0;
#pragma unroll
            for (int q = 0; q < 32; ++q) mask |= (__uint_as_float(w[q]) <= thr ? 1u : 0u) << q;
            while (mask) {
                const int q = __ffs(mask) - 1;
                mask &= mask - 1;
                const float val = __uint_as_float(pick32(w, q));
                const int64_t j = jbase + q;
                if (!(val <= (COLLECT ? cthr : sel.thr))) continue;
                if (j >= a.N || (uint32_t)j == myrow) continue;
                if (j < ibeg || j >= iend) continue;   // another instance
                if (a.comp && (tcomp != kInvalid ? tcomp == mycomp : a.comp_pos[j] == mycomp)) continue;
                if (COLLECT) {
                    const int64_t sl = slot0 + myrow_slot;
                    const uint32_t p = atomicAdd(&a.coll_cnt[sl], 1u);
                    if ((int64_t)p < a.coll_cap) a.coll_j[sl * a.coll_cap + p] = (uint32_t)j;
                } else {
                    sel.insert(val, (uint32_t)j, a.sc, rc, bv, bj, kRowTile);
                }
            }
        };
        for (int q = 0;; ++q) {
            const int b = q & 1;
            if (!mbar_wait_warp(&sh->tfull[b], (q >> 1) & 1, abort_flag, wait_ns)) {
                *abort_flag = 1;
                break;
            }
            // the tile number comes from lane 0 so that the whole warp decides alike
            tc_fence_after();
            // tile number (-1: end) and this warp's bit of the mask in one word
            int tw = 0;
            uint32_t tcm = kInvalid;
            if (lane == 0) {
                const int tl = ((volatile int *)sh->info_tile)[q % kInfoQ];
                const unsigned int m = ((volatile unsigned int *)sh->info_mask)[q % kInfoQ];
                tw = tl < 0 ? -1 : (tl << 1) | (int)((m >> warp) & 1u);
                tcm = ((volatile uint32_t *)sh->info_comp)[q % kInfoQ];
            }
            tw = __shfl_sync(0xffffffffu, tw, 0);
            if (tw < 0) break;
            const int tile = tw >> 1;
            const int64_t col0 = (int64_t)tile * kBN;
            if (!(tw & 1)) {
                // no row of this warp can have a candidate in the tile: release the buffer
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->tempty[b]);
                continue;
            }
            // the tile's component travelled with it through the plan and the ring
            if (a.comp) tcomp = __shfl_sync(0xffffffffu, tcm, 0);
            // a row of the tile's own component has nothing eligible in it
            const bool own = a.comp && tcomp != kInvalid && tcomp == mycomp;
            const uint32_t taddr = lane_base + (uint32_t)((b * 2 + half) * kBN);
#pragma unroll 1
            for (int hh = 0; hh < kBN / 64; ++hh) {
                uint32_t va[32], vb[32];
                tmem_ld32(taddr + hh * 64, va);
                tmem_ld32(taddr + hh * 64 + 32, vb);
                tmem_wait_ld(va);
                reg_fence(vb);
                if (hh == kBN / 64 - 1) {
                    // every load of this tile has landed: hand the TMEM buffer back early
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh->tempty[b]);
                }
                const int ithr = __float_as_int(COLLECT ? cthr : sel.thr);
                const int m0 = imin32(va), m1 = imin32(vb);
                if (!own && min(m0, m1) <= ithr) {
                    if (m0 <= ithr) walk(va, col0 + hh * 64);
                    if (m1 <= __float_as_int(COLLECT ? cthr : sel.thr)) walk(vb, col0 + hh * 64 + 32);
                }
                __syncwarp();
            }
            if (!COLLECT && a.splits > 1 && valid)
                sel.bound(shared_thr_exchange(&a.slot_thr[slot0 + myrow_slot], sel.thr));
            if (a.prune) {
                publish();
                if (!published) {
                    __syncwarp();
                    if (lane == 0) atomicAdd(&sh->npub, 1);
                    published = true;
                }
            }
        }
        if (!COLLECT && valid) {
            const int64_t rec = (slot0 + myrow_slot) * a.splits + split;
            sel.write(a.out_v + rec * kListC, a.out_j + rec * kListC, a.out_ovf + rec, bv, bj, kRowTile);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && sh->abort_flag) atomicExch(a.err_flag, 1);
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

size_t sweep_tc_smem_bytes(int kpad, int band)
{
    // at least ~half of the SM's shared memory keeps one CTA per SM (it holds all of TMEM)
    const size_t need = (size_t)kRowTile * kpad * 2 + (size_t)tc_stages(kpad, band) * kBN * kpad * 2 + kShBytes +
                        (size_t)band * kRowTile * 8 + 1024;
    const size_t one_per_sm = 120 * 1024;
    return need > one_per_sm ? need : one_per_sm;
}

template <int KC, int CB, bool COLL>
static cudaError_t go_tc(const SweepArgs &a, dim3 grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = set_max_dynamic_smem(k_sweep_tc<KC, CB, COLL>);
    if (e != cudaSuccess) return e;
    k_sweep_tc<KC, CB, COLL><<<grid, kThreadsTc, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int CB>
static cudaError_t go_tc_band(const SweepArgs &a, bool collect, dim3 grid, cudaStream_t s)
{
    const size_t smem = sweep_tc_smem_bytes(a.kpad, CB);
    if (tc_stages(a.kpad, CB) < 2 || a.kpad > 16 * kMaxKSteps || a.kpad % 16) return cudaErrorInvalidValue;
    if (collect) return go_tc<1, CB, true>(a, grid, smem, s);
    if (a.kc <= 1) return go_tc<1, CB, false>(a, grid, smem, s);
    if (a.kc <= 2) return go_tc<2, CB, false>(a, grid, smem, s);
    if (a.kc <= 4) return go_tc<4, CB, false>(a, grid, smem, s);
    if (a.kc <= 8) return go_tc<8, CB, false>(a, grid, smem, s);
    return go_tc<16, CB, false>(a, grid, smem, s);
}

cudaError_t launch_sweep_tc(const SweepArgs &a, bool collect, cudaStream_t s)
{
    dim3 grid((unsigned)((a.nslots + kRowTile - 1) / kRowTile), (unsigned)a.splits);
    if (a.band > 32) return go_tc_band<kBandWide>(a, collect, grid, s);
    return go_tc_band<32>(a, collect, grid, s);
}

}  // namespace nnm
