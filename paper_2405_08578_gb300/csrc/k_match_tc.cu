// Nearest-neighbour matching (Sec. 2.4, Eq. 6) with BF16 tensor cores
// (tcgen05) for sm_103a, re-ranked in FP32 so that every decision equals the
// plain FP32 form's.
//
// Stage 1, k_match_tc (persistent, one CTA per SM, 10 warps):
//   warp 0    TMA producer: per work unit a 256-row A block (2 x 32 KB boxes,
//             128-byte swizzle), then 128-row B tiles (2 x 16 KB boxes) into a
//             4-stage ring.
//   warp 1    allocates all 512 TMEM columns; one lane issues
//             tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 128, K = 16,
//             BF16 x BF16 -> FP32): 2 row blocks x 8 K-steps per B tile, into
//             one of two TMEM accumulator buffers; tcgen05.commit releases the
//             B stage and hands the buffer to the epilogue.
//   warps 2-9 epilogue: each thread owns one A row, reads its 128 FP32 dot
//             products per tile with tcgen05.ld (32x32b.x32), forms
//             v = |b~|^2 - 2 a~.b~ and keeps the row's 8 smallest v in
//             registers; no distance matrix is written.
//   A work unit is (256-row block of A, one of S column splits of B); units
//   are dealt round-robin to the persistent CTAs.  Every mbarrier wait is
//   bounded by a 2 s clock limit; on expiry the CTA records LP_ERR_TIMEOUT,
//   drains, frees its TMEM and returns.
//
// Stage 2, k_rerank (one warp per row): candidates whose BF16 value lies
//   within 2*delta of the row's second-smallest BF16 value are re-scored
//   with exactly the FP32 form's arithmetic (sequential FMA over k, then
//   fma(-2, dot, |b|^2)), so their values are bit-identical to the FP32
//   form's.  With unit, non-negative descriptors and BF16 unit roundoff
//   u = 2^-8, |v~_j - v_j| <= 3u + 3u^2 + 1.1e-4 = delta for every column j
//   (derivation in the design doc).  The row is certified when the smallest
//   eighth-best BF16 value over the splits, minus delta, exceeds the exact
//   second-best: then no column outside the candidates can enter the top 2.
//   Uncertified rows are queued.
// Stage 3: queued rows are re-scanned with the FP32 form's arithmetic.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "lp_internal.cuh"

namespace lp {

__global__ void k_row_norms(const float* d, const uint8_t* v, long long n, float* out, float invalid_value);
__global__ void k_match_finish(const float4* part, int S, long long NA, const float* na, const uint8_t* vA,
                               float ratio2, float delta_s2, int32_t* match, float* d1, float* d2);

namespace {

constexpr int kRowsPerUnit = 256;       // two M = 128 row blocks
constexpr int kTileN = 128;             // B rows per tile (MMA N)
constexpr int kStages = 4;              // B ring depth
constexpr int kThreadsTC = 320;         // 10 warps
constexpr int kEpiWarps = 8;
constexpr uint32_t kABytes = kRowsPerUnit * 128 * 2;   // 64 KB
constexpr uint32_t kBBytes = kTileN * 128 * 2;         // 32 KB per stage
constexpr uint32_t kNbBytes = kEpiWarps * kTileN * 4;   // per-warp copy of one tile's |b~|^2
constexpr uint32_t kSmemTC = kABytes + kStages * kBBytes + kNbBytes + 1024 /*barriers*/ + 1024 /*align slack*/;
constexpr int kTopK = 8;
// |b~|^2 of an invalid or masked column: finite (so that the column tag below
// never turns it into a NaN) and far above any real value; treated as +inf by
// the re-rank.
constexpr float kNoColumn = 3.0e38f;
// 3u + 3u^2 (BF16 rounding) + FP32 accumulation allowance + the column tag
// that the epilogue writes into the 5 low mantissa bits (<= 31 ulp)
constexpr float kDelta = 3.0f / 256.0f + 3.0f / 65536.0f + 1e-4f + 1e-5f;

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: true when the phase completed, false on abort/timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int32_t* status)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > 2000000000ull) {   // 2 s
                *abort_flag = 1;
                set_status(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 128 B stacked every 1024 B (SBO); LBO unused for this layout (set to 16 B);
// descriptor version 1; swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = FP32, A = B = BF16, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Issue a 32-column TMEM load (lane = row, 32 consecutive FP32 columns).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Wait for this thread's outstanding TMEM loads.  The registers of the load
// being waited for are in/out operands, so no use of them can be scheduled
// above the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// ------------------------------------------------------------------ work split
struct TcParams {
    long long NA, NB;
    int nrp;               // number of 256-row blocks
    int S;                 // column splits
    long long cps;         // columns per split (multiple of kTileN)
    const float* nb16;     // |b~_j|^2 (+inf when invalid), length NB
    float4* pv;            // [S][NA][2] the kTopK smallest values
    int4* pj;              // [S][NA][2] their columns (-1 = none)
    int32_t* status;
};

// Unit u = (256-row block rp, column split): consecutive units share a row
// block, and each CTA takes a contiguous run of units, so the A block is
// usually reused and each split's list can start from the previous split's
// k-th best.
__device__ __forceinline__ void unit_range(const TcParams& p, int u, int& rp, int& split, long long& c0, int& ntiles)
{
    rp = u / p.S;
    split = u - rp * p.S;
    c0 = (long long)split * p.cps;
    long long c1 = c0 + p.cps;
    if (c1 > p.NB) c1 = p.NB;
    ntiles = c1 > c0 ? (int)((c1 - c0 + kTileN - 1) / kTileN) : 0;
}

// Sorted top-k (ascending) in registers; every index is a compile-time
// constant after unrolling.
struct TopK {
    float v[kTopK];
    int j[kTopK];
};

__device__ __forceinline__ void topk_insert(TopK& t, float x, int jx)
{
    bool c[kTopK];
#pragma unroll
    for (int i = 0; i < kTopK; ++i) c[i] = x < t.v[i];
#pragma unroll
    for (int i = kTopK - 1; i > 0; --i) {
        t.v[i] = c[i - 1] ? t.v[i - 1] : (c[i] ? x : t.v[i]);
        t.j[i] = c[i - 1] ? t.j[i - 1] : (c[i] ? jx : t.j[i]);
    }
    t.v[0] = c[0] ? x : t.v[0];
    t.j[0] = c[0] ? jx : t.j[0];
}

// v with its 5 low mantissa bits replaced by the column's position i in the
// chunk: the chunk minimum then also names its column.
__device__ __forceinline__ float tag(float v, int i)
{
    return __uint_as_float((__float_as_uint(v) & ~31u) | (uint32_t)i);
}

__global__ void __launch_bounds__(kThreadsTC, 1)
k_match_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kABytes;
    float* snb = reinterpret_cast<float*>(smem + kABytes + kStages * kBBytes);   // [kEpiWarps][kTileN]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kABytes + kStages * kBBytes + kNbBytes);
    // barrier slots
    uint64_t* full = bars;                 // [kStages]
    uint64_t* empty = bars + kStages;      // [kStages]
    uint64_t* tfull = bars + 2 * kStages;  // [2]
    uint64_t* tempty = tfull + 2;          // [2]
    uint64_t* afull = tempty + 2;          // [1]
    uint64_t* aempty = afull + 1;          // [1]
    uint64_t* drain = aempty + 1;          // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int U = p.nrp * p.S;
    const int per = U / (int)gridDim.x, rem = U % (int)gridDim.x;
    const int u_begin = (int)blockIdx.x * per + min((int)blockIdx.x, rem);
    const int u_end = u_begin + per + ((int)blockIdx.x < rem ? 1 : 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(afull), 1);
        mbar_init(smem_u32(aempty), 1);
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        tma_prefetch_desc(&tmA);
        tma_prefetch_desc(&tmB);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            long long n = 0;   // tile counter of this CTA (non-empty units only)
            int v = 0;         // non-empty unit counter of this CTA
            int armed[kStages];
            int a_armed = -1;
            for (int s = 0; s < kStages; ++s) armed[s] = -1;
            bool ok = true;
            int prev_rp = -1;
            for (int u = u_begin; u < u_end && ok; ++u) {
                int rp, split, ntiles;
                long long c0;
                unit_range(p, u, rp, split, c0, ntiles);
                if (ntiles == 0) continue;
                if (rp != prev_rp) {
                    ok = mbar_wait(smem_u32(aempty), (v & 1) ^ 1, abort_flag, p.status);
                    if (!ok) break;
                    mbar_expect_tx(smem_u32(afull), kABytes);
                    tma_load_2d(smem_u32(sA), &tmA, 0, rp * kRowsPerUnit, smem_u32(afull));
                    tma_load_2d(smem_u32(sA + kABytes / 2), &tmA, 64, rp * kRowsPerUnit, smem_u32(afull));
                    a_armed = v;
                    ++v;
                    prev_rp = rp;
                }
                for (int t = 0; t < ntiles; ++t, ++n) {
                    const int s = (int)(n % kStages);
                    const uint32_t k = (uint32_t)(n / kStages);
                    ok = mbar_wait(smem_u32(&empty[s]), (k & 1) ^ 1, abort_flag, p.status);
                    if (!ok) break;
                    uint8_t* dst = sB + s * kBBytes;
                    const int y = (int)(c0 + (long long)t * kTileN);
                    mbar_expect_tx(smem_u32(&full[s]), kBBytes);
                    tma_load_2d(smem_u32(dst), &tmB, 0, y, smem_u32(&full[s]));
                    tma_load_2d(smem_u32(dst + kBBytes / 2), &tmB, 64, y, smem_u32(&full[s]));
                    armed[s] = (int)k;
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the copies this thread issued to land
                for (int s = 0; s < kStages; ++s) {
                    if (armed[s] < 0) continue;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try(smem_u32(&full[s]), (uint32_t)armed[s] & 1u) && globaltimer() - t0 < 200000000ull) {
                    }
                }
                if (a_armed >= 0) {
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try(smem_u32(afull), (uint32_t)a_armed & 1u) && globaltimer() - t0 < 200000000ull) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            long long n = 0;
            int v = 0;
            bool ok = true;
            int prev_rp = -1;
            for (int u = u_begin; u < u_end && ok; ++u) {
                int rp, split, ntiles;
                long long c0;
                unit_range(p, u, rp, split, c0, ntiles);
                if (ntiles == 0) continue;
                if (rp != prev_rp) {
                    // release the previous A block once its MMAs are done, then
                    // wait for the new one
                    if (v > 0) mma_commit(smem_u32(aempty));
                    ok = mbar_wait(smem_u32(afull), v & 1, abort_flag, p.status);
                    ++v;
                    prev_rp = rp;
                    if (!ok) break;
                    tc_fence_after();
                }
                for (int t = 0; t < ntiles; ++t, ++n) {
                    const int s = (int)(n % kStages);
                    const uint32_t k = (uint32_t)(n / kStages);
                    const int b = (int)(n & 1);
                    const uint32_t kb = (uint32_t)(n >> 1);
                    ok = mbar_wait(smem_u32(&tempty[b]), (kb & 1) ^ 1, abort_flag, p.status);
                    if (!ok) break;
                    ok = mbar_wait(smem_u32(&full[s]), k & 1, abort_flag, p.status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t bbase = smem_u32(sB + s * kBBytes);
#pragma unroll
                    for (int rb = 0; rb < 2; ++rb) {
                        const uint32_t d = tmem + (uint32_t)((b * 2 + rb) * kTileN);
                        const uint32_t abase = smem_u32(sA) + rb * (128 * 128);
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = sdesc(abase + h * (kABytes / 2) + kk * 32);
                                const uint64_t bd = sdesc(bbase + h * (kBBytes / 2) + kk * 32);
                                mma_bf16(d, ad, bd, (h | kk) ? 1u : 0u);
                            }
                    }
                    mma_commit(smem_u32(&empty[s]));
                    mma_commit(smem_u32(&tfull[b]));
                }
            }
            // wait (bounded) for every MMA this thread issued before TMEM is freed
            mma_commit(smem_u32(drain));
            const uint64_t t0 = globaltimer();
            while (!mbar_try(smem_u32(drain), 0) && globaltimer() - t0 < 2000000000ull) {
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int rb = (warp - 2) >> 2;         // row block 0 (warps 2-5) or 1 (warps 6-9)
        const int row_in_unit = rb * 128 + q * 32 + lane;
        long long n = 0;
        bool ok = true;
        int prev_rp = -1;
        float warm = INFINITY;
        for (int u = u_begin; u < u_end && ok; ++u) {
            int rp, split, ntiles;
            long long c0;
            unit_range(p, u, rp, split, c0, ntiles);
            long long c1 = c0 + p.cps;
            if (c1 > p.NB) c1 = p.NB;
            // a split of the same row block starts from the previous split's
            // k-th best: placeholders (column -1) at that value.  Columns never
            // stored are then still >= the list's last value, the bound the
            // re-rank uses.
            const float t0 = (rp == prev_rp && ntiles > 0) ? warm : INFINITY;
            TopK tk;
#pragma unroll
            for (int i = 0; i < kTopK; ++i) { tk.v[i] = t0; tk.j[i] = -1; }
            float* wnb = snb + (warp - 2) * kTileN;
            // |b~|^2 of tile t, lane l holding columns 4l .. 4l+3 (+inf past the split)
            auto load_nb = [&](int t) {
                const long long j = c0 + (long long)t * kTileN + 4 * lane;
                if (j + 4 <= c1) return __ldg(reinterpret_cast<const float4*>(p.nb16 + j));
                float4 w;
                w.x = j + 0 < c1 ? __ldg(p.nb16 + j + 0) : kNoColumn;
                w.y = j + 1 < c1 ? __ldg(p.nb16 + j + 1) : kNoColumn;
                w.z = j + 2 < c1 ? __ldg(p.nb16 + j + 2) : kNoColumn;
                w.w = j + 3 < c1 ? __ldg(p.nb16 + j + 3) : kNoColumn;
                return w;
            };
            float4 nb_next = ntiles > 0 ? load_nb(0) : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int t = 0; t < ntiles; ++t, ++n) {
                const int b = (int)(n & 1);
                const uint32_t kb = (uint32_t)(n >> 1);
                // stage this tile's norms, start fetching the next tile's
                __syncwarp();
                const float4 nb_cur = nb_next;
                reinterpret_cast<float4*>(wnb)[lane] = nb_cur;
                if (t + 1 < ntiles) nb_next = load_nb(t + 1);
                __syncwarp();
                ok = mbar_wait(smem_u32(&tfull[b]), kb & 1, abort_flag, p.status);
                if (!ok) break;
                tc_fence_after();
                const long long cbase = c0 + (long long)t * kTileN;
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((b * 2 + rb) * kTileN);
                uint32_t ra[32], rb2[32];
                tmem_ld32(tbase, ra);
                tmem_wait(ra);
#pragma unroll
                for (int ch = 0; ch < kTileN / 32; ++ch) {
                    uint32_t (&cur)[32] = (ch & 1) ? rb2 : ra;
                    uint32_t (&nxt)[32] = (ch & 1) ? ra : rb2;
                    if (ch + 1 < kTileN / 32) tmem_ld32(tbase + (uint32_t)((ch + 1) * 32), nxt);
                    // tagged v_j = |b~_j|^2 - 2 s_j and the chunk minimum
                    float kv[32];
                    const float4* nb4 = reinterpret_cast<const float4*>(wnb + ch * 32);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 w = nb4[i];
                        kv[4 * i + 0] = tag(fmaf(-2.f, __uint_as_float(cur[4 * i + 0]), w.x), 4 * i + 0);
                        kv[4 * i + 1] = tag(fmaf(-2.f, __uint_as_float(cur[4 * i + 1]), w.y), 4 * i + 1);
                        kv[4 * i + 2] = tag(fmaf(-2.f, __uint_as_float(cur[4 * i + 2]), w.z), 4 * i + 2);
                        kv[4 * i + 3] = tag(fmaf(-2.f, __uint_as_float(cur[4 * i + 3]), w.w), 4 * i + 3);
                    }
                    float m16[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) m16[i] = fminf(kv[i], kv[i + 16]);
#pragma unroll
                    for (int i = 0; i < 8; ++i) m16[i] = fminf(m16[i], m16[i + 8]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) m16[i] = fminf(m16[i], m16[i + 4]);
                    float cand = fminf(fminf(m16[0], m16[2]), fminf(m16[1], m16[3]));
                    // insert this row's qualifying columns, smallest first; the
                    // loop runs only while some row of the warp still qualifies
                    bool act = cand < tk.v[kTopK - 1];
                    const int j0 = (int)(cbase + ch * 32);
                    while (__any_sync(0xFFFFFFFFu, act)) {
                        if (act) topk_insert(tk, cand, j0 + (int)(__float_as_uint(cand) & 31u));
                        float nx = INFINITY;
#pragma unroll
                        for (int i = 0; i < 32; ++i) nx = fminf(nx, kv[i] > cand ? kv[i] : INFINITY);
                        cand = nx;
                        act = act && cand < tk.v[kTopK - 1];
                    }
                    if (ch + 1 < kTileN / 32) tmem_wait(nxt);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
            }
            if (!ok) break;
            const long long row = (long long)rp * kRowsPerUnit + row_in_unit;
            if (row < p.NA) {
                float4* pv = p.pv + ((long long)split * p.NA + row) * 2;
                int4* pj = p.pj + ((long long)split * p.NA + row) * 2;
                pv[0] = make_float4(tk.v[0], tk.v[1], tk.v[2], tk.v[3]);
                pv[1] = make_float4(tk.v[4], tk.v[5], tk.v[6], tk.v[7]);
                pj[0] = make_int4(tk.j[0], tk.j[1], tk.j[2], tk.j[3]);
                pj[1] = make_int4(tk.j[4], tk.j[5], tk.j[6], tk.j[7]);
            }
            if (ntiles > 0) {
                prev_rp = rp;
                warm = tk.v[kTopK - 1];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// |b~|^2 of the bf16 rows in FP32 (+inf when invalid).
__global__ void k_row_norms_bf16(const __nv_bfloat16* d, const uint8_t* v, long long n, float* out)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const uint2 raw = reinterpret_cast<const uint2*>(d + w * 128)[lane];
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
    const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
    const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
    float s = a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) out[w] = v[w] ? s : kNoColumn;
}

// ------------------------------------------------------------------ re-rank
// FP32-form value of column j for query a: exactly the FP32 kernel's
// arithmetic (sequential fmaf over k = 0..127, then fmaf(-2, dot, |b|^2)).
__device__ __forceinline__ float fp32_form_value(const float* a, const float* b, float nbj)
{
    float acc = 0.f;
    const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll 8
    for (int k4 = 0; k4 < 32; ++k4) {
        const float4 w = __ldg(b4 + k4);
        acc = fmaf(a[4 * k4 + 0], w.x, acc);
        acc = fmaf(a[4 * k4 + 1], w.y, acc);
        acc = fmaf(a[4 * k4 + 2], w.z, acc);
        acc = fmaf(a[4 * k4 + 3], w.w, acc);
    }
    return fmaf(-2.f, acc, nbj);
}

constexpr int kRerankWarps = 8;
constexpr int kMaxCand = 32 * kTopK;   // S <= 32 splits of kTopK candidates

__device__ __forceinline__ void top2_lex(float& b1, int& j1, float& b2, int& j2, float x, int j)
{
    if (j < 0) return;
    if (x < b1 || (x == b1 && (unsigned)j < (unsigned)j1)) {
        b2 = b1; j2 = j1; b1 = x; j1 = j;
    } else if (x < b2 || (x == b2 && (unsigned)j < (unsigned)j2)) {
        b2 = x; j2 = j;
    }
}

__device__ __forceinline__ void warp_top2(float& b1, int& j1, float& b2, int& j2)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float ob1 = __shfl_xor_sync(0xFFFFFFFFu, b1, o), ob2 = __shfl_xor_sync(0xFFFFFFFFu, b2, o);
        const int oj1 = __shfl_xor_sync(0xFFFFFFFFu, j1, o), oj2 = __shfl_xor_sync(0xFFFFFFFFu, j2, o);
        top2_lex(b1, j1, b2, j2, ob1, oj1);
        top2_lex(b1, j1, b2, j2, ob2, oj2);
    }
}

// One warp per row.  The candidates of all splits whose BF16 value lies in the
// window are pooled in shared memory and re-scored one per lane, so the row
// costs about one FP32-form evaluation whatever the split they came from.
__global__ void __launch_bounds__(kRerankWarps * 32)
k_rerank(const float* A, const uint8_t* vA, const float* B, const float* nb32, const float4* pv, const int4* pj, int S,
         long long NA, float delta, float4* out_part, int32_t* rescan_rows, int32_t* rescan_count)
{
    __shared__ __align__(16) float qa[kRerankWarps][128];
    __shared__ int pool[kRerankWarps][kMaxCand];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * kRerankWarps + warp;
    if (i >= NA) return;
    if (!vA[i]) {   // an invalid query is never matched: nothing to rank
        if (lane == 0) out_part[i] = make_float4(INFINITY, INFINITY, __int_as_float(-1), __int_as_float(-1));
        return;
    }
    reinterpret_cast<float4*>(qa[warp])[lane] = reinterpret_cast<const float4*>(A + i * 128)[lane];
    // lane c holds the kTopK candidates of split c (S <= 32)
    float cv[kTopK];
    int cj[kTopK];
    float t4 = INFINITY;   // smallest k-th best value over the splits
    if (lane < S) {
        const float4* v = pv + ((long long)lane * NA + i) * 2;
        const int4* j = pj + ((long long)lane * NA + i) * 2;
        const float4 v0 = v[0], v1 = v[1];
        const int4 j0 = j[0], j1 = j[1];
        cv[0] = v0.x; cv[1] = v0.y; cv[2] = v0.z; cv[3] = v0.w;
        cv[4] = v1.x; cv[5] = v1.y; cv[6] = v1.z; cv[7] = v1.w;
        cj[0] = j0.x; cj[1] = j0.y; cj[2] = j0.z; cj[3] = j0.w;
        cj[4] = j1.x; cj[5] = j1.y; cj[6] = j1.z; cj[7] = j1.w;
#pragma unroll
        for (int k = 0; k < kTopK; ++k)
            if (cv[k] >= 1.0e38f) { cv[k] = INFINITY; cj[k] = -1; }
        t4 = cv[kTopK - 1];
    } else {
#pragma unroll
        for (int k = 0; k < kTopK; ++k) { cv[k] = INFINITY; cj[k] = -1; }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) t4 = fminf(t4, __shfl_xor_sync(0xFFFFFFFFu, t4, o));
    // second-smallest BF16 value over all candidates
    float m1 = cv[0], m2 = cv[1];
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float o1 = __shfl_xor_sync(0xFFFFFFFFu, m1, o);
        const float o2 = __shfl_xor_sync(0xFFFFFFFFu, m2, o);
        const float n1 = fminf(m1, o1);
        const float n2 = fminf(fmaxf(m1, o1), fminf(m2, o2));
        m1 = n1;
        m2 = n2;
    }
    const float window = m2 + 2.f * delta;
    // pool the window's candidates (lane order, then list order)
    int mine = 0;
#pragma unroll
    for (int k = 0; k < kTopK; ++k) mine += (cj[k] >= 0 && cv[k] <= window);
    int off = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, off, o);
        if (lane >= o) off += v;
    }
    const int n = __shfl_sync(0xFFFFFFFFu, off, 31);
    off -= mine;
#pragma unroll
    for (int k = 0; k < kTopK; ++k)
        if (cj[k] >= 0 && cv[k] <= window) pool[warp][off++] = cj[k];
    __syncwarp();
    // exact FP32-form values, one candidate per lane
    float b1 = INFINITY, b2 = INFINITY;
    int j1 = -1, j2 = -1;
    for (int c = lane; c < n; c += 32) {
        const int j = pool[warp][c];
        top2_lex(b1, j1, b2, j2, fp32_form_value(qa[warp], B + (long long)j * 128, __ldg(nb32 + j)), j);
    }
    warp_top2(b1, j1, b2, j2);
    if (lane == 0) {
        // every column outside the candidates has an FP32-form value >= t4 - delta
        // t4 = inf: no split saw more than kTopK valid columns, so every
        // column was a candidate
        const bool certified = isinf(t4) || b2 < t4 - delta;
        if (certified) {
            out_part[i] = make_float4(b1, b2, __int_as_float(j1), __int_as_float(j2));
        } else {
            const int slot = atomicAdd(rescan_count, 1);
            rescan_rows[slot] = (int32_t)i;
        }
    }
}

// FP32 re-scan of the queued rows.  Work item = (group of up to kRescanRows
// queued rows, one of kRescanGroups column ranges).  The range is walked in
// chunks of 128 columns: the chunk is staged in shared memory with coalesced
// loads (column pitch 132 floats: conflict-free 16-byte reads), then each
// thread forms the FP32 form's value of its column for every row of the group
// (sequential FMA over k, then fma(-2, dot, |b|^2)).  Per row, the item keeps
// the range's two smallest (value, column) pairs.
constexpr int kRescanThreads = 128;
constexpr int kRescanRows = 8;
constexpr int kRescanPitch = 132;
constexpr int kRescanGroups = 64;   // column ranges per queued row (partials per row)
constexpr size_t kRescanSmem = sizeof(float) * (kRescanThreads * kRescanPitch + 2 * kRescanRows * 128);

__global__ void __launch_bounds__(kRescanThreads)
k_rescan(const float* A, const float* B, const float* nb32, long long NB, const int32_t* rows, const int32_t* count,
         float4* part_r)
{
    extern __shared__ __align__(16) float rsm[];
    float* tb = rsm;                                   // [128 columns][kRescanPitch]
    float* qa = tb + kRescanThreads * kRescanPitch;    // [kRescanRows][128]
    float* sv = qa + kRescanRows * 128;                // [kRescanRows][128]
    __shared__ float4 run[kRescanRows];   // running (b1, b2, j1, j2) per row
    const int R = *count;
    const int groups = (R + kRescanRows - 1) / kRescanRows;
    const long long items = (long long)groups * kRescanGroups;
    const long long nchunks = (NB + kRescanThreads - 1) / kRescanThreads;
    const long long cpg = (nchunks + kRescanGroups - 1) / kRescanGroups;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float4* B4 = reinterpret_cast<const float4*>(B);
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int g = (int)(it / kRescanGroups);
        const int cg = (int)(it - (long long)g * kRescanGroups);
        const int r0 = g * kRescanRows, nr = min(kRescanRows, R - r0);
        __syncthreads();
        for (int e = tid; e < kRescanRows * 32; e += kRescanThreads) {
            const int r = e >> 5, q = e & 31;
            reinterpret_cast<float4*>(qa)[e] =
                r < nr ? reinterpret_cast<const float4*>(A + (long long)rows[r0 + r] * 128)[q] : make_float4(0, 0, 0, 0);
        }
        if (tid < kRescanRows)
            run[tid] = make_float4(INFINITY, INFINITY, __int_as_float(-1), __int_as_float(-1));
        for (long long ch = (long long)cg * cpg; ch < min(nchunks, (long long)(cg + 1) * cpg); ++ch) {
            const long long jb = ch * kRescanThreads;
            __syncthreads();
#pragma unroll 8
            for (int q = 0; q < 32; ++q) {   // float4 e = tid + 128 q: column e / 32, quarter e % 32
                const int e = tid + kRescanThreads * q;
                const int col = e >> 5, k4 = e & 31;
                const long long j = jb + col;
                const float4 w = j < NB ? __ldg(B4 + j * 32 + k4) : make_float4(0, 0, 0, 0);
                *reinterpret_cast<float4*>(tb + col * kRescanPitch + 4 * k4) = w;
            }
            __syncthreads();
            const long long j = jb + tid;
            const float nbj = j < NB ? __ldg(nb32 + j) : INFINITY;
            if (!isinf(nbj)) {
                float acc[kRescanRows];
#pragma unroll
                for (int r = 0; r < kRescanRows; ++r) acc[r] = 0.f;
                const float4* b4 = reinterpret_cast<const float4*>(tb + tid * kRescanPitch);
#pragma unroll 4
                for (int k4 = 0; k4 < 32; ++k4) {
                    const float4 w = b4[k4];
#pragma unroll
                    for (int r = 0; r < kRescanRows; ++r) {
                        const float4 a = reinterpret_cast<const float4*>(qa + r * 128)[k4];
                        acc[r] = fmaf(a.x, w.x, acc[r]);
                        acc[r] = fmaf(a.y, w.y, acc[r]);
                        acc[r] = fmaf(a.z, w.z, acc[r]);
                        acc[r] = fmaf(a.w, w.w, acc[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < kRescanRows; ++r) sv[r * 128 + tid] = fmaf(-2.f, acc[r], nbj);
            } else {
#pragma unroll
                for (int r = 0; r < kRescanRows; ++r) sv[r * 128 + tid] = INFINITY;
            }
            __syncthreads();
            // warp w merges rows w and w + 4 of this chunk into the running lists
            for (int r = warp; r < nr; r += kRescanThreads / 32) {
                float b1 = INFINITY, b2 = INFINITY;
                int j1 = -1, j2 = -1;
#pragma unroll
                for (int c = lane; c < kRescanThreads; c += 32) {
                    const float x = sv[r * 128 + c];
                    if (!isinf(x)) top2_lex(b1, j1, b2, j2, x, (int)(jb + c));
                }
                warp_top2(b1, j1, b2, j2);
                if (lane == 0) {
                    float4 q = run[r];
                    float c1 = q.x, c2 = q.y;
                    int i1 = __float_as_int(q.z), i2 = __float_as_int(q.w);
                    top2_lex(c1, i1, c2, i2, b1, j1);
                    top2_lex(c1, i1, c2, i2, b2, j2);
                    run[r] = make_float4(c1, c2, __int_as_float(i1), __int_as_float(i2));
                }
            }
        }
        __syncthreads();
        if (tid < nr) part_r[(long long)(r0 + tid) * kRescanGroups + cg] = run[tid];
    }
}

// Merge the re-scan partials of queued row r into the row's single partial.
__global__ void k_rescan_merge(const float4* part_r, int nchunks, const int32_t* rows, const int32_t* count,
                               float4* out_part)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    if (r >= *count) return;
    float b1 = INFINITY, b2 = INFINITY;
    int j1 = -1, j2 = -1;
    for (int c = lane; c < nchunks; c += 32) {
        const float4 q = part_r[r * nchunks + c];
        top2_lex(b1, j1, b2, j2, q.x, __float_as_int(q.z));
        top2_lex(b1, j1, b2, j2, q.y, __float_as_int(q.w));
    }
    warp_top2(b1, j1, b2, j2);
    if (lane == 0) out_part[rows[r]] = make_float4(b1, b2, __int_as_float(j1), __int_as_float(j2));
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* m, const void* base, long long rows, uint32_t box_rows)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {128, (cuuint64_t)rows};
    cuuint64_t strides[1] = {256};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Column splits S: minimise (rounds of units per CTA) x (tiles per unit + ~2
// tiles of per-unit A reload and pipeline refill).
int pick_tc_splits(int nrp, long long NB, int sms)
{
    const long long tiles = (NB + kTileN - 1) / kTileN;
    int best = 1;
    double best_cost = 1e300;
    for (int S = 1; S <= 32 && S <= tiles; ++S) {
        const long long U = (long long)nrp * S;
        const double rounds = (double)((U + sms - 1) / sms);
        const double cost = rounds * (double)((tiles + S - 1) / S + 2);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = S; }
    }
    return best;
}

struct TcLayout {
    int S;
    size_t off_nb16, off_na, off_nb32, off_pv, off_pj, off_part1, off_rows, off_cnt, off_part_r, total;
};

TcLayout tc_layout(long long NA, long long NB, int sms)
{
    TcLayout L;
    const int nrp = (int)((NA + kRowsPerUnit - 1) / kRowsPerUnit);
    L.S = pick_tc_splits(nrp, NB, sms);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
    L.off_nb16 = take(sizeof(float) * (size_t)NB + 64);
    L.off_na = take(sizeof(float) * (size_t)NA);
    L.off_nb32 = take(sizeof(float) * (size_t)NB);
    L.off_pv = take(sizeof(float4) * 2 * (size_t)L.S * NA);
    L.off_pj = take(sizeof(int4) * 2 * (size_t)L.S * NA);
    L.off_part1 = take(sizeof(float4) * (size_t)NA);
    L.off_rows = take(sizeof(int32_t) * (size_t)NA);
    L.off_cnt = take(64);
    L.off_part_r = take(sizeof(float4) * kRescanGroups * (size_t)NA);
    L.total = o + 256;
    return L;
}

}  // namespace

size_t match_bf16_workspace(int64_t NA, int64_t NB, int num_sms) { return tc_layout(NA, NB, num_sms).total; }

// Number of rows the last BF16 match re-scanned in FP32 (synchronous read).
int64_t match_bf16_rescans(const void* ws, int64_t NA, int64_t NB, int num_sms, cudaStream_t s)
{
    const TcLayout L = tc_layout(NA, NB, num_sms);
    const uint8_t* w = reinterpret_cast<const uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    int32_t c = -1;
    if (cudaMemcpyAsync(&c, w + L.off_cnt, sizeof c, cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return c;
}

cudaError_t launch_match_bf16(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s)
{
    if (a.NA == 0) return cudaSuccess;
    const TcLayout L = tc_layout(a.NA, a.NB, num_sms);
    if (ws_bytes < L.total) return cudaErrorInvalidValue;
    uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    float* nb16 = reinterpret_cast<float*>(w + L.off_nb16);
    float* na = reinterpret_cast<float*>(w + L.off_na);
    float* nb32 = reinterpret_cast<float*>(w + L.off_nb32);
    float4* pv = reinterpret_cast<float4*>(w + L.off_pv);
    int4* pj = reinterpret_cast<int4*>(w + L.off_pj);
    float4* part1 = reinterpret_cast<float4*>(w + L.off_part1);
    int32_t* rows = reinterpret_cast<int32_t*>(w + L.off_rows);
    int32_t* cnt = reinterpret_cast<int32_t*>(w + L.off_cnt);
    float4* part_r = reinterpret_cast<float4*>(w + L.off_part_r);
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    k_row_norms<<<(unsigned)((a.NA * 32 + 255) / 256), 256, 0, s>>>(a.dA, a.vA, a.NA, na, 0.f);
    if (a.NB > 0) {
        k_row_norms<<<(unsigned)((a.NB * 32 + 255) / 256), 256, 0, s>>>(a.dB, a.vB, a.NB, nb32, INFINITY);
        k_row_norms_bf16<<<(unsigned)((a.NB * 32 + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<const __nv_bfloat16*>(a.dB16), a.vB, a.NB, nb16);
        CUtensorMap tA, tB;
        if (!make_map(&tA, a.dA16, a.NA, kRowsPerUnit) || !make_map(&tB, a.dB16, a.NB, kTileN))
            return cudaErrorInvalidValue;
        TcParams p;
        p.NA = a.NA;
        p.NB = a.NB;
        p.nrp = (int)((a.NA + kRowsPerUnit - 1) / kRowsPerUnit);
        p.S = L.S;
        const long long tiles = (a.NB + kTileN - 1) / kTileN;
        p.cps = ((tiles + L.S - 1) / L.S) * kTileN;
        p.nb16 = nb16;
        p.pv = pv;
        p.pj = pj;
        p.status = a.status;
        const int U = p.nrp * p.S;
        const int grid = U < num_sms ? U : num_sms;
        if ((e = cudaFuncSetAttribute(k_match_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC)) !=
            cudaSuccess)
            return e;
        if (a.ev0) cudaEventRecord(a.ev0, s);
        k_match_tc<<<grid, kThreadsTC, kSmemTC, s>>>(tA, tB, p);
        if (a.ev1) cudaEventRecord(a.ev1, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_rerank<<<(unsigned)((a.NA + kRerankWarps - 1) / kRerankWarps), kRerankWarps * 32, 0, s>>>(
            a.dA, a.vA, a.dB, nb32, pv, pj, L.S, a.NA, kDelta, part1, rows, cnt);
        if ((e = cudaFuncSetAttribute(k_rescan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRescanSmem)) !=
            cudaSuccess)
            return e;
        k_rescan<<<(unsigned)(4 * num_sms), kRescanThreads, kRescanSmem, s>>>(a.dA, a.dB, nb32, a.NB, rows, cnt,
                                                                               part_r);
        k_rescan_merge<<<(unsigned)((a.NA + 7) / 8), 256, 0, s>>>(part_r, kRescanGroups, rows, cnt, part1);
        k_match_finish<<<(unsigned)((a.NA + 255) / 256), 256, 0, s>>>(part1, 1, a.NA, na, a.vA, a.ratio2, a.delta_s2,
                                                                      a.match, a.d1, a.d2);
    } else {
        k_match_finish<<<(unsigned)((a.NA + 255) / 256), 256, 0, s>>>(part1, 0, a.NA, na, a.vA, a.ratio2, a.delta_s2,
                                                                      a.match, a.d1, a.d2);
    }
    return cudaGetLastError();
}

}  // namespace lp
