// Nearest-neighbour matching (Sec. 2.4, Eq. 6) with BF16 (or E4M3) tensor
// cores (tcgen05) for sm_103a, re-ranked in FP32 so that every decision equals
// the plain FP32 form's.  The E4M3 form runs the same passes on 128-byte
// operand rows with kind::f8f6f4 MMAs (K = 32) and E4M3's error bound; see the
// constants below window_top.
//
// Distances: the accumulator of one MMA holds D = a~.b~ over the eight K-steps
// of the BF16 descriptors.  Valid descriptors have unit norm, so the squared
// distance up to the row constant |a|^2 is v = |b|^2 - 2 a.b, estimated by
// v~ = 1 - 2 D.  An invalid B row is all zero: v~ = 1, outside the candidate
// window of every row whose second-best value is well below 1 (its exact value
// is +inf, so it can never be ranked).
//
// k_match_tc<pass> (persistent, one CTA per SM, 10 warps, no clusters):
//   warp 0    TMA producer: per work unit a 128-row A block (2 x 16 KB boxes,
//             128-byte swizzle), then 256-row B tiles (2 x 32 KB boxes) into
//             a 3-stage ring; plain per-CTA loads.
//   warp 1    allocates all 512 TMEM columns; one lane issues
//             tcgen05.mma.cta_group::1.kind::f16 (M = 128, N = 256, K = 16,
//             BF16 x BF16 -> FP32), 8 per B tile, into one of two 256-column
//             TMEM accumulator buffers; tcgen05.commit releases the B stage
//             and hands the buffer to the epilogue.
//   warps 2-9 epilogue: each thread owns one A row and one 128-column range
//             of every tile (LP_TC_EPI_RANGES = 4: 16 warps, 64-column ranges);
//             it loads its part of the row from TMEM (tcgen05.ld 32x32b.x32),
//             returns the buffer, then works on registers.
//             Pass 1 (every third tile): the two largest 32-column chunk
//             maxima of D per (split, range, row), written as v.  Pass 2 (all
//             tiles): every column with v <= T (a three-input max tree per
//             chunk finds the rare chunks that hold one) is stored in the
//             candidate sub-list of (row, split, range).  Exactly one thread
//             owns a sub-list, so it keeps its count in a register: no
//             atomics, and no store waits for anything.
//   A work unit is (128-row block, one of S column splits of B); a CTA takes
//   a contiguous run of units, so consecutive units usually reuse the A block.
//   Every mbarrier wait is bounded by a 2 s clock limit; on expiry the CTA
//   records LP_ERR_TIMEOUT, drains its copies, frees its TMEM and returns.
//
// k_row_threshold: the certification point x = m2 + margin per row, m2 the
//   second smallest of the pass-1 values.  With unit, non-negative
//   descriptors and BF16 unit roundoff u = 2^-8, a~_k b~_k = a_k b_k (1 + e),
//   |e| <= 2u + u^2, and 2 a.b_j = |b_j|^2 - v_j <= 1 + eps - v_j, so
//   |v~_j - v_j| <= delta(v_j) = c + k (1 + eps - v_j), k = 2u + u^2, c the
//   norm and accumulation allowance.  Pass 2 lists every column with
//   v~ <= T = x + delta(x).  v + delta(v) increases with v, so a column outside
//   the list (v~ > T) has an exact value above x (invalid columns: +inf).
// k_rerank (one warp per row): the candidates are re-scored with exactly the
//   FP32 form's arithmetic (sequential FMA over k, then fma(-2, dot, |b|^2)),
//   so their values are bit-identical to the FP32 form's; a row is certified
//   when its exact second-best is < x.  Rows with an overflowed sub-list
//   or without that margin are re-scanned in FP32 (k_rescan, k_rescan_merge).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "lp_internal.cuh"

namespace lp {

__global__ void k_row_norms(const float* d, const uint8_t* v, long long n, float* out, float invalid_value);
__global__ void k_match_finish(const float4* part, int S, long long NA, const float* na, const uint8_t* vA,
                               float ratio2, float delta_s2, int32_t* match, float* d1, float* d2);

namespace {

constexpr int kRowsPerUnit = 128;       // one M = 128 row block per CTA
constexpr int kTileN = 256;             // B rows per tile (MMA N)
constexpr int kTmemBufs = 2;            // accumulator buffers of kTileN columns (512 TMEM columns)
constexpr int kStages = 3;              // B ring depth
#ifndef LP_TC_EPI_RANGES
#define LP_TC_EPI_RANGES 2
#endif
constexpr int kRanges = LP_TC_EPI_RANGES;       // column ranges of a tile, one epilogue warp per (range, lane quarter)
constexpr int kEpiWarps = 4 * kRanges;
constexpr int kThreadsTC = 64 + 32 * kEpiWarps; // producer warp, MMA warp, epilogue warps
constexpr int kRangeCols = kTileN / kRanges;    // columns of a tile one epilogue thread scans
constexpr int kChunks = kRangeCols / 32;
static_assert(kRanges == 2 || kRanges == 4, "epilogue column ranges");
constexpr uint32_t kABytes = kRowsPerUnit * 128 * 2;   // 32 KB
constexpr uint32_t kBBytes = kTileN * 128 * 2;         // 64 KB per stage
// 32 KB + 3 x 64 KB + 2 KB = 231,424 bytes of the 232,448 a CTA may opt into
static_assert(kABytes + kStages * kBBytes + 2048 <= 232448, "shared memory");
constexpr uint32_t kSmemTC = kABytes + kStages * kBBytes + 1024 /*barriers*/ + 1024 /*align slack*/;
// pass-2 candidates kept per (row, column split, column range); a row with a
// longer sub-list is re-scanned
#ifndef LP_CAND_SUBCAP
#define LP_CAND_SUBCAP 32
#endif
constexpr int kSubCap = LP_CAND_SUBCAP;
constexpr int kMaxSplits = 16;          // column splits S (kRanges S sub-lists per row)
// largest threshold a row may get (rows with fewer than two sampled columns)
constexpr float kCandCap = 1.0e38f;
// margin of the certification point above m2 (about five standard deviations
// of the BF16 rounding error of a value); a row whose exact second-best
// exceeds m2 + kMargin is not certified and is re-scanned
#ifndef LP_CAND_MARGIN
#define LP_CAND_MARGIN 5.0e-3f
#endif
constexpr float kMargin = LP_CAND_MARGIN;
// Pass 1 visits every kPass1Stride-th column tile: its m2 is then the second
// smallest chunk minimum of a spread subset, still the value of a second
// column, so still >= B; the candidate window widens a little.
#ifndef LP_PASS1_STRIDE
#define LP_PASS1_STRIDE 3
#endif
constexpr int kPass1Stride = LP_PASS1_STRIDE;
// |v~ - v| <= delta(v) = kDeltaC + kDeltaK (1 + kNormEps - v) for every valid
// column, v~ = 1 - 2 a~.b~ (the tensor-core value) and v = |b|^2 - 2 a.b (the
// FP32 form's): (2u + u^2) 2 a.b for the BF16 rounding of both operands
// (u = 2^-8, non-negative entries), |1 - |b|^2| <= kNormEps = 5e-5 for FP32
// unit descriptors (their rounding and the FP32 form's own norm
// accumulation), and 1.5e-4 of FP32 accumulation on both sides.
constexpr float kNormEps = 5e-5f;
constexpr float kDeltaK = 2.0f / 256.0f + 1.0f / 65536.0f;
constexpr float kDeltaC = kNormEps + 1.5e-4f;

// Top of the candidate window of a row certified at x: T = x + delta(x).
__host__ __device__ __forceinline__ float window_top(float x)
{
    const float r = 1.f + kNormEps - x;
    return x + kDeltaC + kDeltaK * (r > 0.f ? r : 0.f);
}

// The E4M3 form (LP_PREC_FP8).  Descriptors are scaled by kFp8Scale = 2^8 (a
// unit descriptor's entries lie in [0, 1], so the largest becomes <= 256 <
// 448, the E4M3 maximum) and rounded to E4M3; the accumulator then holds
// 2^16 D.  E4M3 keeps 3 mantissa bits: u = 2^-4 for normal values, and an
// absolute error of at most 2^-10 / kFp8Scale for the entries that fall in
// its subnormal range.  So |v~ - v| <= kDeltaC8 + kDeltaK8 (1 + kNormEps - v)
// with kDeltaK8 = 2u + u^2 and kDeltaC8 the BF16 allowance plus the
// subnormal term, 2 (1 + u) (sum a + sum b) 2^-18 <= 2 * 2.2 * 11.4 * 2^-18.
constexpr float kFp8Scale = 256.0f;
constexpr float kFp8AccScale = 65536.0f;                  // kFp8Scale^2
constexpr float kDeltaK8 = 2.0f / 16.0f + 1.0f / 256.0f;
constexpr float kDeltaC8 = kDeltaC + 2.0e-4f;
// margin of the certification point above m2 for the E4M3 form (its values
// carry about 16 times the BF16 rounding error)
constexpr float kMargin8 = 2.0e-2f;

template <int kElem>
__host__ __device__ __forceinline__ float window_top_e(float x)
{
    if (kElem == 0) return window_top(x);
    const float r = 1.f + kNormEps - x;
    return x + kDeltaC8 + kDeltaK8 * (r > 0.f ? r : 0.f);
}

// Operand sizes of one element type: BF16 rows are 256 bytes (two 128-byte
// swizzle atoms, two TMA boxes), E4M3 rows 128 bytes (one of each).
template <int kElem>
struct Opnd {
    static constexpr uint32_t kA = kRowsPerUnit * 128 * (kElem ? 1 : 2);
    static constexpr uint32_t kB = kTileN * 128 * (kElem ? 1 : 2);
    static constexpr int kBoxes = kElem ? 1 : 2;
};

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

// One try of a phase wait; the thread may be suspended for up to kSuspendNs
// (it resumes as soon as the phase completes), so waiting warps take few
// issue slots from the epilogue.
#ifndef LP_TC_SUSPEND_NS
#define LP_TC_SUSPEND_NS 10000
#endif
constexpr uint32_t kSuspendNs = LP_TC_SUSPEND_NS;
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
        if ((it & 15u) == 0) {
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
// N = kTileN = 256, M = 128.
constexpr uint32_t kIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kRowsPerUnit >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor, kind::f8f6f4: D = FP32, A = B = E4M3 (format 0),
// both K-major, N = kTileN = 256, M = 128.
constexpr uint32_t kIdesc8 = (1u << 4) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kRowsPerUnit >> 4) << 24);

__device__ __forceinline__ void mma_e4m3(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(kIdesc8), "r"(accumulate)
        : "memory");
}

// Arrive on the mbarrier at `bar` when this thread's MMAs complete.
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
    int nrb;               // number of 128-row blocks
    int S;                 // column splits (<= kMaxSplits)
    long long cps;         // columns per split (multiple of kTileN)
    float2* pm;            // pass 1 output [kRanges S][NA]: per split and column range, the two smallest chunk minima
    const float* thr;      // pass 2 input [NA]: candidate threshold per row (-inf: none)
    int32_t* cand;         // pass 2 output [NA][kRanges S][kSubCap]: candidate columns per (row, split, range)
    int32_t* ncand;        // pass 2 output [NA][kRanges S]: candidates found per sub-list (may exceed kSubCap)
    int tstride;           // tiles visited: every tstride-th 256-column tile of a split
    int32_t* status;
};

// Unit u = (128-row block rb, column split).  Consecutive units share a row
// block and each CTA takes a contiguous run of units, so the A block is
// usually reused.
__device__ __forceinline__ void unit_range(const TcParams& p, int u, int& rb, int& split, long long& c0, int& ntiles)
{
    rb = u / p.S;
    split = u - rb * p.S;
    c0 = (long long)split * p.cps;
    long long c1 = c0 + p.cps;
    if (c1 > p.NB) c1 = p.NB;
    const int all = c1 > c0 ? (int)((c1 - c0 + kTileN - 1) / kTileN) : 0;
    ntiles = (all + p.tstride - 1) / p.tstride;
}

__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int kPass, int kElem>
__global__ void __launch_bounds__(kThreadsTC, 1)
k_match_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcParams p)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    constexpr uint32_t kAB = Opnd<kElem>::kA, kBB = Opnd<kElem>::kB;
    constexpr int kBoxes = Opnd<kElem>::kBoxes;
    uint8_t* sB = smem + kAB;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * kBB);
    // barrier slots
    uint64_t* full = bars;                 // [kStages]
    uint64_t* empty = bars + kStages;      // [kStages]
    uint64_t* tfull = bars + 2 * kStages;  // [kTmemBufs]
    uint64_t* tempty = tfull + kTmemBufs;  // [kTmemBufs]
    uint64_t* afull = tempty + kTmemBufs;  // [1]
    uint64_t* aempty = afull + 1;          // [1]
    uint64_t* drain = aempty + 1;          // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int U = p.nrb * p.S;
    const int nct = (int)gridDim.x, cta = (int)blockIdx.x;
    const int per = U / nct, rem = U % nct;
    const int u_begin = cta * per + min(cta, rem);
    const int u_end = u_begin + per + (cta < rem ? 1 : 0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < kTmemBufs; ++b) {
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
            int v = 0;         // A block counter of this CTA
            int armed[kStages];
            int a_armed = -1;
            for (int s = 0; s < kStages; ++s) armed[s] = -1;
            bool ok = true;
            int prev_rb = -1;
            for (int u = u_begin; u < u_end && ok; ++u) {
                int rb, split, ntiles;
                long long c0;
                unit_range(p, u, rb, split, c0, ntiles);
                if (ntiles == 0) continue;
                if (rb != prev_rb) {
                    ok = mbar_wait(smem_u32(aempty), (v & 1) ^ 1, abort_flag, p.status);
                    if (!ok) break;
                    mbar_expect_tx(smem_u32(afull), kAB);
#pragma unroll
                    for (int h = 0; h < kBoxes; ++h)
                        tma_load_2d(smem_u32(sA + h * (kAB / kBoxes)), &tmA, 64 * h, rb * kRowsPerUnit,
                                    smem_u32(afull));
                    a_armed = v;
                    ++v;
                    prev_rb = rb;
                }
                for (int t = 0; t < ntiles; ++t, ++n) {
                    const int s = (int)(n % kStages);
                    const uint32_t k = (uint32_t)(n / kStages);
                    ok = mbar_wait(smem_u32(&empty[s]), (k & 1) ^ 1, abort_flag, p.status);
                    if (!ok) break;
                    uint8_t* dst = sB + s * kBB;
                    const int y = (int)(c0 + (long long)t * p.tstride * kTileN);
                    mbar_expect_tx(smem_u32(&full[s]), kBB);
#pragma unroll
                    for (int h = 0; h < kBoxes; ++h)
                        tma_load_2d(smem_u32(dst + h * (kBB / kBoxes)), &tmB, 64 * h, y, smem_u32(&full[s]));
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
            // descriptors of the fixed buffers; an operand at byte offset o from
            // a base is the base descriptor + (o >> 4) (the 14-bit start field
            // never carries: shared addresses stay below 256 KB)
            const uint64_t dA0 = sdesc(smem_u32(sA)), dB0 = sdesc(smem_u32(sB));
            long long n = 0;
            int v = 0;
            bool ok = true;
            int prev_rb = -1;
            for (int u = u_begin; u < u_end && ok; ++u) {
                int rb, split, ntiles;
                long long c0;
                unit_range(p, u, rb, split, c0, ntiles);
                if (ntiles == 0) continue;
                if (rb != prev_rb) {
                    // release the previous A block once its MMAs are done, then
                    // wait for the new one
                    if (v > 0) mma_commit(smem_u32(aempty));
                    ok = mbar_wait(smem_u32(afull), v & 1, abort_flag, p.status);
                    ++v;
                    prev_rb = rb;
                    if (!ok) break;
                    tc_fence_after();
                }
                for (int t = 0; t < ntiles; ++t, ++n) {
                    const int s = (int)(n % kStages);
                    const uint32_t k = (uint32_t)(n / kStages);
                    const int b = (int)(n % kTmemBufs);
                    const uint32_t kb = (uint32_t)(n / kTmemBufs);
                    ok = mbar_wait(smem_u32(&tempty[b]), (kb & 1) ^ 1, abort_flag, p.status);
                    if (!ok) break;
                    ok = mbar_wait(smem_u32(&full[s]), k & 1, abort_flag, p.status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint64_t dB = dB0 + (uint64_t)((s * kBB) >> 4);
                    const uint32_t d = tmem + (uint32_t)(b * kTileN);
                    // 32 bytes of K per MMA: K = 16 BF16 or K = 32 E4M3 values
#pragma unroll
                    for (int h = 0; h < kBoxes; ++h)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = dA0 + (uint64_t)((h * (kAB / kBoxes) + kk * 32) >> 4);
                            const uint64_t bd = dB + (uint64_t)((h * (kBB / kBoxes) + kk * 32) >> 4);
                            if (kElem == 0)
                                mma_bf16(d, ad, bd, (h | kk) ? 1u : 0u);
                            else
                                mma_e4m3(d, ad, bd, (h | kk) ? 1u : 0u);
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
        // The accumulator holds D = -v / 2: smaller v is larger D.
        // Pass 1: per (split, range, row) the two largest chunk maxima of D (a
        //   chunk = 32 columns), which name two different columns; written as v.
        // Pass 2: every column with v <= T (D >= -T / 2) is a candidate, stored
        //   in this thread's own sub-list of the row.
        const int q = warp & 3;                 // TMEM lane quarter this warp may access
        const int rg = (warp - 2) >> 2;         // columns [rg kRangeCols, (rg + 1) kRangeCols) of a tile
        const int row_in_unit = q * 32 + lane;
        long long n = 0;
        bool ok = true;
        for (int u = u_begin; u < u_end && ok; ++u) {
            int rb, split, ntiles;
            long long c0;
            unit_range(p, u, rb, split, c0, ntiles);
            long long c1 = c0 + p.cps;
            if (c1 > p.NB) c1 = p.NB;
            const long long row = (long long)rb * kRowsPerUnit + row_in_unit;
            const bool live = row < p.NA;
            const long long sub = (live ? row : 0) * (kRanges * p.S) + split * kRanges + rg;
            int32_t* const dst = p.cand + sub * kSubCap;
            float d1 = -INFINITY, d2 = -INFINITY;                                    // pass 1
            // pass 2: v~ = 1 - 2 D <= T  <=>  D >= (1 - T) / 2 (1e-6 lower: rounding of TD)
            // (the E4M3 accumulator holds kFp8AccScale D: the threshold is scaled
            // instead of every value, exactly, by a power of two)
            const float TD = (kPass == 2 && live)
                                 ? (0.5f * (1.f - window_top_e<kElem>(p.thr[row])) - 1e-6f) *
                                       (kElem ? kFp8AccScale : 1.f)
                                 : INFINITY;
            int nc = 0;
            for (int t = 0; t < ntiles; ++t, ++n) {
                const int b = (int)(n % kTmemBufs);
                const uint32_t kb = (uint32_t)(n / kTmemBufs);
                ok = mbar_wait(smem_u32(&tfull[b]), kb & 1, abort_flag, p.status);
                if (!ok) break;
                tc_fence_after();
                const long long cbase = c0 + (long long)t * p.tstride * kTileN + rg * kRangeCols;
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kTileN + rg * kRangeCols);
                // the thread's columns of the tile row in registers, then the buffer goes back to the MMA
                uint32_t r[kChunks][32];
#pragma unroll
                for (int ch = 0; ch < kChunks; ++ch) tmem_ld32(tbase + 32 * ch, r[ch]);
#pragma unroll
                for (int ch = 0; ch < kChunks; ++ch) tmem_wait(r[ch]);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
#pragma unroll
                for (int ch = 0; ch < kChunks; ++ch) {
                    float dv[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) dv[i] = __uint_as_float(r[ch][i]);
                    const long long j0 = cbase + ch * 32;
                    if (j0 + 32 > c1) {   // columns past the split or past NB (zero-filled rows)
#pragma unroll
                        for (int i = 0; i < 32; ++i) dv[i] = j0 + i < c1 ? dv[i] : -INFINITY;
                    }
                    float gx[4];
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        gx[g] = max3f(max3f(dv[8 * g + 0], dv[8 * g + 1], dv[8 * g + 2]),
                                      max3f(dv[8 * g + 3], dv[8 * g + 4], dv[8 * g + 5]),
                                      fmaxf(dv[8 * g + 6], dv[8 * g + 7]));
                    const float cmax = max3f(gx[0], gx[1], fmaxf(gx[2], gx[3])) * (kElem && kPass == 1 ? 1.f / kFp8AccScale : 1.f);
                    if (kPass == 1) {
                        const float lo = fminf(d1, cmax);
                        d1 = fmaxf(d1, cmax);
                        d2 = fmaxf(d2, lo);
                    } else if (cmax >= TD) {
                        // bit i: column j0 + i qualifies; one store per candidate
                        uint32_t m = 0;
#pragma unroll
                        for (int i = 0; i < 32; ++i) m |= (dv[i] >= TD ? 1u : 0u) << i;
                        while (m) {
                            const int j = (int)j0 + __ffs(m) - 1;
                            m &= m - 1;
                            if (nc < kSubCap) dst[nc] = j;
                            ++nc;
                        }
                    }
                }
            }
            if (!ok) break;
            if (kPass == 1 && live)
                p.pm[((long long)split * kRanges + rg) * p.NA + row] = make_float2(1.f - 2.f * d1, 1.f - 2.f * d2);
            if (kPass == 2 && live) p.ncand[sub] = nc;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ batched passes
// k_match_tc_batch: pass 1, the row thresholds and pass 2 of up to
// kBatchPairs pairs in one persistent launch.  Work units (pair, pass, 128-row
// block, column split) come from an atomic queue in a fixed order -- every
// pass-1 unit of every pair before any pass-2 unit -- so a unit a CTA waits for
// was taken earlier by a running CTA and every wait ends.  The producer warp
// takes the units and hands them to the MMA and epilogue warps through a ring
// of unit slots in shared memory.  A pass-1 epilogue warp, once its part of the
// row block's pass-1 values is written, adds 1 (release) to the row block's
// counter; a pass-2 unit's epilogue warps wait (bounded, 2 s, acquire) until
// the counter reaches 8 warps x S splits (+ a diagnostic hold), then form the
// row thresholds themselves (the arithmetic of k_row_threshold).  A wait that
// gives up records LP_ERR_TIMEOUT; every other wait of the launch then stops at
// its next check of the status word, and the CTAs drain and return.
constexpr int kBatchPairs = 64;
constexpr int kUnitSlots = 8;

struct TcBatchPair {
    long long NA, NB;
    int nrb, S;
    long long cps;
    float2* pm;            // [kRanges S][NA]
    float* thr;            // [NA] (written by pass 2 for the re-rank)
    int32_t* cand;         // [NA][kRanges S][kSubCap]
    int32_t* ncand;        // [NA][kRanges S]
    int32_t* done;         // [nrb] pass-1 warps finished per row block (zero at launch)
    const uint8_t* vA;     // [NA] query validity
    int tstride;           // pass-1 tile stride
};

struct TcBatch {
    CUtensorMap tA[kBatchPairs], tB[kBatchPairs];
    TcBatchPair pr[kBatchPairs];
    int u1[kBatchPairs + 1];   // prefix sums of pass-1 units (nrb S per pair)
    int n;                     // pairs
    int hold;                  // extra pass-1 completions a pass-2 unit waits for (diagnostic; 0 normally)
    int32_t* queue;            // next unit (zero at launch)
    int32_t* status;
};

struct BUnit {
    int pass, pair, rb, split;
    long long c0;
    int ntiles, stride;
};

__device__ __forceinline__ BUnit batch_unit(const TcBatch& b, int u)
{
    BUnit w;
    const int U1 = b.u1[b.n];
    w.pass = u < U1 ? 1 : 2;
    const int v = u < U1 ? u : u - U1;
    int p = 0;
    while (p + 1 < b.n && v >= b.u1[p + 1]) ++p;
    const TcBatchPair& q = b.pr[p];
    const int loc = v - b.u1[p];
    w.pair = p;
    w.rb = loc / q.S;
    w.split = loc - w.rb * q.S;
    w.c0 = (long long)w.split * q.cps;
    long long c1 = w.c0 + q.cps;
    if (c1 > q.NB) c1 = q.NB;
    const int all = c1 > w.c0 ? (int)((c1 - w.c0 + kTileN - 1) / kTileN) : 0;
    w.stride = w.pass == 1 ? q.tstride : 1;
    w.ntiles = (all + w.stride - 1) / w.stride;
    return w;
}

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu(int32_t* p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait of one lane for *cnt >= target; false on timeout or when the
// launch already failed (status word set).
__device__ __forceinline__ bool wait_count(const int32_t* cnt, int target, int32_t* status, volatile int* abort_flag)
{
    if (ld_acquire_gpu(cnt) >= target) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        __nanosleep(200);
        if (ld_acquire_gpu(cnt) >= target) return true;
        if ((it & 15u) == 0) {
            if (*abort_flag || ld_acquire_gpu(status) != 0) return false;
            if (globaltimer() - t0 > 2000000000ull) {
                set_status(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreadsTC, 1) k_match_tc_batch(const __grid_constant__ TcBatch b)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + kABytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + kStages * kBBytes);
    uint64_t* full = bars;                 // [kStages]
    uint64_t* empty = bars + kStages;      // [kStages]
    uint64_t* tfull = bars + 2 * kStages;  // [kTmemBufs]
    uint64_t* tempty = tfull + kTmemBufs;  // [kTmemBufs]
    uint64_t* afull = tempty + kTmemBufs;  // [1]
    uint64_t* aempty = afull + 1;          // [1]
    uint64_t* drain = aempty + 1;          // [1]
    uint64_t* ufull = drain + 1;           // [kUnitSlots] a unit id is in the slot
    uint64_t* uempty = ufull + kUnitSlots; // [kUnitSlots] the MMA lane and the 8 epilogue warps read it
    int32_t* uslot = reinterpret_cast<int32_t*>(uempty + kUnitSlots);   // [kUnitSlots]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(uslot + kUnitSlots);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int U = 2 * b.u1[b.n];

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int q = 0; q < kTmemBufs; ++q) {
            mbar_init(smem_u32(&tfull[q]), 1);
            mbar_init(smem_u32(&tempty[q]), kEpiWarps);
        }
        mbar_init(smem_u32(afull), 1);
        mbar_init(smem_u32(aempty), 1);
        mbar_init(smem_u32(drain), 1);
        for (int q = 0; q < kUnitSlots; ++q) {
            mbar_init(smem_u32(&ufull[q]), 1);
            mbar_init(smem_u32(&uempty[q]), 1 + kEpiWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
        // ---------------------------------------------------------- queue + TMA producer
        if (lane == 0) {
            long long n = 0;   // tile counter
            int v = 0;         // A block counter
            int armed[kStages];
            int a_armed = -1;
            for (int s = 0; s < kStages; ++s) armed[s] = -1;
            bool ok = true;
            int prev_key = -1, prev_pair = -1;
            for (int m = 0; ok; ++m) {
                const int slot = m % kUnitSlots;
                ok = mbar_wait(smem_u32(&uempty[slot]), ((uint32_t)(m / kUnitSlots) & 1) ^ 1, abort_flag, b.status);
                if (!ok) break;
                const int u = atomicAdd(b.queue, 1);
                uslot[slot] = u < U ? u : -1;
                mbar_arrive(smem_u32(&ufull[slot]));
                if (u >= U) break;
                const BUnit w = batch_unit(b, u);
                if (w.ntiles == 0) continue;
                if (w.pair != prev_pair) {
                    tma_prefetch_desc(&b.tA[w.pair]);
                    tma_prefetch_desc(&b.tB[w.pair]);
                    prev_pair = w.pair;
                }
                const int key = w.pair * 65536 + w.rb;
                if (key != prev_key) {
                    ok = mbar_wait(smem_u32(aempty), (v & 1) ^ 1, abort_flag, b.status);
                    if (!ok) break;
                    mbar_expect_tx(smem_u32(afull), kABytes);
                    tma_load_2d(smem_u32(sA), &b.tA[w.pair], 0, w.rb * kRowsPerUnit, smem_u32(afull));
                    tma_load_2d(smem_u32(sA + kABytes / 2), &b.tA[w.pair], 64, w.rb * kRowsPerUnit, smem_u32(afull));
                    a_armed = v;
                    ++v;
                    prev_key = key;
                }
                const int st = w.stride;
                for (int t = 0; t < w.ntiles; ++t, ++n) {
                    const int s = (int)(n % kStages);
                    const uint32_t k = (uint32_t)(n / kStages);
                    ok = mbar_wait(smem_u32(&empty[s]), (k & 1) ^ 1, abort_flag, b.status);
                    if (!ok) break;
                    uint8_t* dst = sB + s * kBBytes;
                    const int y = (int)(w.c0 + (long long)t * st * kTileN);
                    mbar_expect_tx(smem_u32(&full[s]), kBBytes);
                    tma_load_2d(smem_u32(dst), &b.tB[w.pair], 0, y, smem_u32(&full[s]));
                    tma_load_2d(smem_u32(dst + kBBytes / 2), &b.tB[w.pair], 64, y, smem_u32(&full[s]));
                    armed[s] = (int)k;
                }
            }
            if (!ok) {
                *abort_flag = 1;
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
            const uint64_t dA0 = sdesc(smem_u32(sA)), dB0 = sdesc(smem_u32(sB));
            long long n = 0;
            int v = 0;
            bool ok = true;
            int prev_key = -1;
            for (int m = 0; ok; ++m) {
                const int slot = m % kUnitSlots;
                ok = mbar_wait(smem_u32(&ufull[slot]), (uint32_t)(m / kUnitSlots) & 1, abort_flag, b.status);
                if (!ok) break;
                const int u = uslot[slot];
                mbar_arrive(smem_u32(&uempty[slot]));
                if (u < 0) break;
                const BUnit w = batch_unit(b, u);
                if (w.ntiles == 0) continue;
                const int key = w.pair * 65536 + w.rb;
                if (key != prev_key) {
                    if (v > 0) mma_commit(smem_u32(aempty));
                    ok = mbar_wait(smem_u32(afull), v & 1, abort_flag, b.status);
                    ++v;
                    prev_key = key;
                    if (!ok) break;
                    tc_fence_after();
                }
                for (int t = 0; t < w.ntiles; ++t, ++n) {
                    const int s = (int)(n % kStages);
                    const uint32_t k = (uint32_t)(n / kStages);
                    const int bb = (int)(n % kTmemBufs);
                    const uint32_t kb = (uint32_t)(n / kTmemBufs);
                    ok = mbar_wait(smem_u32(&tempty[bb]), (kb & 1) ^ 1, abort_flag, b.status);
                    if (!ok) break;
                    ok = mbar_wait(smem_u32(&full[s]), k & 1, abort_flag, b.status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint64_t dB = dB0 + (uint64_t)((s * kBBytes) >> 4);
                    const uint32_t d = tmem + (uint32_t)(bb * kTileN);
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = dA0 + (uint64_t)((h * (kABytes / 2) + kk * 32) >> 4);
                            const uint64_t bd = dB + (uint64_t)((h * (kBBytes / 2) + kk * 32) >> 4);
                            mma_bf16(d, ad, bd, (h | kk) ? 1u : 0u);
                        }
                    mma_commit(smem_u32(&empty[s]));
                    mma_commit(smem_u32(&tfull[bb]));
                }
            }
            mma_commit(smem_u32(drain));
            const uint64_t t0 = globaltimer();
            while (!mbar_try(smem_u32(drain), 0) && globaltimer() - t0 < 2000000000ull) {
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int q = warp & 3;
        const int rg = (warp - 2) >> 2;
        const int row_in_unit = q * 32 + lane;
        long long n = 0;
        for (int m = 0;; ++m) {
            const int slot = m % kUnitSlots;
            // every lane waits; the warp acts on one decision (they differ only after a timeout)
            if (!__all_sync(0xFFFFFFFFu, mbar_wait(smem_u32(&ufull[slot]), (uint32_t)(m / kUnitSlots) & 1, abort_flag,
                                                   b.status)))
                break;
            const int u = uslot[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&uempty[slot]));
            if (u < 0) break;
            const BUnit w = batch_unit(b, u);
            const TcBatchPair& pp = b.pr[w.pair];
            long long c1 = w.c0 + pp.cps;
            if (c1 > pp.NB) c1 = pp.NB;
            const long long row = (long long)w.rb * kRowsPerUnit + row_in_unit;
            const bool live = row < pp.NA;
            const long long sub = (live ? row : 0) * (kRanges * pp.S) + w.split * kRanges + rg;
            int32_t* const dst = pp.cand + sub * kSubCap;
            float TD = INFINITY;
            if (w.pass == 2) {
                // the row block's pass-1 values: every epilogue warp of its S pass-1 units has released them
                bool got = true;
                if (lane == 0) got = wait_count(pp.done + w.rb, kEpiWarps * pp.S + b.hold, b.status, abort_flag);
                if (!__shfl_sync(0xFFFFFFFFu, got, 0)) {
                    *abort_flag = 1;
                    break;
                }
                if (live) {
                    // x = m2 + margin (k_row_threshold's arithmetic), -inf for an invalid query row
                    float m1 = INFINITY, m2 = INFINITY;
                    for (int s2 = 0; s2 < kRanges * pp.S; ++s2) {
                        const float2 qv = pp.pm[(long long)s2 * pp.NA + row];
                        const float lo = fminf(qv.x, qv.y), hi = fmaxf(qv.x, qv.y);
                        m2 = fminf(fminf(m2, hi), fmaxf(m1, lo));
                        m1 = fminf(m1, lo);
                    }
                    const float xt = pp.vA[row] ? fminf(m2 + kMargin, kCandCap) : -INFINITY;
                    if (rg == 0) pp.thr[row] = xt;
                    TD = 0.5f * (1.f - window_top(xt)) - 1e-6f;
                }
            }
            float d1 = -INFINITY, d2 = -INFINITY;
            int nc = 0;
            bool ok = true;
            for (int t = 0; t < w.ntiles; ++t, ++n) {
                const int bb = (int)(n % kTmemBufs);
                const uint32_t kb = (uint32_t)(n / kTmemBufs);
                ok = mbar_wait(smem_u32(&tfull[bb]), kb & 1, abort_flag, b.status);
                if (!__all_sync(0xFFFFFFFFu, ok)) { ok = false; break; }
                tc_fence_after();
                const long long cbase = w.c0 + (long long)t * w.stride * kTileN + rg * kRangeCols;
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(bb * kTileN + rg * kRangeCols);
                uint32_t r[kChunks][32];
#pragma unroll
                for (int ch = 0; ch < kChunks; ++ch) tmem_ld32(tbase + 32 * ch, r[ch]);
#pragma unroll
                for (int ch = 0; ch < kChunks; ++ch) tmem_wait(r[ch]);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[bb]));
#pragma unroll
                for (int ch = 0; ch < kChunks; ++ch) {
                    float dv[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) dv[i] = __uint_as_float(r[ch][i]);
                    const long long j0 = cbase + ch * 32;
                    if (j0 + 32 > c1) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) dv[i] = j0 + i < c1 ? dv[i] : -INFINITY;
                    }
                    float gx[4];
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        gx[g] = max3f(max3f(dv[8 * g + 0], dv[8 * g + 1], dv[8 * g + 2]),
                                      max3f(dv[8 * g + 3], dv[8 * g + 4], dv[8 * g + 5]),
                                      fmaxf(dv[8 * g + 6], dv[8 * g + 7]));
                    const float cmax = max3f(gx[0], gx[1], fmaxf(gx[2], gx[3]));
                    if (w.pass == 1) {
                        const float lo = fminf(d1, cmax);
                        d1 = fmaxf(d1, cmax);
                        d2 = fmaxf(d2, lo);
                    } else if (cmax >= TD) {
                        uint32_t mk = 0;
#pragma unroll
                        for (int i = 0; i < 32; ++i) mk |= (dv[i] >= TD ? 1u : 0u) << i;
                        while (mk) {
                            const int j = (int)j0 + __ffs(mk) - 1;
                            mk &= mk - 1;
                            if (nc < kSubCap) dst[nc] = j;
                            ++nc;
                        }
                    }
                }
            }
            if (!ok) break;
            if (w.pass == 1) {
                if (live)
                    pp.pm[((long long)w.split * kRanges + rg) * pp.NA + row] =
                        make_float2(1.f - 2.f * d1, 1.f - 2.f * d2);
                __syncwarp();
                if (lane == 0) red_release_gpu(pp.done + w.rb, 1);
            } else if (live) {
                pp.ncand[sub] = nc;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
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

// Per row, the certification point x = m2 + kMargin (m2 the second smallest
// pass-1 value; capped for rows with fewer than two sampled columns), -inf for
// an invalid query row.
__global__ void k_row_threshold(const float2* pm, int S, long long NA, const uint8_t* vA, float* thr, float margin)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NA) return;
    float m1 = INFINITY, m2 = INFINITY;
    for (int s = 0; s < S; ++s) {
        const float2 q = pm[(long long)s * NA + i];
        const float lo = fminf(q.x, q.y), hi = fmaxf(q.x, q.y);
        m2 = fminf(fminf(m2, hi), fmaxf(m1, lo));
        m1 = fminf(m1, lo);
    }
    thr[i] = vA[i] ? fminf(m2 + margin, kCandCap) : -INFINITY;
}

// One warp per row: every candidate of the row's kRanges S sub-lists is re-scored
// with exactly the FP32 form's arithmetic, and the top 2 kept by (value,
// column).  Every column outside the lists has a BF16 value > window_top(x)
// and so an FP32-form value > x: the row is certified when its exact
// second-best is < x.  Rows with an overflowed sub-list or without that margin
// are queued for the FP32 re-scan.
__global__ void __launch_bounds__(kRerankWarps * 32)
k_rerank(const float* A, const uint8_t* vA, const float* B, const float* nb32, const int32_t* cand,
         const int32_t* ncand, int nsub, const float* thr, long long NA, float4* out_part, int32_t* rescan_rows,
         int32_t* rescan_count)
{
    __shared__ __align__(16) float qa[kRerankWarps][128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * kRerankWarps + warp;
    if (i >= NA) return;
    if (!vA[i]) {   // an invalid query is never matched: nothing to rank
        if (lane == 0) out_part[i] = make_float4(INFINITY, INFINITY, __int_as_float(-1), __int_as_float(-1));
        return;
    }
    const int32_t* cnt = ncand + i * nsub;
    const int32_t* lst = cand + i * (long long)nsub * kSubCap;
    const float T = thr[i];
    bool over = false;
    for (int q = lane; q < nsub; q += 32) over |= (unsigned)cnt[q] > (unsigned)kSubCap;
    bool ok = !__any_sync(0xFFFFFFFFu, over);
    float b1 = INFINITY, b2 = INFINITY;
    int j1 = -1, j2 = -1;
    if (ok) {
        reinterpret_cast<float4*>(qa[warp])[lane] = reinterpret_cast<const float4*>(A + i * 128)[lane];
        __syncwarp();
        // the row's candidates, 32 sub-lists at a time: lane l holds sub-list
        // l's count; an exclusive warp scan gives where each starts, and the
        // lane scoring candidate c finds its sub-list by binary search
        for (int s0 = 0; s0 < nsub; s0 += 32) {
            const int n_l = s0 + lane < nsub ? cnt[s0 + lane] : 0;
            int incl = n_l;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += v;
            }
            const int excl = incl - n_l, total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            for (int c0 = 0; c0 < total; c0 += 32) {
                const int c = c0 + lane;
                int lo = 0;
#pragma unroll
                for (int st = 16; st; st >>= 1) {
                    const int e = __shfl_sync(0xFFFFFFFFu, excl, lo + st);
                    if (e <= c) lo += st;
                }
                const int base = __shfl_sync(0xFFFFFFFFu, excl, lo);
                if (c < total) {
                    const int j = lst[(s0 + lo) * kSubCap + (c - base)];
                    top2_lex(b1, j1, b2, j2, fp32_form_value(qa[warp], B + (long long)j * 128, __ldg(nb32 + j)), j);
                }
            }
        }
        warp_top2(b1, j1, b2, j2);
        ok = b2 < T;   // T = x, the row's certification point
    }
    if (lane == 0) {
        if (ok) {
            out_part[i] = make_float4(b1, b2, __int_as_float(j1), __int_as_float(j2));
        } else {
            rescan_rows[atomicAdd(rescan_count, 1)] = (int32_t)i;
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
constexpr int kRescanGroups = 64;   // partial slots per row of A in the workspace

// Column ranges per queued row: as many as the workspace holds for R queued
// rows (R * G <= NA * kRescanGroups), at most one 128-column chunk each.
__device__ __forceinline__ int rescan_groups(int R, long long NA, long long nchunks)
{
    long long g = R > 0 ? (NA * kRescanGroups) / R : 1;
    if (g > nchunks) g = nchunks;
    return (int)(g < 1 ? 1 : g);
}
constexpr size_t kRescanSmem = sizeof(float) * (kRescanThreads * kRescanPitch + 2 * kRescanRows * 128);

__global__ void __launch_bounds__(kRescanThreads)
k_rescan(const float* A, const float* B, const float* nb32, long long NA, long long NB, const int32_t* rows,
         const int32_t* count, float4* part_r)
{
    extern __shared__ __align__(16) float rsm[];
    float* tb = rsm;                                   // [128 columns][kRescanPitch]
    float* qa = tb + kRescanThreads * kRescanPitch;    // [kRescanRows][128]
    float* sv = qa + kRescanRows * 128;                // [kRescanRows][128]
    __shared__ float4 run[kRescanRows];   // running (b1, b2, j1, j2) per row
    const int R = *count;
    const int groups = (R + kRescanRows - 1) / kRescanRows;
    const long long nchunks = (NB + kRescanThreads - 1) / kRescanThreads;
    const int G = rescan_groups(R, NA, nchunks);
    const long long items = (long long)groups * G;
    const long long cpg = (nchunks + G - 1) / G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float4* B4 = reinterpret_cast<const float4*>(B);
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const int g = (int)(it / G);
        const int cg = (int)(it - (long long)g * G);
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
        if (tid < nr) part_r[(long long)(r0 + tid) * G + cg] = run[tid];
    }
}

// Merge the re-scan partials of queued row r into the row's single partial
// (one warp per queued row, grid-stride: the queue is usually short).
__global__ void k_rescan_merge(const float4* part_r, long long NA, long long NB, const int32_t* rows,
                               const int32_t* count, float4* out_part)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int R = *count;
    const int nchunks = rescan_groups(R, NA, (NB + kRescanThreads - 1) / kRescanThreads);
    for (long long r = (long long)blockIdx.x * nw + warp; r < R; r += (long long)gridDim.x * nw) {
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
}

// E4M3 operands of the FP8 form: each entry times kFp8Scale, rounded to
// nearest E4M3 (saturating; unit descriptors stay below 256 < 448).  One
// thread converts four consecutive entries; invalid rows become zero.
__global__ void k_to_e4m3(const float* d, const uint8_t* v, long long n, uint8_t* out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 32) return;
    const float4 x = reinterpret_cast<const float4*>(d)[t];
    const __nv_fp8x2_storage_t lo =
        __nv_cvt_float2_to_fp8x2(make_float2(x.x * kFp8Scale, x.y * kFp8Scale), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi =
        __nv_cvt_float2_to_fp8x2(make_float2(x.z * kFp8Scale, x.w * kFp8Scale), __NV_SATFINITE, __NV_E4M3);
    reinterpret_cast<uint32_t*>(out)[t] = v[t >> 5] ? ((uint32_t)lo | ((uint32_t)hi << 16)) : 0u;
}

// ------------------------------------------------------------------ host side
bool make_map(CUtensorMap* m, const void* base, long long rows, uint32_t box_rows)
{
    return encode_tiled_2d(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, 128, (uint64_t)rows, 256, 64, box_rows,
                           CU_TENSOR_MAP_SWIZZLE_128B);
}

// E4M3 rows: 128 one-byte entries, one 128-byte box per row
bool make_map8(CUtensorMap* m, const void* base, long long rows, uint32_t box_rows)
{
    return encode_tiled_2d(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, base, 128, (uint64_t)rows, 128, 128, box_rows,
                           CU_TENSOR_MAP_SWIZZLE_128B);
}

// Column splits S: minimise (rounds of units per CTA) x (tiles per unit + ~1
// tile of per-unit A reload and pipeline refill).
int pick_tc_splits(int nrb, long long NB, int ctas)
{
    const long long tiles = (NB + kTileN - 1) / kTileN;
    int best = 1;
    double best_cost = 1e300;
    for (int S = 1; S <= kMaxSplits && S <= tiles; ++S) {
        const long long U = (long long)nrb * S;
        const double rounds = (double)((U + ctas - 1) / ctas);
        const double cost = rounds * (double)((tiles + S - 1) / S + 1);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = S; }
    }
    return best;
}

struct TcLayout {
    int S;
    size_t off_na, off_nb32, off_pm, off_thr, off_cand, off_ncand, off_part1, off_rows, off_cnt, off_part_r,
        total;
};

// S_force > 0: that many column splits (at most kMaxSplits and the tile count)
TcLayout tc_layout(long long NA, long long NB, int sms, int S_force = 0)
{
    TcLayout L;
    const int nrb = (int)((NA + kRowsPerUnit - 1) / kRowsPerUnit);
    const long long tiles = std::max<long long>(1, (NB + kTileN - 1) / kTileN);
    L.S = S_force > 0 ? (int)std::min<long long>(std::min(S_force, kMaxSplits), tiles)
                      : pick_tc_splits(nrb, NB, std::max(1, sms));
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
    L.off_na = take(sizeof(float) * (size_t)NA);
    L.off_nb32 = take(sizeof(float) * (size_t)NB);
    L.off_pm = take(sizeof(float2) * kRanges * (size_t)L.S * NA);
    L.off_thr = take(sizeof(float) * (size_t)NA);
    L.off_cand = take(sizeof(int32_t) * kSubCap * kRanges * (size_t)L.S * NA);
    L.off_ncand = take(sizeof(int32_t) * kRanges * (size_t)L.S * NA);
    L.off_part1 = take(sizeof(float4) * (size_t)NA);
    L.off_rows = take(sizeof(int32_t) * (size_t)NA);
    L.off_cnt = take(64);
    L.off_part_r = take(sizeof(float4) * kRescanGroups * (size_t)NA);
    L.total = o + 256;
    return L;
}

// ---------------------------------------------------------------- batched host side
// Words of the batch's sync block: per launch of up to kBatchPairs pairs, a
// queue counter and one pass-1 counter per row block of each pair.
size_t batch_sync_words_impl(const MatchArgs* args, int P)
{
    size_t w = 0;
    int in_launch = 0;
    for (int i = 0; i < P; ++i) {
        if (args[i].NA == 0 || args[i].NB == 0) continue;
        if (in_launch == 0) w += 1;
        w += (size_t)((args[i].NA + kRowsPerUnit - 1) / kRowsPerUnit);
        if (++in_launch == kBatchPairs) in_launch = 0;
    }
    return w;
}

}  // namespace

size_t match_bf16_batch_sync_words(const MatchArgs* args, int P) { return batch_sync_words_impl(args, P); }

cudaError_t launch_match_bf16_batch(const MatchArgs* args, void* const* ws, const size_t* ws_bytes, int P,
                                    int32_t* sync, int hold, int num_sms, cudaStream_t s)
{
    cudaError_t e;
    const size_t words = batch_sync_words_impl(args, P);
    if (words == 0) return cudaSuccess;
    if ((e = cudaMemsetAsync(sync, 0, words * sizeof(int32_t), s)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_match_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC)) !=
        cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match_tc_batch, kThreadsTC, kSmemTC)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    TcBatch b;   // about 22 KB of kernel parameters; the launch copies it
    int32_t* cursor = sync;
    for (int i0 = 0; i0 < P;) {
        memset(&b, 0, sizeof b);
        b.queue = cursor++;
        b.status = args[i0].status;
        b.hold = hold;
        int n = 0;
        for (; i0 < P && n < kBatchPairs; ++i0) {
            const MatchArgs& a = args[i0];
            if (a.NA == 0 || a.NB == 0) continue;
            const TcLayout L = tc_layout(a.NA, a.NB, num_sms, a.splits);
            if (ws_bytes[i0] < L.total) return cudaErrorInvalidValue;
            uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws[i0]) + 255) & ~uintptr_t(255));
            if (!make_map(&b.tA[n], a.dA16, a.NA, kRowsPerUnit) || !make_map(&b.tB[n], a.dB16, a.NB, kTileN))
                return cudaErrorInvalidValue;
            TcBatchPair& q = b.pr[n];
            q.NA = a.NA;
            q.NB = a.NB;
            q.nrb = (int)((a.NA + kRowsPerUnit - 1) / kRowsPerUnit);
            q.S = L.S;
            const long long tiles = (a.NB + kTileN - 1) / kTileN;
            q.cps = ((tiles + L.S - 1) / L.S) * kTileN;
            q.pm = reinterpret_cast<float2*>(w + L.off_pm);
            q.thr = reinterpret_cast<float*>(w + L.off_thr);
            q.cand = reinterpret_cast<int32_t*>(w + L.off_cand);
            q.ncand = reinterpret_cast<int32_t*>(w + L.off_ncand);
            q.vA = a.vA;
            q.tstride = a.pass1_stride > 0 ? a.pass1_stride : kPass1Stride;
            q.done = cursor;
            cursor += q.nrb;
            b.u1[n + 1] = b.u1[n] + q.nrb * q.S;
            ++n;
        }
        if (n == 0) break;
        b.n = n;
        const int U = 2 * b.u1[n];
        k_match_tc_batch<<<(unsigned)std::min(U, per_sm * num_sms), kThreadsTC, kSmemTC, s>>>(b);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Re-rank, re-scan and finish of a pair whose distance passes ran in
// k_match_tc_batch (thresholds and candidate sub-lists in its workspace); the
// row norms come in a.normA (query rows) and a.normB (+inf for invalid rows).
cudaError_t launch_match_bf16_tail(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s)
{
    if (a.NA == 0) return cudaSuccess;
    const TcLayout L = tc_layout(a.NA, a.NB, num_sms, a.splits);
    if (ws_bytes < L.total || !a.normA || (a.NB > 0 && !a.normB)) return cudaErrorInvalidValue;
    uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    const float* thr = reinterpret_cast<const float*>(w + L.off_thr);
    const int32_t* cand = reinterpret_cast<const int32_t*>(w + L.off_cand);
    const int32_t* ncand = reinterpret_cast<const int32_t*>(w + L.off_ncand);
    float4* part1 = reinterpret_cast<float4*>(w + L.off_part1);
    int32_t* rows = reinterpret_cast<int32_t*>(w + L.off_rows);
    int32_t* cnt = reinterpret_cast<int32_t*>(w + L.off_cnt);
    float4* part_r = reinterpret_cast<float4*>(w + L.off_part_r);
    cudaError_t e;
    if (a.NB == 0) {
        k_match_finish<<<(unsigned)((a.NA + 255) / 256), 256, 0, s>>>(part1, 0, a.NA, a.normA, a.vA, a.ratio2,
                                                                      a.delta_s2, a.match, a.d1, a.d2);
        return cudaGetLastError();
    }
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    k_rerank<<<(unsigned)((a.NA + kRerankWarps - 1) / kRerankWarps), kRerankWarps * 32, 0, s>>>(
        a.dA, a.vA, a.dB, a.normB, cand, ncand, kRanges * L.S, thr, a.NA, part1, rows, cnt);
    if ((e = cudaFuncSetAttribute(k_rescan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRescanSmem)) !=
        cudaSuccess)
        return e;
    k_rescan<<<(unsigned)(4 * num_sms), kRescanThreads, kRescanSmem, s>>>(a.dA, a.dB, a.normB, a.NA, a.NB, rows, cnt,
                                                                           part_r);
    k_rescan_merge<<<(unsigned)std::min<long long>((a.NA + 7) / 8, 2ll * num_sms), 256, 0, s>>>(part_r, a.NA, a.NB,
                                                                                             rows, cnt, part1);
    k_match_finish<<<(unsigned)((a.NA + 255) / 256), 256, 0, s>>>(part1, 1, a.NA, a.normA, a.vA, a.ratio2, a.delta_s2,
                                                                  a.match, a.d1, a.d2);
    return cudaGetLastError();
}

cudaError_t launch_row_norms(const float* d, const uint8_t* v, int64_t n, float* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_row_norms<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(d, v, n, out, INFINITY);
    return cudaGetLastError();
}

namespace {
}  // namespace

bool encode_tiled_2d(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                     uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swizzle)
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
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The E4M3 form keeps its operand copies after the shared layout (whose offsets
// match_bf16_rescans recomputes).
size_t match_bf16_workspace(int64_t NA, int64_t NB, int num_sms, int S, int elem)
{
    const size_t t = tc_layout(NA, NB, num_sms, S).total;
    return elem ? t + (((size_t)NA * 128 + 255) & ~size_t(255)) + (size_t)NB * 128 + 256 : t;
}

int match_bf16_default_splits(int64_t NA, int64_t NB, int num_sms) { return tc_layout(NA, NB, num_sms).S; }

// Number of rows the last BF16 match re-scanned in FP32 (synchronous read).
int64_t match_bf16_rescans(const void* ws, int64_t NA, int64_t NB, int num_sms, int S, cudaStream_t s)
{
    const TcLayout L = tc_layout(NA, NB, num_sms, S);
    const uint8_t* w = reinterpret_cast<const uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    int32_t c = -1;
    if (cudaMemcpyAsync(&c, w + L.off_cnt, sizeof c, cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return c;
}

template <int kElem>
cudaError_t launch_tc_passes(const CUtensorMap& tA, const CUtensorMap& tB, const TcParams& p, const TcParams& p1,
                             int U, int num_sms, cudaStream_t s, const float2* pm, int nsub, long long NA,
                             const uint8_t* vA, float* thr)
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_match_tc<1, kElem>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_match_tc<2, kElem>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTC)) !=
            cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match_tc<1, kElem>, kThreadsTC, kSmemTC)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)std::min(U, per_sm * num_sms));
    k_match_tc<1, kElem><<<grid, kThreadsTC, kSmemTC, s>>>(tA, tB, p1);
    k_row_threshold<<<(unsigned)((NA + 255) / 256), 256, 0, s>>>(pm, nsub, NA, vA, thr, kElem ? kMargin8 : kMargin);
    k_match_tc<2, kElem><<<grid, kThreadsTC, kSmemTC, s>>>(tA, tB, p);
    return cudaGetLastError();
}

cudaError_t launch_match_bf16(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s)
{
    if (a.NA == 0) return cudaSuccess;
    const TcLayout L = tc_layout(a.NA, a.NB, num_sms, a.splits);
    if (ws_bytes < match_bf16_workspace(a.NA, a.NB, num_sms, a.splits, a.elem)) return cudaErrorInvalidValue;
    uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    float* na = reinterpret_cast<float*>(w + L.off_na);
    float* nb32 = reinterpret_cast<float*>(w + L.off_nb32);
    float2* pm = reinterpret_cast<float2*>(w + L.off_pm);
    float* thr = reinterpret_cast<float*>(w + L.off_thr);
    int32_t* cand = reinterpret_cast<int32_t*>(w + L.off_cand);
    int32_t* ncand = reinterpret_cast<int32_t*>(w + L.off_ncand);
    float4* part1 = reinterpret_cast<float4*>(w + L.off_part1);
    int32_t* rows = reinterpret_cast<int32_t*>(w + L.off_rows);
    int32_t* cnt = reinterpret_cast<int32_t*>(w + L.off_cnt);
    float4* part_r = reinterpret_cast<float4*>(w + L.off_part_r);
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
    // the FP32 norms are needed only by the re-rank (B) and the finish (A): with
    // a fork they run on the auxiliary streams beside the tensor-core passes
    const bool forked = a.fork != nullptr && a.NB > 0;
    if (forked) {
        if ((e = cudaEventRecord(a.fork->fork_ev, s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(a.fork->aux[0], a.fork->fork_ev, 0)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(a.fork->aux[1], a.fork->fork_ev, 0)) != cudaSuccess)
            return e;
    }
    k_row_norms<<<(unsigned)((a.NA * 32 + 255) / 256), 256, 0, forked ? a.fork->aux[0] : s>>>(a.dA, a.vA, a.NA, na,
                                                                                             0.f);
    if (forked && (e = cudaEventRecord(a.fork->join_ev[0], a.fork->aux[0])) != cudaSuccess) return e;
    if (a.NB > 0) {
        k_row_norms<<<(unsigned)((a.NB * 32 + 255) / 256), 256, 0, forked ? a.fork->aux[1] : s>>>(a.dB, a.vB, a.NB,
                                                                                                 nb32, INFINITY);
        if (forked && (e = cudaEventRecord(a.fork->join_ev[1], a.fork->aux[1])) != cudaSuccess) return e;
        CUtensorMap tA, tB;
        if (a.elem) {
            // E4M3 copies of both operands, after the shared layout
            uint8_t* a8 = w + L.total;
            uint8_t* b8 = a8 + (((size_t)a.NA * 128 + 255) & ~size_t(255));
            k_to_e4m3<<<(unsigned)((a.NA * 32 + 255) / 256), 256, 0, s>>>(a.dA, a.vA, a.NA, a8);
            k_to_e4m3<<<(unsigned)((a.NB * 32 + 255) / 256), 256, 0, s>>>(a.dB, a.vB, a.NB, b8);
            if (!make_map8(&tA, a8, a.NA, kRowsPerUnit) || !make_map8(&tB, b8, a.NB, kTileN))
                return cudaErrorInvalidValue;
        } else if (!make_map(&tA, a.dA16, a.NA, kRowsPerUnit) || !make_map(&tB, a.dB16, a.NB, kTileN)) {
            return cudaErrorInvalidValue;
        }
        TcParams p;
        p.NA = a.NA;
        p.NB = a.NB;
        p.nrb = (int)((a.NA + kRowsPerUnit - 1) / kRowsPerUnit);
        p.S = L.S;
        const long long tiles = (a.NB + kTileN - 1) / kTileN;
        p.cps = ((tiles + L.S - 1) / L.S) * kTileN;
        p.pm = pm;
        p.thr = thr;
        p.cand = cand;
        p.ncand = ncand;
        p.tstride = 1;
        p.status = a.status;
        const int U = p.nrb * p.S;
        if (a.ev0) cudaEventRecord(a.ev0, s);
        TcParams p1 = p;
        p1.tstride = a.pass1_stride > 0 ? a.pass1_stride : kPass1Stride;
        e = a.elem ? launch_tc_passes<1>(tA, tB, p, p1, U, num_sms, s, pm, kRanges * L.S, a.NA, a.vA, thr)
                   : launch_tc_passes<0>(tA, tB, p, p1, U, num_sms, s, pm, kRanges * L.S, a.NA, a.vA, thr);
        if (e != cudaSuccess) return e;
        if (a.ev1) cudaEventRecord(a.ev1, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (forked && ((e = cudaStreamWaitEvent(s, a.fork->join_ev[1], 0)) != cudaSuccess ||
                       (e = cudaStreamWaitEvent(s, a.fork->join_ev[0], 0)) != cudaSuccess))
            return e;
        k_rerank<<<(unsigned)((a.NA + kRerankWarps - 1) / kRerankWarps), kRerankWarps * 32, 0, s>>>(
            a.dA, a.vA, a.dB, nb32, cand, ncand, kRanges * L.S, thr, a.NA, part1, rows, cnt);
        if ((e = cudaFuncSetAttribute(k_rescan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRescanSmem)) !=
            cudaSuccess)
            return e;
        k_rescan<<<(unsigned)(4 * num_sms), kRescanThreads, kRescanSmem, s>>>(a.dA, a.dB, nb32, a.NA, a.NB, rows,
                                                                               cnt, part_r);
        k_rescan_merge<<<(unsigned)std::min<long long>((a.NA + 7) / 8, 2ll * num_sms), 256, 0, s>>>(
            part_r, a.NA, a.NB, rows, cnt, part1);
        k_match_finish<<<(unsigned)((a.NA + 255) / 256), 256, 0, s>>>(part1, 1, a.NA, na, a.vA, a.ratio2, a.delta_s2,
                                                                      a.match, a.d1, a.d2);
    } else {
        k_match_finish<<<(unsigned)((a.NA + 255) / 256), 256, 0, s>>>(part1, 0, a.NA, na, a.vA, a.ratio2, a.delta_s2,
                                                                      a.match, a.d1, a.d2);
    }
    return cudaGetLastError();
}

}  // namespace lp
