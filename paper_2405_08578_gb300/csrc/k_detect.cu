// Multiscale local-peak detection (Sec. 2.1-2.2, Eq. 1-2) for sm_103a.
//
// Eq. 1 adds alpha*(raster index + 1) to every pixel so that each window has a
// unique maximum and minimum.  With alpha -> 0+ the ramp only breaks ties, which
// is exactly the order of the 32-bit key (intensity << 24) | raster index for
// H*W <= 2^24.  Peaks are therefore max/min of keys, and the result is
// independent of the order of reduction (bit-exact, no atomics).
//
// Fast path (nested scales, Lmax <= 128): one CTA per Lmax x Lmax tile.  The
// tile is streamed from HBM once with 16-byte loads (RGB converted to
// intensity on the fly and written back as the dense intensity image).  When
// the finest side is a multiple of 16, each thread reduces its 16 pixels to
// their extreme keys in registers; otherwise the tile is staged in shared
// memory and reduced per row segment of the finest window.  Finest-window
// extrema follow, then each coarser level combines its children.
// General path: one CTA per window per scale (any L set, any Lmax).
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kDetectThreads = 256;

struct DetectParams {
    const uint8_t* img;
    uint8_t* gray;
    uint32_t* kp;
    int H, W, pitch;
    int TS;                 // tile side (multiple of 16 and of every L)
    int nL;
    int L[LP_MAX_SCALES];
    int nwx[LP_MAX_SCALES];
    int nwy[LP_MAX_SCALES];
    long long off[LP_MAX_SCALES];
    int lvl_off[LP_MAX_SCALES + 1];   // start of each level's window keys in shared memory
};

// floor(s / 1000) for 0 <= s < 2^32 / 704: with C = ceil(2^32 / 1000) =
// 4,294,968 and C * 1000 - 2^32 = 704, s C / 2^32 = s / 1000 + s 704 / (1000 2^32),
// and the added term stays below 1/1000 for such s, so the high word of s C is
// floor(s / 1000).  Intensity sums are at most 255,500.
__device__ __forceinline__ uint32_t div1000(uint32_t s) { return __umulhi(s, 4294968u); }

__device__ __forceinline__ uint8_t rgb2gray(uint32_t r, uint32_t g, uint32_t b)
{
    return (uint8_t)div1000(299u * r + 587u * g + 114u * b + 500u);
}

__device__ __forceinline__ uint8_t byte_of(const uint4& v, int i)
{
    uint32_t w = i < 4 ? v.x : i < 8 ? v.y : i < 12 ? v.z : v.w;
    return (uint8_t)(w >> (8 * (i & 3)));
}

// The division by 1000 on the FP32 pipes.  The dot products start from
// kS0 = 0x4B000000 + 500, so v = 0x4B000000 + s with s = 299 R + 587 G + 114 B
// + 500 < 2^18: as a float, v is 2^23 + s exactly, and f = v - 2^23 = s.  Then
// fma_rz(f, 0.001f, 2^23) = 2^23 + floor(s * 0.001f): in [2^23, 2^24) the float
// spacing is 1 and round-toward-zero keeps the integer part.  0.001f exceeds
// 1/1000 by less than 4.8e-11, so s * 0.001f stays below the next integer for
// every s < 255,501 that is not a multiple of 1000 (the fraction is then at
// most 0.999, the excess at most 1.2e-5), and floor(s * 0.001f) = floor(s /
// 1000) for every such s (checked for all of them).  The result's low byte is
// the intensity.
constexpr uint32_t kS0 = 0x4B000000u + 500u;
__device__ __forceinline__ uint32_t fdiv1000(uint32_t v)
{
    const float f = __int_as_float((int)v) - 8388608.0f;
    return (uint32_t)__float_as_int(__fmaf_rz(f, 0.001f, 8388608.0f));
}

// 16 interleaved RGB pixels (48 bytes, 12 words) -> 16 intensities.
// 299 R + 587 G + 114 B + 500 is formed exactly with two dot products of
// 16-bit weights with byte pairs (dp2a), taken straight from the interleaved
// words: pixel 4g + j's bytes sit at byte offsets 3j .. 3j + 2 of words
// 3g .. 3g + 2, so each pixel needs one or two words and no byte gathering.
// The division by 1000 runs on the FP32 pipes (fdiv1000).
__device__ __forceinline__ uint4 gray16(const uint4& c0, const uint4& c1, const uint4& c2)
{
    const uint32_t w[12] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
    // weight pairs (the low 16 bits multiply the lower byte of the selected pair)
    constexpr uint32_t kRG = 299u | (587u << 16), kB_ = 114u, k_R = 299u << 16, kGB = 587u | (114u << 16);
    uint32_t q[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const uint32_t a = w[3 * g], b = w[3 * g + 1], c = w[3 * g + 2];
        q[4 * g] = fdiv1000(__dp2a_hi(kB_, a, __dp2a_lo(kRG, a, kS0)));
        q[4 * g + 1] = fdiv1000(__dp2a_lo(kGB, b, __dp2a_hi(k_R, a, kS0)));
        q[4 * g + 2] = fdiv1000(__dp2a_lo(kB_, c, __dp2a_hi(kRG, b, kS0)));
        q[4 * g + 3] = fdiv1000(__dp2a_hi(kGB, c, __dp2a_lo(k_R, c, kS0)));
    }
    // four intensities (each < 256) per word: bytes (q0, q1, q2, q3)
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        o[k] = __byte_perm(__byte_perm(q[4 * k], q[4 * k + 1], 0x0040u), __byte_perm(q[4 * k + 2], q[4 * k + 3], 0x0040u),
                           0x5410u);
    return make_uint4(o[0], o[1], o[2], o[3]);
}

__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Extreme keys of 16 consecutive pixels of one row (raster index of the first:
// base).  Within the group, (intensity << 8) | position orders pixels exactly
// as the key does; one byte permutation builds two such 16-bit values (the
// intensity bytes next to position bytes), so the maximum and minimum run as
// packed 16-bit pairs.
__device__ __forceinline__ void group_keys(const uint4& v, uint32_t base, uint32_t& kmax, uint32_t& kmin)
{
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t mx = 0u, mn = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // positions 4k .. 4k + 3 in bytes 0 .. 3
        const uint32_t pos = (4u * k) | ((4u * k + 1u) << 8) | ((4u * k + 2u) << 16) | ((4u * k + 3u) << 24);
        const uint32_t lo = __byte_perm(w[k], pos, 0x1504u);   // (b0 << 8 | 4k, b1 << 8 | 4k + 1)
        const uint32_t hi = __byte_perm(w[k], pos, 0x3726u);   // (b2 << 8 | 4k + 2, b3 << 8 | 4k + 3)
        mx = max_u16x2(mx, max_u16x2(lo, hi));
        mn = min_u16x2(mn, min_u16x2(lo, hi));
    }
    const uint32_t M = max(mx & 0xFFFFu, mx >> 16), m = min(mn & 0xFFFFu, mn >> 16);
    kmax = ((M >> 8) << 24) | (base + (M & 15u));
    kmin = ((m >> 8) << 24) | (base + (m & 15u));
}

// One TS x TS tile (tile column bx, tile row by) of one image.
template <int CH>
__device__ __forceinline__ void detect_tile(const DetectParams& p, int bx, int by)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int TS = p.TS;
    const int L0 = p.L[0];
    const bool fused = (L0 & 15) == 0;       // 16-pixel groups reduced in registers
    const int spr = fused ? TS / 16 : TS / L0;   // segments per tile row
    const int gpw = fused ? L0 / 16 : 1;         // segments per finest-window row
    const int nseg = TS * spr;
    uint8_t* tile = sm;
    uint32_t* smx = reinterpret_cast<uint32_t*>(sm + (fused ? 0 : TS * TS));
    uint32_t* smn = smx + nseg;
    uint32_t* wmx = smn + nseg;
    uint32_t* wmn = wmx + p.lvl_off[p.nL];

    const int tx0 = bx * TS, ty0 = by * TS;
    const int rows = min(TS, p.H - ty0), cols = min(TS, p.W - tx0);
    const int Hf = (p.H / L0) * L0 - ty0, Wf = (p.W / L0) * L0 - tx0;   // full finest windows

    // ---- stream the tile once: 16 pixels per 16-byte (gray) or 48-byte (RGB)
    // load.  Each pass issues the loads of a thread's next kGroups 16-pixel
    // groups before it uses the first, so two DRAM round trips overlap.
    constexpr int kGroups = 2;
    const int gpr = TS / 16, ng = TS * gpr;
    for (int g0 = 0; g0 < ng; g0 += kGroups * kDetectThreads) {
        uint4 raw[kGroups][CH];
#pragma unroll
        for (int u = 0; u < kGroups; ++u) {
            const int g = g0 + threadIdx.x + u * kDetectThreads;
            const int r = g / gpr, c = (g - r * gpr) * 16;
#pragma unroll
            for (int q = 0; q < CH; ++q) raw[u][q] = make_uint4(0, 0, 0, 0);
            if (g < ng && r < rows && c < cols) {
                const uint8_t* row = p.img + (size_t)(ty0 + r) * p.pitch;
                const int x = tx0 + c;
                if (CH == 1) {
                    raw[u][0] = __ldg(reinterpret_cast<const uint4*>(row + x));
                } else {
                    // chunk q holds bytes [3x + 16q, 3x + 16q + 16); it lies inside the
                    // pitch whenever its first byte is a pixel byte of this row
                    const uint4* src = reinterpret_cast<const uint4*>(row + 3 * (size_t)x);
                    raw[u][0] = __ldg(src);
                    if (3 * x + 16 < 3 * p.W) raw[u][CH > 1 ? 1 : 0] = __ldg(src + 1);
                    if (3 * x + 32 < 3 * p.W) raw[u][CH > 2 ? 2 : 0] = __ldg(src + 2);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kGroups; ++u) {
            const int g = g0 + threadIdx.x + u * kDetectThreads;
            if (g >= ng) break;
            const int r = g / gpr, c = (g - r * gpr) * 16;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (r < rows && c < cols) {
                if (CH == 1) {
                    v = raw[u][0];
                } else {
                    const int x = tx0 + c;
                    v = gray16(raw[u][0], raw[u][CH > 1 ? 1 : 0], raw[u][CH > 2 ? 2 : 0]);
                    uint8_t* gout = p.gray + (size_t)(ty0 + r) * p.W + x;
                    if ((p.W & 15) == 0) {
                        *reinterpret_cast<uint4*>(gout) = v;
                    } else {
                        const int n = min(16, p.W - x);
                        for (int i = 0; i < n; ++i) gout[i] = byte_of(v, i);
                    }
                }
            }
            if (fused) {
                uint32_t kmax = 0u, kmin = 0xFFFFFFFFu;
                if (r < Hf && c < Wf)
                    group_keys(v, (uint32_t)(ty0 + r) * (uint32_t)p.W + (uint32_t)(tx0 + c), kmax, kmin);
                smx[g] = kmax;
                smn[g] = kmin;
            } else {
                *reinterpret_cast<uint4*>(tile + r * TS + c) = v;
            }
        }
    }
    __syncthreads();

    // ---- finest scale: extrema of every L0-pixel row segment of a full window
    for (int s = threadIdx.x; s < (fused ? 0 : nseg); s += kDetectThreads) {
        const int r = s / spr, c0 = (s - r * spr) * L0;
        uint32_t kmax = 0u, kmin = 0xFFFFFFFFu;
        if (r < Hf && c0 < Wf) {
            const uint32_t base = (uint32_t)(ty0 + r) * (uint32_t)p.W + (uint32_t)(tx0 + c0);
            const uint8_t* t = tile + r * TS + c0;
            for (int i = 0; i < L0; ++i) {
                const uint32_t k = ((uint32_t)t[i] << 24) | (base + i);
                kmax = max(kmax, k);
                kmin = min(kmin, k);
            }
        }
        smx[s] = kmax;
        smn[s] = kmin;
    }
    __syncthreads();

    // ---- level 0 windows from their L0 segments
    {
        const int n0 = TS / L0;
        for (int w = threadIdx.x; w < n0 * n0; w += kDetectThreads) {
            const int wr = w / n0, wc = w - wr * n0;
            uint32_t kmax = 0u, kmin = 0xFFFFFFFFu;
            for (int i = 0; i < L0; ++i)
                for (int j = 0; j < gpw; ++j) {
                    const int s = (wr * L0 + i) * spr + wc * gpw + j;
                    kmax = max(kmax, smx[s]);
                    kmin = min(kmin, smn[s]);
                }
            wmx[w] = kmax;
            wmn[w] = kmin;
            const int gy = ty0 / L0 + wr, gx = tx0 / L0 + wc;
            if (gy < p.nwy[0] && gx < p.nwx[0]) {
                uint2 o = make_uint2(kmax & 0xFFFFFFu, kmin & 0xFFFFFFu);
                *reinterpret_cast<uint2*>(p.kp + p.off[0] + 2ll * ((long long)gy * p.nwx[0] + gx)) = o;
            }
        }
    }
    // ---- coarser levels combine their (L_l / L_{l-1})^2 children
    for (int l = 1; l < p.nL; ++l) {
        __syncthreads();
        const int nl = TS / p.L[l], np = TS / p.L[l - 1], q = p.L[l] / p.L[l - 1];
        const uint32_t* cmx = wmx + p.lvl_off[l - 1];
        const uint32_t* cmn = wmn + p.lvl_off[l - 1];
        for (int w = threadIdx.x; w < nl * nl; w += kDetectThreads) {
            const int wr = w / nl, wc = w - wr * nl;
            uint32_t kmax = 0u, kmin = 0xFFFFFFFFu;
            for (int i = 0; i < q; ++i)
                for (int j = 0; j < q; ++j) {
                    const int cidx = (wr * q + i) * np + wc * q + j;
                    kmax = max(kmax, cmx[cidx]);
                    kmin = min(kmin, cmn[cidx]);
                }
            wmx[p.lvl_off[l] + w] = kmax;
            wmn[p.lvl_off[l] + w] = kmin;
            const int gy = ty0 / p.L[l] + wr, gx = tx0 / p.L[l] + wc;
            if (gy < p.nwy[l] && gx < p.nwx[l]) {
                uint2 o = make_uint2(kmax & 0xFFFFFFu, kmin & 0xFFFFFFu);
                *reinterpret_cast<uint2*>(p.kp + p.off[l] + 2ll * ((long long)gy * p.nwx[l] + gx)) = o;
            }
        }
    }
}

template <int CH>
__global__ void __launch_bounds__(kDetectThreads) k_detect_nested(const __grid_constant__ DetectParams p)
{
    detect_tile<CH>(p, blockIdx.x, blockIdx.y);
}

// Several images (same scales and channel count) in one launch: a flat CTA
// index runs over every image's tiles, so a batch fills the GPU that one
// image cannot.
constexpr int kDetectBatch = 12;   // keeps the parameter block under 4 KB
struct DetectBatch {
    DetectParams im[kDetectBatch];   // the shared fields (TS, nL, L, lvl_off) are equal in all
    int tiles_x[kDetectBatch];
    int tile0[kDetectBatch + 1];     // prefix sums of the images' tile counts
    int n;
};

template <int CH>
__global__ void __launch_bounds__(kDetectThreads) k_detect_nested_batch(const __grid_constant__ DetectBatch b)
{
    const int t = blockIdx.x;
    int i = 0;
    while (i + 1 < b.n && t >= b.tile0[i + 1]) ++i;
    const int lt = t - b.tile0[i];
    const int by = lt / b.tiles_x[i], bx = lt - by * b.tiles_x[i];
    detect_tile<CH>(b.im[i], bx, by);
}

// ------------------------------------------------------------------ TMA-fed fast path
// Nested scales drawn from {16, 32, 64, 128} with 16 the finest, 8-bit gray
// or RGB input.  Persistent CTAs (two per SM, so that one CTA's compute
// warps run while the other's wait on their ring) walk a flat list of
// 128 x 128 tiles of up to kDetectBatch images.
//   warp 16     streams whole tiles into a 2-stage shared-memory ring with
//               cp.async.bulk.tensor (one 2-D box of 128 rows x 128 pixels,
//               out-of-image bytes zero-filled).
//   warps 0-15  all work on every tile: warp w holds pixel rows [8 w, 8 w + 8),
//               lane (p, c) = (lane >> 3, lane & 7) the 2 x 16 strip at rows
//               8 w + 2 p, columns 16 c.  A lane converts RGB to intensity,
//               writes the intensity and reduces its keys in registers; two
//               shuffles (xor 8, xor 16) give the 8 x 16 half windows, which
//               go to shared memory (one of two buffers, alternating tiles).
//   warp 17     combines the half windows into the 16-pixel windows and, with
//               shuffles, the 32-, 64- and 128-pixel windows, and writes the
//               keys of the requested scales.
// A window that is not full is dropped at output, so out-of-image pixels
// never reach a kept key.  Every wait is bounded (2 s): on expiry the CTA
// records LP_ERR_TIMEOUT, lets its copies in flight land and returns.
#ifndef LP_DETECT_STAGES
#define LP_DETECT_STAGES 2
#endif
#ifndef LP_DETECT_CTAS_PER_SM
#define LP_DETECT_CTAS_PER_SM 2
#endif
constexpr int kTmaTile = 128;
constexpr int kTmaStages = LP_DETECT_STAGES;             // ring stages per CTA
constexpr int kTmaMinBlocks = LP_DETECT_CTAS_PER_SM;     // resident CTAs per SM the registers allow
constexpr int kTmaCompute = 16;                          // compute warps
constexpr int kTmaThreads = 32 * (kTmaCompute + 2);      // + producer warp + reducer warp

struct TmaImage {
    uint8_t* gray;          // intensity output (RGB input) or nullptr
    uint32_t* kp;
    int H, W;
    int tiles_x;
    int nwx[4], nwy[4];     // windows per row / column at L = 16, 32, 64, 128 (0: scale not requested)
    long long off[4];       // first keypoint of each of those scales
};

struct DetectTmaBatch {
    CUtensorMap map[kDetectBatch];   // 2-D, 4-byte elements: {pitch / 4, H}, box {32 CH, 128}
    TmaImage im[kDetectBatch];
    int tile0[kDetectBatch + 1];     // prefix sums of the images' tile counts
    int n;
    int32_t* status;
};

__device__ __forceinline__ uint32_t d_smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One try of a phase wait.  The thread may be suspended for up to
// kSuspendNs (it resumes as soon as the phase completes), so a waiting warp
// takes few issue slots from the working ones.
#ifndef LP_DETECT_SUSPEND_NS
#define LP_DETECT_SUSPEND_NS 10000
#endif
constexpr uint32_t kSuspendNs = LP_DETECT_SUSPEND_NS;
__device__ __forceinline__ bool d_mbar_try(uint32_t bar, uint32_t parity)
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

__device__ __forceinline__ void d_mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint64_t d_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: true when the phase completed, false on abort or after 2 s.
__device__ __forceinline__ bool d_mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int32_t* status)
{
    if (d_mbar_try(bar, parity)) return true;
    const uint64_t t0 = d_globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (d_mbar_try(bar, parity)) return true;
        if ((it & 15u) == 0) {
            if (*abort_flag) return false;
            if (d_globaltimer() - t0 > 2000000000ull) {
                *abort_flag = 1;
                set_status(status, DEV_TIMEOUT);
                return false;
            }
        }
    }
}

// Global tile t -> (image, tile column, tile row).
__device__ __forceinline__ void tma_tile(const DetectTmaBatch& b, int t, int& i, int& tx, int& ty)
{
    i = 0;
    while (i + 1 < b.n && t >= b.tile0[i + 1]) ++i;
    const int lt = t - b.tile0[i];
    ty = lt / b.im[i].tiles_x;
    tx = lt - ty * b.im[i].tiles_x;
}

__device__ __forceinline__ void key_max_min(uint32_t& kmax, uint32_t& kmin, uint32_t omax, uint32_t omin)
{
    kmax = max(kmax, omax);
    kmin = min(kmin, omin);
}

__device__ __forceinline__ void shfl_key(uint32_t& kmax, uint32_t& kmin, int lanemask)
{
    key_max_min(kmax, kmin, __shfl_xor_sync(0xFFFFFFFFu, kmax, lanemask), __shfl_xor_sync(0xFFFFFFFFu, kmin, lanemask));
}

// Window (gx, gy) of scale slot l: written when the window is full.
__device__ __forceinline__ void put_key(const TmaImage& im, int l, int gx, int gy, uint32_t kmax, uint32_t kmin)
{
    if (gx < im.nwx[l] && gy < im.nwy[l])
        *reinterpret_cast<uint2*>(im.kp + im.off[l] + 2ll * ((long long)gy * im.nwx[l] + gx)) =
            make_uint2(kmax & 0xFFFFFFu, kmin & 0xFFFFFFu);
}

template <int CH>
__global__ void __launch_bounds__(kTmaThreads, kTmaMinBlocks) k_detect_tma(const __grid_constant__ DetectTmaBatch b)
{
    constexpr uint32_t kStageBytes = kTmaTile * kTmaTile * CH;   // 48 KB (RGB) or 16 KB (gray)
    extern __shared__ uint8_t dsm_raw[];
    // 1024-byte aligned, as an offset from the shared array so that every
    // access below stays a shared-memory access (an integer round trip would
    // leave generic pointers)
    uint8_t* dsm = dsm_raw + ((1024u - (d_smem_u32(dsm_raw) & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(dsm + kTmaStages * kStageBytes);
    uint64_t* empty = full + kTmaStages;
    uint64_t* xfull = empty + kTmaStages;    // [2 buffers]: every compute warp wrote its half windows
    uint64_t* xempty = xfull + 2;            // [2 buffers]: the reducer has read them
    uint32_t* hw = reinterpret_cast<uint32_t*>(xempty + 2);   // [2 buffers][16 warps][8 columns][max, min]
    int* hmeta = reinterpret_cast<int*>(hw + 2 * kTmaCompute * 8 * 2);   // [2 buffers][image, tile x, tile y]
    int* tinfo = hmeta + 2 * 4;                                          // [stage][image, tile x, tile y]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tinfo + kTmaStages * 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int T = b.tile0[b.n];
    const int G = (int)gridDim.x;
    const int ntile = (int)blockIdx.x < T ? (T - (int)blockIdx.x + G - 1) / G : 0;   // this CTA's tiles

    if (threadIdx.x == 0) {
        for (int s = 0; s < kTmaStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(d_smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(d_smem_u32(&empty[s])), "r"(kTmaCompute)
                         : "memory");
        }
        for (int q = 0; q < 2; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(d_smem_u32(&xfull[q])), "r"(kTmaCompute)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(d_smem_u32(&xempty[q])) : "memory");
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kTmaCompute) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            for (int i = 0; i < b.n; ++i)
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&b.map[i])) : "memory");
            int armed[kTmaStages];
            for (int s = 0; s < kTmaStages; ++s) armed[s] = -1;
            bool ok = true;
            for (int n = 0; n < ntile && ok; ++n) {
                const int s = n % kTmaStages;
                const uint32_t k = (uint32_t)(n / kTmaStages);
                ok = d_mbar_wait(d_smem_u32(&empty[s]), (k & 1) ^ 1, abort_flag, b.status);
                if (!ok) break;
                int i, tx, ty;
                tma_tile(b, (int)blockIdx.x + n * G, i, tx, ty);
                // the tile's place, for the compute warps (published by the arrival below)
                tinfo[4 * s] = i;
                tinfo[4 * s + 1] = tx;
                tinfo[4 * s + 2] = ty;
                const uint32_t bar = d_smem_u32(&full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kStageBytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3}], [%4];" ::"r"(d_smem_u32(dsm + s * kStageBytes)),
                    "l"(reinterpret_cast<uint64_t>(&b.map[i])), "r"(tx * 32 * CH), "r"(ty * kTmaTile), "r"(bar)
                    : "memory");
                armed[s] = (int)k;
            }
            if (!ok) {
                // let the copies in flight land (bounded) before the CTA exits
                for (int s = 0; s < kTmaStages; ++s) {
                    if (armed[s] < 0) continue;
                    const uint64_t t0 = d_globaltimer();
                    while (!d_mbar_try(d_smem_u32(&full[s]), (uint32_t)armed[s] & 1u) &&
                           d_globaltimer() - t0 < 200000000ull) {
                    }
                }
            }
        }
        return;
    }

    if (warp == kTmaCompute + 1) {
        // ------------------------------------------------------------ reducer
        // lane (q, c) = (lane >> 3, lane & 7): the 16-pixel windows at window
        // rows q (set A) and q + 4 (set B), window column c
        const int q = lane >> 3, c = lane & 7;
        for (int n = 0; n < ntile; ++n) {
            const int xb = n & 1;
            const uint32_t use = (uint32_t)(n >> 1);
            if (!__all_sync(0xFFFFFFFFu, d_mbar_wait(d_smem_u32(&xfull[xb]), use & 1, abort_flag, b.status))) break;
            const uint32_t* hx = hw + xb * (kTmaCompute * 16);
            // window row r = 16-pixel rows of half-window warps 2 r and 2 r + 1
            uint32_t amax = max(hx[(2 * q) * 16 + 2 * c], hx[(2 * q + 1) * 16 + 2 * c]);
            uint32_t amin = min(hx[(2 * q) * 16 + 2 * c + 1], hx[(2 * q + 1) * 16 + 2 * c + 1]);
            uint32_t bmax = max(hx[(2 * q + 8) * 16 + 2 * c], hx[(2 * q + 9) * 16 + 2 * c]);
            uint32_t bmin = min(hx[(2 * q + 8) * 16 + 2 * c + 1], hx[(2 * q + 9) * 16 + 2 * c + 1]);
            const int i = hmeta[4 * xb], tx = hmeta[4 * xb + 1], ty = hmeta[4 * xb + 2];
            __syncwarp();
            if (lane == 0) d_mbar_arrive(d_smem_u32(&xempty[xb]));
            const TmaImage& im = b.im[i];
            if (im.nwx[0]) {
                put_key(im, 0, tx * 8 + c, ty * 8 + q, amax, amin);
                put_key(im, 0, tx * 8 + c, ty * 8 + q + 4, bmax, bmin);
            }
            // 32-pixel windows: column pairs (xor 1), row pairs (xor 8)
            shfl_key(amax, amin, 1);
            shfl_key(amax, amin, 8);
            shfl_key(bmax, bmin, 1);
            shfl_key(bmax, bmin, 8);
            if (im.nwx[1] && (c & 1) == 0 && (q & 1) == 0) {
                put_key(im, 1, tx * 4 + (c >> 1), ty * 4 + (q >> 1), amax, amin);
                put_key(im, 1, tx * 4 + (c >> 1), ty * 4 + 2 + (q >> 1), bmax, bmin);
            }
            // 64-pixel windows: column quads (xor 2), row quads (xor 16); A is
            // the top half of the tile, B the bottom half
            shfl_key(amax, amin, 2);
            shfl_key(amax, amin, 16);
            shfl_key(bmax, bmin, 2);
            shfl_key(bmax, bmin, 16);
            if (im.nwx[2] && (c & 3) == 0 && q == 0) {
                put_key(im, 2, tx * 2 + (c >> 2), ty * 2, amax, amin);
                put_key(im, 2, tx * 2 + (c >> 2), ty * 2 + 1, bmax, bmin);
            }
            // 128-pixel window: both halves, both column halves (xor 4)
            key_max_min(amax, amin, bmax, bmin);
            shfl_key(amax, amin, 4);
            if (im.nwx[3] && lane == 0) put_key(im, 3, tx, ty, amax, amin);
        }
        return;
    }

    // ---------------------------------------------------------------- compute warps
    const int p = lane >> 3, c = lane & 7;
    const int row0 = 8 * warp + 2 * p;               // first tile row of this lane's strip
    for (int n = 0; n < ntile; ++n) {
        const int s = n % kTmaStages;
        const uint32_t k = (uint32_t)(n / kTmaStages);
        // every lane waits; the warp acts on one decision (they differ only
        // after a timeout)
        if (!__all_sync(0xFFFFFFFFu, d_mbar_wait(d_smem_u32(&full[s]), k & 1, abort_flag, b.status))) break;
        const int i = tinfo[4 * s], tx = tinfo[4 * s + 1], ty = tinfo[4 * s + 2];
        const TmaImage& im = b.im[i];
        const int x0 = tx * kTmaTile + 16 * c;           // first column of the strip
        const uint8_t* src = dsm + s * kStageBytes + row0 * (kTmaTile * CH) + 16 * CH * c;
        const int y0 = ty * kTmaTile + row0;
        // rows of the strip whose intensity is written (inside the image)
        const int nrow = x0 < im.W ? max(0, min(2, im.H - y0)) : 0;
        const uint32_t base = (uint32_t)y0 * (uint32_t)im.W + (uint32_t)x0;
        uint4 v[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (CH == 1) {
                v[r] = *reinterpret_cast<const uint4*>(src + r * kTmaTile);
            } else {
                const uint4* qs = reinterpret_cast<const uint4*>(src + r * kTmaTile * 3);
                v[r] = gray16(qs[0], qs[1], qs[2]);
            }
        }
        // the stage is no longer read: hand it back to the producer
        __syncwarp();
        if (lane == 0) d_mbar_arrive(d_smem_u32(&empty[s]));
        if (CH == 3) {
            uint8_t* gout = im.gray + (size_t)y0 * im.W + x0;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (r < nrow) {
                    if ((im.W & 15) == 0) {
                        *reinterpret_cast<uint4*>(gout + (size_t)r * im.W) = v[r];
                    } else {
                        const int nb = min(16, im.W - x0);
                        for (int j = 0; j < nb; ++j) gout[(size_t)r * im.W + j] = byte_of(v[r], j);
                    }
                }
            }
        }
        uint32_t kmax, kmin, omax, omin;
        group_keys(v[0], base, kmax, kmin);
        group_keys(v[1], base + (uint32_t)im.W, omax, omin);
        key_max_min(kmax, kmin, omax, omin);
        // 8 x 16 half windows: the four row pairs of a column (xor 8, xor 16)
        shfl_key(kmax, kmin, 8);
        shfl_key(kmax, kmin, 16);
        const int xb = n & 1;
        const uint32_t use = (uint32_t)(n >> 1);
        if (!__all_sync(0xFFFFFFFFu, d_mbar_wait(d_smem_u32(&xempty[xb]), (use & 1) ^ 1, abort_flag, b.status)))
            break;
        if (p == 0) {
            uint32_t* h = hw + xb * (kTmaCompute * 16) + warp * 16 + 2 * c;
            h[0] = kmax;
            h[1] = kmin;
        }
        if (warp == 0 && lane == 0) {   // the tile's place, for the reducer
            hmeta[4 * xb] = i;
            hmeta[4 * xb + 1] = tx;
            hmeta[4 * xb + 2] = ty;
        }
        __syncwarp();
        if (lane == 0) d_mbar_arrive(d_smem_u32(&xfull[xb]));
    }
}

// General path: one CTA per full window of one scale.
template <int CH>
__global__ void __launch_bounds__(kDetectThreads) k_detect_window(const uint8_t* img, int H, int W, int pitch,
                                                                   int L, int nwx, long long off, uint32_t* kp)
{
    const int w = blockIdx.x;
    const int wy = w / nwx, wx = w - wy * nwx;
    uint32_t kmax = 0u, kmin = 0xFFFFFFFFu;
    const int n = L * L;
    for (int i = threadIdx.x; i < n; i += kDetectThreads) {
        const int r = i / L, c = i - r * L;
        const int y = wy * L + r, x = wx * L + c;
        const uint8_t* px = img + (size_t)y * pitch + (size_t)CH * x;
        const uint32_t g = CH == 1 ? px[0] : rgb2gray(px[0], px[1], px[2]);
        const uint32_t k = (g << 24) | ((uint32_t)y * (uint32_t)W + (uint32_t)x);
        kmax = max(kmax, k);
        kmin = min(kmin, k);
    }
    for (int o = 16; o; o >>= 1) {
        kmax = max(kmax, __shfl_xor_sync(0xFFFFFFFFu, kmax, o));
        kmin = min(kmin, __shfl_xor_sync(0xFFFFFFFFu, kmin, o));
    }
    __shared__ uint32_t rmx[kDetectThreads / 32], rmn[kDetectThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        rmx[threadIdx.x >> 5] = kmax;
        rmn[threadIdx.x >> 5] = kmin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kDetectThreads / 32; ++i) {
            kmax = max(kmax, rmx[i]);
            kmin = min(kmin, rmn[i]);
        }
        kp[off + 2ll * w] = kmax & 0xFFFFFFu;
        kp[off + 2ll * w + 1] = kmin & 0xFFFFFFu;
    }
    (void)H;
}

// Eq. 1 with a finite alpha: M_n = g + alpha * (raster index + 1) in FP64, one
// rounding for the product and one for the sum (no contraction); the maximum
// and minimum of each window, equal values going to the earlier raster
// position (the first in the window's row-major scan).
template <int CH>
__global__ void __launch_bounds__(kDetectThreads) k_detect_window_ramp(const uint8_t* img, int W, int pitch, int L,
                                                                        int nwx, long long off, double alpha,
                                                                        uint32_t* kp)
{
    const int w = blockIdx.x;
    const int wy = w / nwx, wx = w - wy * nwx;
    double vmax = -INFINITY, vmin = INFINITY;
    uint32_t imax = 0xFFFFFFFFu, imin = 0xFFFFFFFFu;
    const int n = L * L;
    for (int i = threadIdx.x; i < n; i += kDetectThreads) {
        const int r = i / L, c = i - r * L;
        const int y = wy * L + r, x = wx * L + c;
        const uint8_t* px = img + (size_t)y * pitch + (size_t)CH * x;
        const uint32_t g = CH == 1 ? px[0] : rgb2gray(px[0], px[1], px[2]);
        const uint32_t id = (uint32_t)y * (uint32_t)W + (uint32_t)x;
        const double v = __dadd_rn((double)g, __dmul_rn(alpha, (double)id + 1.0));
        if (v > vmax || (v == vmax && id < imax)) { vmax = v; imax = id; }
        if (v < vmin || (v == vmin && id < imin)) { vmin = v; imin = id; }
    }
    for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_xor_sync(0xFFFFFFFFu, vmax, o);
        const uint32_t oi = __shfl_xor_sync(0xFFFFFFFFu, imax, o);
        if (ov > vmax || (ov == vmax && oi < imax)) { vmax = ov; imax = oi; }
        const double nv = __shfl_xor_sync(0xFFFFFFFFu, vmin, o);
        const uint32_t ni = __shfl_xor_sync(0xFFFFFFFFu, imin, o);
        if (nv < vmin || (nv == vmin && ni < imin)) { vmin = nv; imin = ni; }
    }
    __shared__ double rv[2][kDetectThreads / 32];
    __shared__ uint32_t ri[2][kDetectThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        rv[0][threadIdx.x >> 5] = vmax; ri[0][threadIdx.x >> 5] = imax;
        rv[1][threadIdx.x >> 5] = vmin; ri[1][threadIdx.x >> 5] = imin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < kDetectThreads / 32; ++q) {
            if (rv[0][q] > vmax || (rv[0][q] == vmax && ri[0][q] < imax)) { vmax = rv[0][q]; imax = ri[0][q]; }
            if (rv[1][q] < vmin || (rv[1][q] == vmin && ri[1][q] < imin)) { vmin = rv[1][q]; imin = ri[1][q]; }
        }
        kp[off + 2ll * w] = imax;
        kp[off + 2ll * w + 1] = imin;
    }
}

__global__ void k_rgb_to_gray(const uint8_t* img, int H, int W, int pitch, uint8_t* gray)
{
    const long long n = (long long)H * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (long long)y * W);
        const uint8_t* px = img + (size_t)y * pitch + 3 * (size_t)x;
        gray[i] = rgb2gray(px[0], px[1], px[2]);
    }
}

__global__ void k_diag_gray(const uint8_t* rgb, long long n, uint8_t* gray)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        gray[i] = rgb2gray(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2]);
}

}  // namespace

namespace {

// The fast path's tile side: nested scales with Lmax <= 128; TS holds whole
// 16-byte loads and at most 4096 finest-scale segments.  false: general path.
bool nested_tile(const ScaleTable& st, int* TS_out)
{
    bool nested = st.L[st.nL - 1] <= 128;
    for (int l = 1; l < st.nL && nested; ++l) nested = st.L[l] % st.L[l - 1] == 0;
    int TS = st.L[st.nL - 1];
    if (nested && TS % 16 != 0) {
        nested = (16 % TS == 0);
        TS = 16;
    }
    if (nested && (long long)TS * TS / st.L[0] > 4096) nested = false;
    *TS_out = TS;
    return nested;
}

// Parameters of one image on the fast path; returns the dynamic shared memory.
size_t fill_nested(DetectParams& p, const uint8_t* img, int H, int W, int pitch, const ScaleTable& st, int TS,
                   uint32_t* kp, uint8_t* gray)
{
    p.img = img; p.gray = gray; p.kp = kp; p.H = H; p.W = W; p.pitch = pitch; p.TS = TS; p.nL = st.nL;
    int acc = 0;
    for (int l = 0; l < st.nL; ++l) {
        p.L[l] = st.L[l]; p.nwx[l] = st.nwx[l]; p.nwy[l] = st.nwy[l]; p.off[l] = st.off[l];
        p.lvl_off[l] = acc;
        acc += (TS / st.L[l]) * (TS / st.L[l]);
    }
    for (int l = st.nL; l <= LP_MAX_SCALES; ++l) p.lvl_off[l] = acc;
    if (st.L[0] % 16 == 0) return 8u * (size_t)(TS * TS / 16) + 8u * acc;   // no staged tile
    const int nseg = TS * TS / st.L[0];
    return (size_t)TS * TS + 8u * nseg + 8u * acc;
}

// The TMA path takes scale sets drawn from {16, 32, 64, 128} with 16 the finest.
bool tma_scales(const ScaleTable& st)
{
    if (st.nL < 1 || st.L[0] != 16) return false;
    for (int l = 0; l < st.nL; ++l)
        if (st.L[l] != 16 && st.L[l] != 32 && st.L[l] != 64 && st.L[l] != 128) return false;
    return true;
}

// the ring, up to 1 KB of alignment slack, then barriers (96 B), the half
// windows (2 KB), the tile slots (96 B) and the abort flag: 4 KB reserved
size_t tma_smem(int ch) { return (size_t)kTmaStages * kTmaTile * kTmaTile * ch + 1024 + 4096; }

// Up to N images in launches of kDetectBatch on the TMA path.
cudaError_t launch_detect_tma(const uint8_t* const* imgs, const int* Hs, const int* Ws, const int* pitches, int N,
                              int ch, const ScaleTable* sts, uint32_t* const* kps, uint8_t* const* grays,
                              int32_t* status, int num_sms, cudaStream_t s)
{
    const size_t smem = tma_smem(ch);
    cudaError_t e;
    auto kern = ch == 1 ? k_detect_tma<1> : k_detect_tma<3>;
    // the shared-memory opt-in and the resident CTAs per SM, once per device
    // and channel count (host calls that would otherwise precede every launch)
    static int per_sm_cache[2][64];
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int& per_sm = per_sm_cache[ch == 3][dev & 63];
    if (per_sm == 0 || dev >= 64) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int n = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kTmaThreads, smem)) != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        per_sm = n;
    }
    for (int i0 = 0; i0 < N; i0 += kDetectBatch) {
        DetectTmaBatch b;
        memset(&b, 0, sizeof b);
        b.n = N - i0 < kDetectBatch ? N - i0 : kDetectBatch;
        b.status = status;
        b.tile0[0] = 0;
        for (int k = 0; k < b.n; ++k) {
            const int i = i0 + k;
            const ScaleTable& st = sts[i];
            // the image as rows of pitch / 4 four-byte elements; a box is one tile
            if (!encode_tiled_2d(&b.map[k], CU_TENSOR_MAP_DATA_TYPE_UINT32, imgs[i], (uint64_t)pitches[i] / 4,
                                 (uint64_t)Hs[i], (uint64_t)pitches[i], 32u * ch, kTmaTile, CU_TENSOR_MAP_SWIZZLE_NONE))
                return cudaErrorInvalidValue;
            TmaImage& im = b.im[k];
            im.gray = grays ? grays[i] : nullptr;
            im.kp = kps[i];
            im.H = Hs[i];
            im.W = Ws[i];
            im.tiles_x = (Ws[i] + kTmaTile - 1) / kTmaTile;
            for (int l = 0; l < st.nL; ++l) {
                const int slot = st.L[l] == 16 ? 0 : st.L[l] == 32 ? 1 : st.L[l] == 64 ? 2 : 3;
                im.nwx[slot] = st.nwx[l];
                im.nwy[slot] = st.nwx[l] > 0 ? st.nwy[l] : 0;
                im.off[slot] = st.off[l];
            }
            b.tile0[k + 1] = b.tile0[k] + im.tiles_x * ((Hs[i] + kTmaTile - 1) / kTmaTile);
        }
        const int T = b.tile0[b.n];
        if (T == 0) continue;
        const int grid = std::min(T, per_sm * num_sms);
        if (ch == 1)
            k_detect_tma<1><<<grid, kTmaThreads, smem, s>>>(b);
        else
            k_detect_tma<3><<<grid, kTmaThreads, smem, s>>>(b);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_detect_batch(const uint8_t* const* imgs, const int* Hs, const int* Ws, const int* pitches, int N,
                                int ch, const ScaleTable* sts, uint32_t* const* kps, uint8_t* const* grays,
                                int32_t* status, int num_sms, cudaStream_t s, bool* done)
{
    *done = false;
    if (N < 1) return cudaSuccess;
    bool tma = true;
    for (int i = 0; i < N && tma; ++i) tma = tma_scales(sts[i]) && Hs[i] >= kTmaTile && pitches[i] >= kTmaTile * ch;
    if (tma) {
        const cudaError_t e = launch_detect_tma(imgs, Hs, Ws, pitches, N, ch, sts, kps, grays, status, num_sms, s);
        *done = e == cudaSuccess;
        return e;
    }
    int TS = 0;
    if (!nested_tile(sts[0], &TS)) return cudaSuccess;   // the caller detects image by image
    for (int i0 = 0; i0 < N; i0 += kDetectBatch) {
        DetectBatch b;
        b.n = N - i0 < kDetectBatch ? N - i0 : kDetectBatch;
        b.tile0[0] = 0;
        size_t smem = 0;
        for (int k = 0; k < b.n; ++k) {
            const int i = i0 + k;
            smem = fill_nested(b.im[k], imgs[i], Hs[i], Ws[i], pitches[i], sts[i], TS, kps[i], grays[i]);
            b.tiles_x[k] = (Ws[i] + TS - 1) / TS;
            b.tile0[k + 1] = b.tile0[k] + b.tiles_x[k] * ((Hs[i] + TS - 1) / TS);
        }
        if (b.tile0[b.n] == 0) continue;
        cudaError_t e;
        if (ch == 1) {
            if (smem > 48 * 1024 &&
                (e = cudaFuncSetAttribute(k_detect_nested_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)) != cudaSuccess)
                return e;
            k_detect_nested_batch<1><<<(unsigned)b.tile0[b.n], kDetectThreads, smem, s>>>(b);
        } else {
            if (smem > 48 * 1024 &&
                (e = cudaFuncSetAttribute(k_detect_nested_batch<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)) != cudaSuccess)
                return e;
            k_detect_nested_batch<3><<<(unsigned)b.tile0[b.n], kDetectThreads, smem, s>>>(b);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    *done = true;
    return cudaSuccess;
}

cudaError_t launch_detect(const uint8_t* img, int H, int W, int pitch, int ch, const ScaleTable& st, double alpha,
                          uint32_t* kp, uint8_t* gray, int32_t* status, int num_sms, cudaStream_t s)
{
    if (alpha == 0.0 && tma_scales(st) && H >= kTmaTile && pitch >= kTmaTile * ch)
        return launch_detect_tma(&img, &H, &W, &pitch, 1, ch, &st, &kp, &gray, status, num_sms, s);
    if (alpha > 0.0) {
        if (ch == 3) k_rgb_to_gray<<<1216, 256, 0, s>>>(img, H, W, pitch, gray);
        for (int l = 0; l < st.nL; ++l) {
            const int nw = st.nwx[l] * st.nwy[l];
            if (nw == 0) continue;
            if (ch == 1)
                k_detect_window_ramp<1><<<nw, kDetectThreads, 0, s>>>(img, W, pitch, st.L[l], st.nwx[l], st.off[l],
                                                                      alpha, kp);
            else
                k_detect_window_ramp<3><<<nw, kDetectThreads, 0, s>>>(img, W, pitch, st.L[l], st.nwx[l], st.off[l],
                                                                      alpha, kp);
        }
        return cudaGetLastError();
    }
    int TS = 0;
    const bool nested = nested_tile(st, &TS);
    if (nested) {
        DetectParams p;
        const size_t smem = fill_nested(p, img, H, W, pitch, st, TS, kp, gray);
        dim3 grid((W + TS - 1) / TS, (H + TS - 1) / TS);
        if (ch == 1) {
            if (smem > 48 * 1024) cudaFuncSetAttribute(k_detect_nested<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_detect_nested<1><<<grid, kDetectThreads, smem, s>>>(p);
        } else {
            if (smem > 48 * 1024) cudaFuncSetAttribute(k_detect_nested<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_detect_nested<3><<<grid, kDetectThreads, smem, s>>>(p);
        }
        return cudaGetLastError();
    }
    if (ch == 3) k_rgb_to_gray<<<1216, 256, 0, s>>>(img, H, W, pitch, gray);
    for (int l = 0; l < st.nL; ++l) {
        const int nw = st.nwx[l] * st.nwy[l];
        if (nw == 0) continue;
        if (ch == 1)
            k_detect_window<1><<<nw, kDetectThreads, 0, s>>>(img, H, W, pitch, st.L[l], st.nwx[l], st.off[l], kp);
        else
            k_detect_window<3><<<nw, kDetectThreads, 0, s>>>(img, H, W, pitch, st.L[l], st.nwx[l], st.off[l], kp);
    }
    return cudaGetLastError();
}

cudaError_t launch_diag_gray(const uint8_t* rgb, int64_t n, uint8_t* gray, cudaStream_t s)
{
    k_diag_gray<<<1216, 256, 0, s>>>(rgb, n, gray);
    return cudaGetLastError();
}

}  // namespace lp
