// Orientation and 128-d description of feature points (Sec. 2.3, Eq. 3-5)
// for sm_103a.
//
// One warp per feature point, four points per 128-thread CTA; scales are
// grouped into launches by shared-memory footprint, heaviest first.  The warp
// copies the point's clamped neighbourhood (radius ceil(2*sqrt(2)*w_s + 1.5) +
// 1) from the L2-resident intensity image into shared memory once.
//
// Orientation (integer, exact): 36-bin histogram over the upright
// (4 w_s + 1)^2 window of Eq. 5 gradients.  Bin and weight come from one
// table word per gradient (a, b) that tabulates the exact functions below
// (10-degree sector of atan2(b, a) in bits 25..30; round(65536*sqrt(a^2+b^2))
// by integer square root in bits 0..24), built once per context on the
// device: one gather per sample.  Each weight (< 2^25) is added to two 32-bit
// shared counters per bin, its low 16 and its high 9 bits (for w_s <= 15 at
// most 61^2 samples: no overflow), recombined in 64 bits; the argmax (lowest
// bin on ties) is therefore exact.  Scales above w_s = 15 split each point
// over many CTAs (64-bit bins summed with integer atomics), or take a
// global-memory kernel with per-lane histogram columns when a cell's grid does
// not fit in shared memory.
//
// Descriptor (FP32): the gradient taps p +- e_u, p +- e_v of grid point (u, v)
// are the grid points (u +- 1, v), (u, v +- 1) of the same turned grid, so the
// warp first interpolates the intensity once at every point of the grid
// extended by one sample on each side, then takes Eq. 5 differences.  Lanes 2c
// and 2c+1 own cell c and sum its samples in a private slice (no atomics,
// fixed order); the vector is L2-normalised, clamped at 0.2 and normalised
// again with warp reductions.
#include <cuda_bf16.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kWarps = 4;
constexpr int kAccStride = 9;                  // 8 bins + 1 pad word per lane
constexpr int kAccBytes = 32 * kAccStride * 4;
constexpr int kHistBytes = 36 * 32 * 4;        // [bin][lane] u32
constexpr int kLutBins = 511 * 511;
constexpr int kLutWeights = 2 * 255 * 255 + 1;

struct DescParams {
    const uint8_t* gray;
    int H, W, pitch;
    const uint32_t* kp;
    long long k0, n;        // first point and number of points of this launch
    int ws, P;              // scale of a single-scale launch
    int nl;                 // scales of a multi-scale launch
    long long off[LP_MAX_SCALES + 1];
    int wsl[LP_MAX_SCALES], Pl[LP_MAX_SCALES];
    float cs[36][2];        // cos, sin of (k + 0.5) * 10 degrees
    int upright;
    int hard;               // 1: each magnitude whole in its 45-degree sector, fixed-point grid
    int cq[36], sq[36];     // round(2^11 cos), round(2^11 sin) of (k + 0.5) * 10 degrees
    int warp_bytes, patch_bytes, mid_bytes;
    int word_ok;           // gray base 4-byte aligned and pitch % 4 == 0: interior patches load 32-bit words
    const uint32_t* lut_bw;    // (bin << 25) | weight per gradient (a, b): one gather per orientation sample
    uint8_t* ori;
    float* desc;
    __nv_bfloat16* desc16;
    uint8_t* valid;
};

// 10-degree sector of the direction atan2(b, a) in [0, 360); (a, b) != 0.
// Axes are decided by sign; every other integer gradient with |a|, |b| <= 255
// lies more than 6e-5 sectors from an edge, far above the FP32 error here.
__device__ __forceinline__ int orient_bin(int a, int b)
{
    if (b == 0) return a > 0 ? 0 : 18;
    if (a == 0) return b > 0 ? 9 : 27;
    float phi = atan2f((float)b, (float)a);
    if (phi < 0.f) phi += 6.28318530717958647692f;
    const int k = (int)(phi * 5.72957795130823208768f);   // 36 / (2 pi)
    return k > 35 ? 35 : k;
}

// round(65536 * sqrt(s)) exactly: integer square root of N = s * 2^32 from an
// FP32 estimate, corrected by integer comparisons, then rounded half up
// (sqrt(N) >= r + 1/2  <=>  N > r^2 + r for integers N, r).
__device__ __forceinline__ uint32_t orient_weight(int s)
{
    const unsigned long long N = (unsigned long long)s << 32;
    unsigned long long r = (unsigned long long)(sqrtf((float)s) * 65536.0f);
    while (r * r > N) --r;
    while ((r + 1) * (r + 1) <= N) ++r;
    return (uint32_t)(r + (N > r * r + r ? 1ull : 0ull));
}

// The orientation table: for every integer gradient (a, b) in [-255, 255]^2,
// its 10-degree bin (bits 25..30) and its exact weight round(65536 sqrt(a^2 +
// b^2)) (< 2^25, bits 0..24).
__global__ void k_build_luts(uint32_t* bw)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kLutBins) {
        const int a = i / 511 - 255, b = i % 511 - 255;
        const int bin = (a == 0 && b == 0) ? 0 : orient_bin(a, b);
        bw[i] = ((uint32_t)bin << 25) | orient_weight(a * a + b * b);
    }
}

__global__ void k_diag_orient(int32_t* bins, uint32_t* weights)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (bins && i < kLutBins) {
        const int a = i / 511 - 255, b = i % 511 - 255;
        bins[i] = (a == 0 && b == 0) ? 0 : orient_bin(a, b);
    }
    if (weights && i < kLutWeights) weights[i] = orient_weight(i);
}

// Gradient (a, b) -> magnitude m and direction o in units of 45 degrees,
// o in [0, 8) measured like atan2(b, a).  The 8 descriptor bins are the 8
// octants, so the octant comes exactly from the signs and from |a| vs |b|;
// inside it, atan(t) * 4 / pi for t = min/max in [0, 1] is an odd polynomial
// of degree 13, a least-squares fit at Chebyshev nodes (max error 5e-7 of an
// octant in FP32).  m = x rsqrt(x) (approximate reciprocal square root).
// The zero gradient gives m = 0 and o = 0, so callers may add its weights
// without a test.
__device__ __forceinline__ void grad_polar(float a, float b, float x2, float& m, float& o)
{
    m = x2 * rsqrtf(fmaxf(x2, 1e-30f));
    const float aa = fabsf(a), ab = fabsf(b);
    const float t = __fdividef(fminf(aa, ab), fmaxf(fmaxf(aa, ab), 1e-30f));
    const float u = t * t;
    float g = 0.008711903356015682f;
    g = fmaf(g, u, -0.04294002428650856f);
    g = fmaf(g, u, 0.10161746293306351f);
    g = fmaf(g, u, -0.16867199540138245f);
    g = fmaf(g, u, 0.2522694766521454f);
    g = fmaf(g, u, -0.42422178387641907f);
    g = fmaf(g, u, 1.2732352018356323f);
    g *= t;                                    // atan(t) * 4 / pi
    const float q = ab > aa ? 2.f - g : g;     // angle of (|a|, |b|) in [0, 2]
    o = b >= 0.f ? (a >= 0.f ? q : 4.f - q) : (a >= 0.f ? 8.f - q : 4.f + q);
    if (o >= 8.f) o -= 8.f;
}

// Sec. 2.3 read literally: the sector [45k, 45(k + 1)) degrees that holds
// atan2(b, a), by signs and magnitude comparisons (a direction on an edge
// belongs to the sector it starts); (a, b) != 0.
template <typename T>
__device__ __forceinline__ int octant(T a, T b)
{
    if (b >= 0 && a > 0) return b < a ? 0 : 1;
    if (a <= 0 && b > 0) return b > -a ? 2 : 3;
    if (b <= 0 && a < 0) return -b < -a ? 4 : 5;
    return a < -b ? 6 : 7;
}

// Fixed point of the hard-bin grid: offsets in units of 2^-11 px, intensities
// in units of 2^-22 (every value exact in 32-bit integers: 255 * 2^22 < 2^31).
constexpr int kFx = 11;
constexpr int kFxOne = 1 << kFx;
constexpr float kFxInv2 = 1.f / (float)(1 << (2 * kFx));

// Histogram contribution of the sample at turned-grid point g (row stride G):
// Eq. 5 differences along the turned axes, w0 to bin b0 and w1 to bin
// (b0 + 1) mod 8.  Soft: FP32 grid, the magnitude split linearly between the
// two nearest bins.  Hard: exact fixed-point grid, the whole magnitude in the
// sector of the integer gradient.  False for a zero gradient.
__device__ __forceinline__ bool grid_sample(const float* g, int G, int hard, int& b0, float& w0, float& w1)
{
    if (hard) {
        const int a = __float_as_int(g[G]) - __float_as_int(g[-G]);
        const int b = __float_as_int(g[1]) - __float_as_int(g[-1]);
        if ((a | b) == 0) return false;
        b0 = octant(a, b);
        const float fa = (float)a, fb = (float)b;
        w0 = sqrtf(fa * fa + fb * fb) * kFxInv2;
        w1 = 0.f;
        return true;
    }
    const float a = g[G] - g[-G];
    const float b = g[1] - g[-1];
    const float x2 = a * a + b * b;
    if (!(x2 > 0.f)) return false;
    float m, o;
    grad_polar(a, b, x2, m, o);
    b0 = (int)o;
    const float t = o - (float)b0;
    w0 = m * (1.f - t);
    w1 = m * t;
    return true;
}

// Shared-memory row stride of an S-wide patch: room for the up-to-3-byte shift
// of word-aligned rows.
__host__ __device__ __forceinline__ int patch_stride(int S) { return 4 * ((S + 6) / 4); }

// Bilinear intensity at (row, col) offsets relative to the patch centre;
// nested linear interpolation, exact on flat neighbourhoods.
__device__ __forceinline__ float bilinear(const uint8_t* patch, int S, int P, float r, float c)
{
    const float r0 = floorf(r), c0 = floorf(c);
    const float fr = r - r0, fc = c - c0;
    const uint8_t* q = patch + ((int)r0 + P) * S + (int)c0 + P;
    const float v00 = q[0], v01 = q[1], v10 = q[S], v11 = q[S + 1];
    const float top = v00 + fc * (v01 - v00);
    const float bot = v10 + fc * (v11 - v10);
    return top + fr * (bot - top);
}

// 2^22 * bilinear intensity at the fixed-point offset (r, c) * 2^-11 from the
// patch centre, exact.
__device__ __forceinline__ int bilinear_fx(const uint8_t* patch, int S, int P, int r, int c)
{
    const int fr = r & (kFxOne - 1), fc = c & (kFxOne - 1);
    const uint8_t* q = patch + ((r >> kFx) + P) * S + (c >> kFx) + P;
    const int top = (int)q[0] * (kFxOne - fc) + (int)q[1] * fc;
    const int bot = (int)q[S] * (kFxOne - fc) + (int)q[S + 1] * fc;
    return top * (kFxOne - fr) + bot * fr;
}

// One turned-grid value at frame offset (fu, fv): the FP32 bilinear intensity
// at (fu c - fv s, fu s + fv c), or (hard) the exact fixed-point one at
// (fu cq - fv sq, fu sq + fv cq) * 2^-11, its int bits kept in the float word.
__device__ __forceinline__ void grid_value(float* dst, const uint8_t* patch, int S, int P, int fu, int fv, float c,
                                           float s, int hard, int cq, int sq)
{
    if (hard)
        *dst = __int_as_float(bilinear_fx(patch, S, P, fu * cq - fv * sq, fu * sq + fv * cq));
    else
        *dst = bilinear(patch, S, P, (float)fu * c - (float)fv * s, (float)fu * s + (float)fv * c);
}

// Argmax of the 36 exact orientation sums (lowest bin on ties), one warp: each
// sum v < 2^37 becomes the key (v << 6) | (63 - bin), unique per bin, and the
// key's maximum is taken as two 32-bit warp reductions (high word, then the low
// word among the lanes holding the maximal high word; a real key's low word is
// never 0).
__device__ __forceinline__ int hist_argmax(const uint32_t* hlo, const uint32_t* hhi, int lane)
{
    unsigned long long key = ((((unsigned long long)hhi[lane] << 16) + hlo[lane]) << 6) | (unsigned)(63 - lane);
    if (lane < 4) {
        const int b1 = lane + 32;
        const unsigned long long k1 = ((((unsigned long long)hhi[b1] << 16) + hlo[b1]) << 6) | (unsigned)(63 - b1);
        key = k1 > key ? k1 : key;
    }
    const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
    const uint32_t top = __reduce_max_sync(0xFFFFFFFFu, hi);
    const uint32_t low = __reduce_max_sync(0xFFFFFFFFu, hi == top ? lo : 0u);
    return 63 - (int)(low & 63u);
}

// Row y and column x of pixel id (< 2^24) of a W-wide image: a float quotient
// corrected by integer steps.
__device__ __forceinline__ void pixel_yx(uint32_t id, int W, int& y, int& x)
{
    y = (int)__fdividef((float)id, (float)W);
    x = (int)id - y * W;
    while (x < 0) { --y; x += W; }
    while (x >= W) { ++y; x -= W; }
}

// Walk the flattened index e = lane, lane + 32, ... of an n-wide 2-D range
// without divisions.
struct Walk2D {
    int r, c, dr, dc, n;
    __device__ __forceinline__ Walk2D(int lane, int n_) : n(n_)
    {
        // lane / n_ and 32 / n_ (n_ <= 127): (x + 1/2) / n_ lies at least
        // 1/(2 n_) from an integer, far above the quotient's 2-ulp error
        const float rn = __fdividef(1.f, (float)n_);
        r = (int)(((float)lane + 0.5f) * rn); c = lane - r * n_;
        dr = (int)(32.5f * rn); dc = 32 - dr * n_;
    }
    __device__ __forceinline__ void next()
    {
        r += dr; c += dc;
        if (c >= n) { c -= n; ++r; }
    }
};

// kHard: the hard 8-direction histogram on the fixed-point grid (a compile-time
// choice, so the soft path's loops carry no test of it).
template <int kHard>
__global__ void __launch_bounds__(kWarps * 32) k_describe_all(const DescParams p)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // heaviest points (last in canonical order) first
    const long long idx = (long long)blockIdx.x * kWarps + warp;
    if (idx >= p.n) return;
    const long long k = p.k0 + p.n - 1 - idx;
    int l = 0;
    while (l + 1 < p.nl && k >= p.off[l + 1]) ++l;
    // the turned grid first, then the neighbourhood and the orientation
    // counters; the descriptor accumulators reuse those bytes once the grid
    // is built
    uint8_t* const base = sm + warp * p.warp_bytes + p.mid_bytes;
    uint8_t* patch = base;
    float* grid = reinterpret_cast<float*>(sm + warp * p.warp_bytes);
    uint32_t* hlo = reinterpret_cast<uint32_t*>(base + p.patch_bytes);   // [36]
    uint32_t* hhi = hlo + 36;                                           // [36]
    float* acc = reinterpret_cast<float*>(base);
    const int ws = p.wsl[l], R = 2 * ws, P = p.Pl[l], S = 2 * P + 1, SP = patch_stride(S);
    const uint32_t id = __ldg(p.kp + k);
    int y, x;
    pixel_yx(id, p.W, y, x);

    // neighbourhood: aligned 32-bit words for interior points (row r of the
    // patch starts `off` bytes into shared row r), clamped bytes near the edge
    if (p.word_ok && y >= P && y + P < p.H && x >= P && x + P + 3 < p.W) {
        const int off = (x - P) & 3, nw = (off + S + 3) >> 2;
        const uint8_t* src = p.gray + (size_t)(y - P) * p.pitch + (x - P - off);
        Walk2D w(lane, nw);
#pragma unroll 2
        for (; w.r < S; w.next())
            reinterpret_cast<uint32_t*>(base + w.r * SP)[w.c] =
                __ldg(reinterpret_cast<const uint32_t*>(src + (size_t)w.r * p.pitch) + w.c);
        patch = base + off;
    } else {
        Walk2D w(lane, S);
#pragma unroll 4
        for (; w.r < S; w.next()) {
            const int yy = min(max(y - P + w.r, 0), p.H - 1), xx = min(max(x - P + w.c, 0), p.W - 1);
            patch[w.r * SP + w.c] = __ldg(p.gray + (size_t)yy * p.pitch + xx);
        }
    }
    if (lane < 36) { hlo[lane] = 0u; hhi[lane] = 0u; }
    if (lane < 4) { hlo[lane + 32] = 0u; hhi[lane + 32] = 0u; }
    __syncwarp();

    // ---- orientation: exact integer histogram over the upright window; each
    // weight (< 2^25) is added as its low 16 and high 9 bits to two 32-bit
    // counters, which cannot overflow for w_s <= 15
    int best = 0;
    if (!p.upright) {
        const int n = 2 * R + 1;
        const uint8_t* c0 = patch + (P - R) * SP + (P - R);
        Walk2D w(lane, n);
        for (; w.r < n; w.next()) {
            const uint8_t* q = c0 + w.r * SP + w.c;
            const int a = (int)q[SP] - (int)q[-SP];
            const int b = (int)q[1] - (int)q[-1];
            // the table's entry for a zero gradient is bin 0, weight 0
            const uint32_t e = __ldg(p.lut_bw + (a + 255) * 511 + (b + 255));
            const int bin = (int)(e >> 25);
            const uint32_t wt = e & 0x1FFFFFFu;
            atomicAdd(&hlo[bin], wt & 0xFFFFu);
            atomicAdd(&hhi[bin], wt >> 16);
        }
        __syncwarp();
        best = hist_argmax(hlo, hhi, lane);
    }
    const float c = p.upright ? 1.f : p.cs[best][0];
    const float s = p.upright ? 0.f : p.cs[best][1];
    const int cq = p.upright ? kFxOne : p.cq[best], sq = p.upright ? 0 : p.sq[best];

    // ---- intensities of the turned grid, extended by one sample on each side
    const int G = 2 * R + 2;
    {
        Walk2D w(lane, G);
        for (; w.r < G; w.next())
            grid_value(grid + w.r * G + w.c, patch, SP, P, w.r - R - 1, w.c - R - 1, c, s, kHard, cq, sq);
    }
    __syncwarp();   // every lane is done with the neighbourhood
    float* mine = acc + lane * kAccStride;
#pragma unroll
    for (int q = 0; q < 8; ++q) mine[q] = 0.f;
    __syncwarp();

    // ---- descriptor samples: Eq. 5 differences along the turned axes
    const int cell = lane >> 1, cr = cell >> 2, cc = cell & 3;
    int iu = 0, iv = lane & 1;
    while (iv >= ws) { iv -= ws; ++iu; }
    for (; iu < ws;) {
        int b0;
        float w0, w1;
        const float* g = grid + (cr * ws + iu + 1) * G + cc * ws + iv + 1;
        if (kHard) {
            if (grid_sample(g, G, 1, b0, w0, w1)) mine[b0] += w0;
        } else {
            // a zero gradient adds zero to bin 0
            const float a = g[G] - g[-G], b = g[1] - g[-1];
            float m, o;
            grad_polar(a, b, a * a + b * b, m, o);
            b0 = (int)o;
            const float t = o - (float)b0;
            mine[b0] += m * (1.f - t);
            mine[(b0 + 1) & 7] += m * t;
        }
        iv += 2;
        while (iv >= ws) { iv -= ws; ++iu; }
    }
    __syncwarp();
    // lane L owns outputs 4L..4L+3: cell L/2, bins 4*(L&1) .. +3
    const float* e0 = acc + (2 * cell) * kAccStride + 4 * (lane & 1);
    const float* e1 = e0 + kAccStride;
    float v[4];
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = e0[q] + e1[q];
        ss += v[q] * v[q];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    const float nrm = sqrtf(ss);
    const bool ok = nrm > 0.f;
    const float inv = ok ? 1.f / nrm : 0.f;
    float ss2 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = fminf(v[q] * inv, 0.2f);
        ss2 += v[q] * v[q];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss2 += __shfl_xor_sync(0xFFFFFFFFu, ss2, o);
    const float inv2 = ok ? 1.f / sqrtf(ss2) : 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] *= inv2;
    reinterpret_cast<float4*>(p.desc + k * 128)[lane] = make_float4(v[0], v[1], v[2], v[3]);
    if (p.desc16) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&lo);
        w.y = *reinterpret_cast<uint32_t*>(&hi);
        reinterpret_cast<uint2*>(p.desc16 + k * 128)[lane] = w;
    }
    if (lane == 0) {
        p.ori[k] = (uint8_t)best;
        p.valid[k] = ok ? 1 : 0;
    }
}

// Large scales (few points, long loops): one 128-thread CTA per point, the
// same arithmetic as k_describe_all with the loops spread over four warps.
// Cell c's samples are split over threads 8c .. 8c+7 (one warp holds four
// cells); their partial histograms are added in a fixed shuffle order.
constexpr int kCtaThreads = 128;

__global__ void __launch_bounds__(kCtaThreads) k_describe_cta(const DescParams p)
{
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ uint32_t hlo[36], hhi[36];
    __shared__ float red[kCtaThreads / 32];
    __shared__ int best_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long k = p.k0 + p.n - 1 - blockIdx.x;   // heaviest first
    const int ws = p.ws, R = 2 * ws, P = p.P, S = 2 * P + 1, G = 2 * R + 2, SP = patch_stride(S);
    uint8_t* patch = sm;
    float* grid = reinterpret_cast<float*>(sm + p.patch_bytes);
    const uint32_t id = __ldg(p.kp + k);
    int y, x;
    pixel_yx(id, p.W, y, x);
    if (p.word_ok && y >= P && y + P < p.H && x >= P && x + P + 3 < p.W) {
        const int off = (x - P) & 3, nw = (off + S + 3) >> 2;
        const uint8_t* src = p.gray + (size_t)(y - P) * p.pitch + (x - P - off);
        for (int e = tid; e < S * nw; e += kCtaThreads) {
            const int r = e / nw, c = e - (e / nw) * nw;
            reinterpret_cast<uint32_t*>(sm + r * SP)[c] = __ldg(reinterpret_cast<const uint32_t*>(src + (size_t)r * p.pitch) + c);
        }
        patch = sm + off;
    } else {
        for (int e = tid; e < S * S; e += kCtaThreads) {
            const int r = e / S, c = e - (e / S) * S;
            const int yy = min(max(y - P + r, 0), p.H - 1), xx = min(max(x - P + c, 0), p.W - 1);
            patch[r * SP + c] = __ldg(p.gray + (size_t)yy * p.pitch + xx);
        }
    }
    if (tid < 36) { hlo[tid] = 0u; hhi[tid] = 0u; }
    __syncthreads();
    int best = 0;
    if (!p.upright) {
        const int n = 2 * R + 1;
        const uint8_t* c0 = patch + (P - R) * SP + (P - R);
        for (int e = tid; e < n * n; e += kCtaThreads) {
            const int r = e / n, c = e - (e / n) * n;
            const uint8_t* q = c0 + r * SP + c;
            const int a = (int)q[SP] - (int)q[-SP];
            const int b = (int)q[1] - (int)q[-1];
            if (a | b) {
                const uint32_t e = __ldg(p.lut_bw + (a + 255) * 511 + (b + 255));
                const int bin = (int)(e >> 25);
                const uint32_t wt = e & 0x1FFFFFFu;
                atomicAdd(&hlo[bin], wt & 0xFFFFu);
                atomicAdd(&hhi[bin], wt >> 16);
            }
        }
        __syncthreads();
        if (warp == 0) {
            const int bb = hist_argmax(hlo, hhi, lane);
            if (lane == 0) best_s = bb;
        }
        __syncthreads();
        best = best_s;
    }
    const float c = p.upright ? 1.f : p.cs[best][0];
    const float s = p.upright ? 0.f : p.cs[best][1];
    const int cq = p.upright ? kFxOne : p.cq[best], sq = p.upright ? 0 : p.sq[best];
    for (int e = tid; e < G * G; e += kCtaThreads) {
        const int iu = e / G, iv = e - (e / G) * G;
        grid_value(grid + e, patch, SP, P, iu - R - 1, iv - R - 1, c, s, p.hard, cq, sq);
    }
    __syncthreads();
    const int cell = tid >> 3, sub = tid & 7, cr = cell >> 2, cc = cell & 3;
    float h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = 0.f;
    for (int i = sub; i < ws * ws; i += 8) {
        const int iu = i / ws, iv = i - (i / ws) * ws;
        int b0;
        float w0, w1;
        if (grid_sample(grid + (cr * ws + iu + 1) * G + cc * ws + iv + 1, G, p.hard, b0, w0, w1)) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                h[q] += (q == b0) ? w0 : 0.f;
                h[q] += (q == ((b0 + 1) & 7)) ? w1 : 0.f;
            }
        }
    }
    // sum the 8 threads of the cell (fixed shuffle order)
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
        for (int q = 0; q < 8; ++q) h[q] += __shfl_xor_sync(0xFFFFFFFFu, h[q], o);
    // thread t keeps output (cell t/8, bin t%8)
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) v = (q == sub) ? h[q] : v;
    float ss = v * v;
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    ss = red[0] + red[1] + red[2] + red[3];
    const float nrm = sqrtf(ss);
    const bool ok = nrm > 0.f;
    v = fminf(v * (ok ? 1.f / nrm : 0.f), 0.2f);
    float ss2 = v * v;
#pragma unroll
    for (int o = 16; o; o >>= 1) ss2 += __shfl_xor_sync(0xFFFFFFFFu, ss2, o);
    __syncthreads();
    if (lane == 0) red[warp] = ss2;
    __syncthreads();
    ss2 = red[0] + red[1] + red[2] + red[3];
    v *= ok ? 1.f / sqrtf(ss2) : 0.f;
    p.desc[k * 128 + tid] = v;
    if (p.desc16) p.desc16[k * 128 + tid] = __float2bfloat16_rn(v);
    if (tid == 0) {
        p.ori[k] = (uint8_t)best;
        p.valid[k] = ok ? 1 : 0;
    }
}

// Fallback for scales whose neighbourhood does not fit in shared memory: the
// same arithmetic with clamped reads from the (L2-resident) intensity image
// and four bilinear evaluations per descriptor sample.
__global__ void __launch_bounds__(kWarps * 32) k_describe_global(const DescParams p)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long idx = (long long)blockIdx.x * kWarps + warp;
    if (idx >= p.n) return;
    const long long k = p.k0 + idx;
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(sm + warp * (2 * kHistBytes + kAccBytes));
    float* acc = reinterpret_cast<float*>(sm + warp * (2 * kHistBytes + kAccBytes) + 2 * kHistBytes);
    const int ws = p.ws, R = 2 * ws;
    const uint32_t id = __ldg(p.kp + k);
    int y, x;
    pixel_yx(id, p.W, y, x);
    auto px = [&](int r, int c) -> int {
        const int yy = min(max(y + r, 0), p.H - 1), xx = min(max(x + c, 0), p.W - 1);
        return __ldg(p.gray + (size_t)yy * p.pitch + xx);
    };
    auto bil = [&](float r, float c) -> float {
        const float r0 = floorf(r), c0 = floorf(c);
        const float fr = r - r0, fc = c - c0;
        const int yi = (int)r0, xi = (int)c0;
        const float v00 = px(yi, xi), v01 = px(yi, xi + 1), v10 = px(yi + 1, xi), v11 = px(yi + 1, xi + 1);
        const float top = v00 + fc * (v01 - v00);
        const float bot = v10 + fc * (v11 - v10);
        return top + fr * (bot - top);
    };
    int best = 0;
    if (!p.upright) {
        for (int b = 0; b < 36; ++b) hist[b * 32 + lane] = 0ull;
        for (int u = -R; u <= R; ++u)
            for (int v = lane - R; v <= R; v += 32) {
                const int a = px(u + 1, v) - px(u - 1, v);
                const int b = px(u, v + 1) - px(u, v - 1);
                if (a | b) {
                    const uint32_t e = __ldg(p.lut_bw + (a + 255) * 511 + (b + 255));
                    hist[(e >> 25) * 32 + lane] += e & 0x1FFFFFFu;
                }
            }
        __syncwarp();
        unsigned long long t0 = 0, t1 = 0;
        for (int l = 0; l < 32; ++l) t0 += hist[lane * 32 + ((l + lane) & 31)];
        if (lane < 4)
            for (int l = 0; l < 32; ++l) t1 += hist[(lane + 32) * 32 + ((l + lane) & 31)];
        unsigned long long bv = t0;
        int bb = lane;
        if (lane < 4 && t1 > t0) { bv = t1; bb = lane + 32; }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long ov = __shfl_xor_sync(0xFFFFFFFFu, bv, o);
            const int ob = __shfl_xor_sync(0xFFFFFFFFu, bb, o);
            if (ov > bv || (ov == bv && ob < bb)) { bv = ov; bb = ob; }
        }
        best = bb;
    }
    const float c = p.upright ? 1.f : p.cs[best][0];
    const float s = p.upright ? 0.f : p.cs[best][1];
    const int cq = p.upright ? kFxOne : p.cq[best], sq = p.upright ? 0 : p.sq[best];
    auto bil_fx = [&](int r, int c_) -> int {
        const int fr = r & (kFxOne - 1), fc = c_ & (kFxOne - 1), yi = r >> kFx, xi = c_ >> kFx;
        const int top = px(yi, xi) * (kFxOne - fc) + px(yi, xi + 1) * fc;
        const int bot = px(yi + 1, xi) * (kFxOne - fc) + px(yi + 1, xi + 1) * fc;
        return top * (kFxOne - fr) + bot * fr;
    };
    float* mine = acc + lane * kAccStride;
    for (int q = 0; q < 8; ++q) mine[q] = 0.f;
    const int cell = lane >> 1, cr = cell >> 2, cc = cell & 3;
    for (int i = lane & 1; i < ws * ws; i += 2) {
        const int iu = -R + cr * ws + i / ws, iv = -R + cc * ws + i % ws;
        // the sample's four neighbours along the turned axes, as a 3 x 3 grid
        // patch with the unused corners left out
        float nb[9];
        if (p.hard) {
            const int pr = iu * cq - iv * sq, pc = iu * sq + iv * cq;
            nb[1] = __int_as_float(bil_fx(pr - cq, pc - sq));
            nb[7] = __int_as_float(bil_fx(pr + cq, pc + sq));
            nb[3] = __int_as_float(bil_fx(pr + sq, pc - cq));
            nb[5] = __int_as_float(bil_fx(pr - sq, pc + cq));
        } else {
            const float fu = (float)iu, fv = (float)iv;
            const float dy = fu * c - fv * s, dx = fu * s + fv * c;
            nb[1] = bil(dy - c, dx - s);
            nb[7] = bil(dy + c, dx + s);
            nb[3] = bil(dy + s, dx - c);
            nb[5] = bil(dy - s, dx + c);
        }
        int b0;
        float w0, w1;
        if (grid_sample(nb + 4, 3, p.hard, b0, w0, w1)) {
            mine[b0] += w0;
            mine[(b0 + 1) & 7] += w1;
        }
    }
    __syncwarp();
    const float* e0 = acc + (2 * cell) * kAccStride + 4 * (lane & 1);
    const float* e1 = e0 + kAccStride;
    float v[4];
    float ss = 0.f;
    for (int q = 0; q < 4; ++q) { v[q] = e0[q] + e1[q]; ss += v[q] * v[q]; }
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    const float nrm = sqrtf(ss);
    const bool ok = nrm > 0.f;
    float ss2 = 0.f;
    const float inv = ok ? 1.f / nrm : 0.f;
    for (int q = 0; q < 4; ++q) { v[q] = fminf(v[q] * inv, 0.2f); ss2 += v[q] * v[q]; }
    for (int o = 16; o; o >>= 1) ss2 += __shfl_xor_sync(0xFFFFFFFFu, ss2, o);
    const float inv2 = ok ? 1.f / sqrtf(ss2) : 0.f;
    for (int q = 0; q < 4; ++q) v[q] *= inv2;
    reinterpret_cast<float4*>(p.desc + k * 128)[lane] = make_float4(v[0], v[1], v[2], v[3]);
    if (p.desc16) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&lo);
        w.y = *reinterpret_cast<uint32_t*>(&hi);
        reinterpret_cast<uint2*>(p.desc16 + k * 128)[lane] = w;
    }
    if (lane == 0) {
        p.ori[k] = (uint8_t)best;
        p.valid[k] = ok ? 1 : 0;
    }
}

// ---------------------------------------------------------------- split path
// Scales with w_s > 15 have few points and long per-point loops, so one point's
// work is spread over many CTAs:
//   k_orient_split   CTA (point, band of rows of the upright (4 w_s + 1)^2
//                    window): Eq. 5 gradient weights summed per bin in shared
//                    memory (low 16 and high 9 bits, as k_describe_cta), then
//                    added to the point's 64-bit bins in global memory.  The
//                    sums are integers, so their order does not matter.
//   k_orient_pick    one thread per point: argmax, the lowest bin on ties.
//   k_desc_cell      CTA (point, cell): the cell's turned (w_s + 2)^2 grid is
//                    interpolated once from the neighbourhood staged in shared
//                    memory; Eq. 5 differences; soft 8-bin histogram summed in
//                    a fixed order; the cell's 8 raw values are written.
//   k_desc_finalize  one warp per point: L2 norm, clamp at 0.2, L2 norm.
// The 36 bins of a point live in its own descriptor row (288 of its 512
// bytes) until k_desc_cell overwrites the row.
constexpr int kSplitThreads = 256;
constexpr int kOrientBandSamples = 4096;

__global__ void __launch_bounds__(kSplitThreads) k_orient_split(const DescParams p, int rows_per_band, int nbands)
{
    __shared__ uint32_t hlo[36], hhi[36];
    const long long idx = blockIdx.x / nbands;
    const int band = (int)(blockIdx.x - idx * nbands);
    const long long k = p.k0 + idx;
    const int R = 2 * p.ws, n = 2 * R + 1;
    const uint32_t id = __ldg(p.kp + k);
    int y, x;
    pixel_yx(id, p.W, y, x);
    auto px = [&](int yy, int xx) -> int {
        yy = min(max(yy, 0), p.H - 1);
        xx = min(max(xx, 0), p.W - 1);
        return __ldg(p.gray + (size_t)yy * p.pitch + xx);
    };
    if (threadIdx.x < 36) { hlo[threadIdx.x] = 0u; hhi[threadIdx.x] = 0u; }
    __syncthreads();
    const int u0 = band * rows_per_band, u1 = min(n, u0 + rows_per_band);
    const int cnt = (u1 - u0) * n;
    for (int e = threadIdx.x; e < cnt; e += kSplitThreads) {
        const int r = u0 + e / n, c = e - (e / n) * n;
        const int yy = y + r - R, xx = x + c - R;
        const int a = px(yy + 1, xx) - px(yy - 1, xx);
        const int b = px(yy, xx + 1) - px(yy, xx - 1);
        if (a | b) {
            const uint32_t e = __ldg(p.lut_bw + (a + 255) * 511 + (b + 255));
            const int bin = (int)(e >> 25);
            const uint32_t wt = e & 0x1FFFFFFu;
            atomicAdd(&hlo[bin], wt & 0xFFFFu);
            atomicAdd(&hhi[bin], wt >> 16);
        }
    }
    __syncthreads();
    if (threadIdx.x < 36) {
        const unsigned long long v = ((unsigned long long)hhi[threadIdx.x] << 16) + hlo[threadIdx.x];
        if (v) atomicAdd(reinterpret_cast<unsigned long long*>(p.desc + k * 128) + threadIdx.x, v);
    }
}

__global__ void __launch_bounds__(128) k_orient_pick(const DescParams p)
{
    const long long idx = (long long)blockIdx.x * 128 + threadIdx.x;
    if (idx >= p.n) return;
    const long long k = p.k0 + idx;
    const unsigned long long* h = reinterpret_cast<const unsigned long long*>(p.desc + k * 128);
    unsigned long long bv = h[0];
    int bb = 0;
    for (int b = 1; b < 36; ++b)
        if (h[b] > bv) { bv = h[b]; bb = b; }
    p.ori[k] = (uint8_t)bb;
}

// Shared memory of k_desc_cell for cell grids of side Gc = w_s + 2: the staged
// neighbourhood (side at most ceil((Gc - 1) sqrt 2) + 6, rows padded to 4
// bytes) and the FP32 grid.
__host__ __device__ __forceinline__ int cell_box_side(int Gc) { return (int)((Gc - 1) * 1.41422f) + 7; }
__host__ __device__ __forceinline__ int cell_box_bytes(int Gc)
{
    const int b = cell_box_side(Gc);
    return ((b * ((b + 3) & ~3)) + 15) / 16 * 16;
}

__global__ void __launch_bounds__(kSplitThreads) k_desc_cell(const DescParams p)
{
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ float red[kSplitThreads / 32][8];
    const long long idx = blockIdx.x >> 4;
    const int cell = blockIdx.x & 15, cr = cell >> 2, cq = cell & 3;
    const long long k = p.k0 + idx;
    const int ws = p.ws, R = 2 * ws, Gc = ws + 2;
    const int bmax = cell_box_side(Gc);
    const uint32_t id = __ldg(p.kp + k);
    int y, x;
    pixel_yx(id, p.W, y, x);
    const int best = p.upright ? 0 : p.ori[k];
    const float c = p.upright ? 1.f : p.cs[best][0];
    const float s = p.upright ? 0.f : p.cs[best][1];
    const int tq = p.upright ? kFxOne : p.cq[best], ts = p.upright ? 0 : p.sq[best];
    // frame points (fu, fv) = (fu0 + iu, fv0 + iv), iu, iv in [0, Gc): image
    // offsets (dy, dx) = (fu c - fv s, fu s + fv c) from the point (hard: the
    // fixed-point turn (tq, ts) * 2^-11)
    const int fu0 = -R + cr * ws - 1, fv0 = -R + cq * ws - 1;
    float ymin = 3.4e38f, ymax = -3.4e38f, xmin = 3.4e38f, xmax = -3.4e38f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int iu = fu0 + ((q & 1) ? Gc - 1 : 0), iv = fv0 + ((q & 2) ? Gc - 1 : 0);
        float dy, dx;
        if (p.hard) {
            dy = (float)((iu * tq - iv * ts) >> kFx);
            dx = (float)((iu * ts + iv * tq) >> kFx);
        } else {
            const float fu = (float)iu, fv = (float)iv;
            dy = fu * c - fv * s;
            dx = fu * s + fv * c;
        }
        ymin = fminf(ymin, dy); ymax = fmaxf(ymax, dy); xmin = fminf(xmin, dx); xmax = fmaxf(xmax, dx);
    }
    // one spare row and column on each side; the taps below are clamped to the box
    const int r0 = (int)floorf(ymin) - 1, c0 = (int)floorf(xmin) - 1;
    const int nr = min(bmax, (int)floorf(ymax) + 3 - r0), nc = min(bmax, (int)floorf(xmax) + 3 - c0);
    const int SPc = (bmax + 3) & ~3;
    uint8_t* box = sm;
    float* grid = reinterpret_cast<float*>(sm + cell_box_bytes(Gc));
    for (int e = threadIdx.x; e < nr * nc; e += kSplitThreads) {
        const int r = e / nc, q = e - (e / nc) * nc;
        const int yy = min(max(y + r0 + r, 0), p.H - 1), xx = min(max(x + c0 + q, 0), p.W - 1);
        box[r * SPc + q] = __ldg(p.gray + (size_t)yy * p.pitch + xx);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Gc * Gc; e += kSplitThreads) {
        const int iu = e / Gc, iv = e - (e / Gc) * Gc;
        if (p.hard) {
            // box-relative fixed-point offset (the box covers every tap; the
            // clamp only keeps reads inside it)
            const int rr = (fu0 + iu) * tq - (fv0 + iv) * ts - r0 * kFxOne;
            const int cc = (fu0 + iu) * ts + (fv0 + iv) * tq - c0 * kFxOne;
            const int ri = min(max(rr >> kFx, 0), nr - 2), ci = min(max(cc >> kFx, 0), nc - 2);
            const int fr = rr & (kFxOne - 1), fc = cc & (kFxOne - 1);
            const uint8_t* b0 = box + ri * SPc + ci;
            const int top = (int)b0[0] * (kFxOne - fc) + (int)b0[1] * fc;
            const int bot = (int)b0[SPc] * (kFxOne - fc) + (int)b0[SPc + 1] * fc;
            grid[e] = __int_as_float(top * (kFxOne - fr) + bot * fr);
            continue;
        }
        const float fu = (float)(fu0 + iu), fv = (float)(fv0 + iv);
        const float rr = fu * c - fv * s - (float)r0, cc = fu * s + fv * c - (float)c0;
        const float rf = floorf(rr), cf = floorf(cc);
        const int ri = min(max((int)rf, 0), nr - 2), ci = min(max((int)cf, 0), nc - 2);
        const float fr = rr - rf, fc = cc - cf;
        const uint8_t* b0 = box + ri * SPc + ci;
        const float v00 = b0[0], v01 = b0[1], v10 = b0[SPc], v11 = b0[SPc + 1];
        const float top = v00 + fc * (v01 - v00);
        const float bot = v10 + fc * (v11 - v10);
        grid[e] = top + fr * (bot - top);
    }
    __syncthreads();
    float h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = 0.f;
    for (int i = threadIdx.x; i < ws * ws; i += kSplitThreads) {
        const int iu = i / ws, iv = i - (i / ws) * ws;
        int b0;
        float w0, w1;
        if (grid_sample(grid + (iu + 1) * Gc + iv + 1, Gc, p.hard, b0, w0, w1)) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                h[q] += (q == b0) ? w0 : 0.f;
                h[q] += (q == ((b0 + 1) & 7)) ? w1 : 0.f;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1)
#pragma unroll
        for (int q = 0; q < 8; ++q) h[q] += __shfl_xor_sync(0xFFFFFFFFu, h[q], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 8; ++q) red[warp][q] = h[q];
    __syncthreads();
    if (threadIdx.x < 8) {
        float v = 0.f;
        for (int w = 0; w < kSplitThreads / 32; ++w) v += red[w][threadIdx.x];
        p.desc[k * 128 + cell * 8 + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(128) k_desc_finalize(const DescParams p)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long idx = (long long)blockIdx.x * 4 + warp;
    if (idx >= p.n) return;
    const long long k = p.k0 + idx;
    const float4 r = reinterpret_cast<const float4*>(p.desc + k * 128)[lane];
    float v[4] = {r.x, r.y, r.z, r.w};
    float ss = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) ss += v[q] * v[q];
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
    const float nrm = sqrtf(ss);
    const bool ok = nrm > 0.f;
    const float inv = ok ? 1.f / nrm : 0.f;
    float ss2 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = fminf(v[q] * inv, 0.2f);
        ss2 += v[q] * v[q];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss2 += __shfl_xor_sync(0xFFFFFFFFu, ss2, o);
    const float inv2 = ok ? 1.f / sqrtf(ss2) : 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] *= inv2;
    reinterpret_cast<float4*>(p.desc + k * 128)[lane] = make_float4(v[0], v[1], v[2], v[3]);
    if (p.desc16) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&lo);
        w.y = *reinterpret_cast<uint32_t*>(&hi);
        reinterpret_cast<uint2*>(p.desc16 + k * 128)[lane] = w;
    }
    if (lane == 0) {
        if (p.upright) p.ori[k] = 0;
        p.valid[k] = ok ? 1 : 0;
    }
}

}  // namespace

size_t describe_lut_bytes() { return (size_t)kLutBins * 4 + 256; }

cudaError_t launch_build_luts(void* luts, cudaStream_t s)
{
    k_build_luts<<<(kLutBins + 255) / 256, 256, 0, s>>>(reinterpret_cast<uint32_t*>(luts));
    return cudaGetLastError();
}

// Border rejection (a paper-literal variant; off by default): a point whose
// neighbourhood of radius P = ceil(2 sqrt(2) w_s + 1.5) + 1 -- every pixel its
// orientation window, turned grid and their taps can read -- does not lie
// inside the image is marked invalid, so no kept description depends on the
// clamp-to-edge reading.
struct BorderParams {
    long long off[LP_MAX_SCALES + 1];
    int pr[LP_MAX_SCALES];
    int nL;
};

__global__ void k_border_reject(const uint32_t* kp, int H, int W, const BorderParams b, uint8_t* valid)
{
    const long long k = (long long)blockIdx.x * 256 + threadIdx.x;
    if (k >= b.off[b.nL]) return;
    int l = 0;
    while (l + 1 < b.nL && k >= b.off[l + 1]) ++l;
    const int P = b.pr[l];
    const uint32_t id = kp[k];
    const int y = (int)(id / (uint32_t)W), x = (int)(id - (uint32_t)y * (uint32_t)W);
    if (x < P || y < P || x + P > W - 1 || y + P > H - 1) valid[k] = 0;
}

cudaError_t launch_describe(const uint8_t* gray, int H, int W, int pitch, const uint32_t* kp,
                            const ScaleTable& st, int upright, int border, int hard, const void* luts, uint8_t* ori,
                            float* desc, uint16_t* desc_bf16, uint8_t* valid, const Fork* fork, cudaStream_t s)
{
    if (border) {
        cudaError_t e = launch_describe(gray, H, W, pitch, kp, st, upright, 0, hard, luts, ori, desc, desc_bf16,
                                        valid, fork, s);
        if (e != cudaSuccess) return e;
        BorderParams b;
        b.nL = st.nL;
        for (int l = 0; l <= st.nL; ++l) b.off[l] = st.off[l];
        for (int l = 0; l < st.nL; ++l) b.pr[l] = st.pr[l];
        const long long K = st.off[st.nL];
        if (K > 0) k_border_reject<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(kp, H, W, b, valid);
        return cudaGetLastError();
    }
    DescParams p;
    p.gray = gray; p.H = H; p.W = W; p.pitch = pitch; p.kp = kp;
    for (int k = 0; k < 36; ++k) {
        const double th = (k + 0.5) * 10.0 * 3.14159265358979323846 / 180.0;
        p.cs[k][0] = (float)cos(th);
        p.cs[k][1] = (float)sin(th);
        p.cq[k] = (int)floor(2048.0 * cos(th) + 0.5);
        p.sq[k] = (int)floor(2048.0 * sin(th) + 0.5);
    }
    p.upright = upright;
    p.hard = hard;
    p.word_ok = ((reinterpret_cast<uintptr_t>(gray) & 3u) == 0 && (pitch & 3) == 0) ? 1 : 0;
    p.lut_bw = reinterpret_cast<const uint32_t*>(luts);
    p.ori = ori; p.desc = desc; p.desc16 = reinterpret_cast<__nv_bfloat16*>(desc_bf16); p.valid = valid;
    // Scales with w_s <= 15 whose per-warp shared memory fits kSmallWarpBytes
    // run one warp per point, each scale in a launch sized for its own
    // footprint (the smallest scale, with most of the points, gets the highest
    // occupancy); every larger footprint runs one CTA per point.  Larger
    // footprints are launched first.
    // Scales with w_s > 15 take the split path (many CTAs per point), or the
    // global-memory kernel when a cell's grid does not fit shared memory.
    int m = 0;
    while (m < st.nL && st.ws[m] <= 15) ++m;
    auto warp_bytes = [&](int l) {
        const int S = 2 * st.pr[l] + 1, G = 4 * st.ws[l] + 2;
        return ((S * patch_stride(S) + 15) / 16) * 16 + ((G * G * 4 + 15) / 16) * 16 + 2 * 36 * 4 + kAccBytes;
    };
    constexpr int kSmallWarpBytes = 7680;
    int first_big = 0;
    while (first_big < m && warp_bytes(first_big) <= kSmallWarpBytes) ++first_big;
    // Three independent groups of launches (the per-point CTA scales, the
    // warp-per-point group, the split scales): with a fork they run
    // concurrently, which fills the tail waves of the smaller launches.
    const int ngroups = (first_big < m ? 1 : 0) + (first_big > 0 ? 1 : 0) + (m < st.nL ? 1 : 0);
    const bool forked = fork && ngroups > 1;
    const cudaStream_t s_cta = forked ? fork->aux[0] : s, s_big = forked ? fork->aux[1] : s;
    if (forked) {
        cudaError_t e = cudaEventRecord(fork->fork_ev, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->aux[0], fork->fork_ev, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fork->aux[1], fork->fork_ev, 0);
        if (e != cudaSuccess) return e;
    }
    auto launch_group = [&](int l0, int l1) -> cudaError_t {
        int Pmax = 0, Gmax = 0;
        for (int l = l0; l < l1; ++l) {
            Pmax = Pmax > st.pr[l] ? Pmax : st.pr[l];
            Gmax = Gmax > 4 * st.ws[l] + 2 ? Gmax : 4 * st.ws[l] + 2;
        }
        p.nl = l1 - l0;
        for (int l = l0; l <= l1; ++l) p.off[l - l0] = st.off[l];
        for (int l = l0; l < l1; ++l) { p.wsl[l - l0] = st.ws[l]; p.Pl[l - l0] = st.pr[l]; }
        p.k0 = st.off[l0];
        p.n = st.off[l1] - st.off[l0];
        if (p.n == 0) return cudaSuccess;
        const int S = 2 * Pmax + 1;
        p.patch_bytes = ((S * patch_stride(S) + 15) / 16) * 16;
        p.mid_bytes = ((Gmax * Gmax * 4) + 15) / 16 * 16;
        // the accumulators alias the neighbourhood and the counters
        const int tail = p.patch_bytes + 2 * 36 * 4;
        p.warp_bytes = p.mid_bytes + (tail > kAccBytes ? tail : kAccBytes);
        const size_t smem = (size_t)kWarps * p.warp_bytes;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(p.hard ? k_describe_all<1> : k_describe_all<0>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        if (p.hard)
            k_describe_all<1><<<(unsigned)((p.n + kWarps - 1) / kWarps), kWarps * 32, smem, s>>>(p);
        else
            k_describe_all<0><<<(unsigned)((p.n + kWarps - 1) / kWarps), kWarps * 32, smem, s>>>(p);
        return cudaGetLastError();
    };
    for (int l = m - 1; l >= first_big; --l) {
        p.k0 = st.off[l];
        p.n = st.off[l + 1] - st.off[l];
        if (p.n == 0) continue;
        p.ws = st.ws[l];
        p.P = st.pr[l];
        const int S = 2 * p.P + 1, G = 4 * p.ws + 2;
        p.patch_bytes = ((S * patch_stride(S) + 15) / 16) * 16;
        const size_t smem = (size_t)p.patch_bytes + (size_t)G * G * 4;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_describe_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_describe_cta<<<(unsigned)p.n, kCtaThreads, smem, s_cta>>>(p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int l = first_big - 1; l >= 0; --l) {
        cudaError_t e = launch_group(l, l + 1);
        if (e != cudaSuccess) return e;
    }
    for (int l = m; l < st.nL; ++l) {
        p.k0 = st.off[l];
        p.n = st.off[l + 1] - st.off[l];
        if (p.n == 0) continue;
        p.ws = st.ws[l];
        p.P = st.pr[l];
        const int Gc = p.ws + 2;
        const size_t csm = (size_t)cell_box_bytes(Gc) + (size_t)Gc * Gc * 4;
        if (csm > 200 * 1024) {
            const unsigned grid = (unsigned)((p.n + kWarps - 1) / kWarps);
            k_describe_global<<<grid, kWarps * 32, (size_t)kWarps * (2 * kHistBytes + kAccBytes), s_big>>>(p);
            continue;
        }
        if (!upright) {
            cudaError_t e = cudaMemsetAsync(desc + p.k0 * 128, 0, sizeof(float) * 128 * (size_t)p.n, s_big);
            if (e != cudaSuccess) return e;
            const int n = 4 * p.ws + 1;
            const int rows = kOrientBandSamples / n > 1 ? kOrientBandSamples / n : 1;
            const int nb = (n + rows - 1) / rows;
            k_orient_split<<<(unsigned)(p.n * nb), kSplitThreads, 0, s_big>>>(p, rows, nb);
            k_orient_pick<<<(unsigned)((p.n + 127) / 128), 128, 0, s_big>>>(p);
        }
        if (csm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_desc_cell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
            if (e != cudaSuccess) return e;
        }
        k_desc_cell<<<(unsigned)(p.n * 16), kSplitThreads, csm, s_big>>>(p);
        k_desc_finalize<<<(unsigned)((p.n + 3) / 4), 128, 0, s_big>>>(p);
    }
    cudaError_t e = cudaGetLastError();
    if (forked) {
        cudaError_t j = cudaEventRecord(fork->join_ev[0], fork->aux[0]);
        if (j == cudaSuccess) j = cudaEventRecord(fork->join_ev[1], fork->aux[1]);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s, fork->join_ev[0], 0);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s, fork->join_ev[1], 0);
        if (e == cudaSuccess) e = j;
    }
    return e;
}

cudaError_t launch_diag_orient(int32_t* bins, uint32_t* weights, cudaStream_t s)
{
    k_diag_orient<<<(kLutBins + 255) / 256, 256, 0, s>>>(bins, weights);
    return cudaGetLastError();
}

}  // namespace lp
