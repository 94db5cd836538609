// Orientation and 128-d description of feature points (Sec. 2.3, Eq. 3-5)
// for sm_103a.
//
// One warp per feature point; four points per 128-thread CTA, heaviest scale
// first so that the long descriptors do not form the tail.  The warp copies
// the point's clamped neighbourhood (radius ceil(2*sqrt(2)*w_s) + 2) from the
// L2-resident intensity image into shared memory once; every tap afterwards is
// a shared-memory read.
//
// Orientation (integer, exact): 36-bin histogram over the upright
// (4 w_s + 1)^2 window of Eq. 5 gradients, weight round(65536*sqrt(a^2+b^2))
// computed with an integer square root, bin = 10-degree sector of
// atan2(b, a) (axes decided by sign; every other integer gradient lies more
// than 6e-5 bins from a sector edge, far above FP32 atan2 error).  Sums are
// 64-bit integer shared atomics, so the argmax (lowest bin on ties) is exact.
//
// Descriptor (FP32): the 4 w_s x 4 w_s grid turned by theta = (k + 0.5)*10
// degrees, bilinear taps, Eq. 5 gradient along the turned axes, 8 soft
// direction bins.  Lane 2c and 2c+1 own cell c and sum its samples in a private
// shared-memory slice (no atomics, fixed order, deterministic); the vector is
// L2-normalised, clamped at 0.2 and normalised again with warp reductions.
#include <cuda_bf16.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kWarps = 4;
constexpr int kHistBytes = 36 * 8;
constexpr int kAccStride = 9;                  // 8 bins + 1 pad word per lane
constexpr int kAccBytes = 32 * kAccStride * 4;

struct DescParams {
    const uint8_t* gray;
    int H, W, pitch;
    const uint32_t* kp;
    long long K;
    int nL;
    long long off[LP_MAX_SCALES + 1];
    int ws[LP_MAX_SCALES];
    int pr[LP_MAX_SCALES];
    float cs[36][2];       // cos, sin of (k + 0.5) * 10 degrees
    int upright;
    int warp_bytes;
    uint8_t* ori;
    float* desc;
    __nv_bfloat16* desc16;
    uint8_t* valid;
};

// 10-degree sector of the direction atan2(b, a) in [0, 360); (a, b) != 0.
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

struct PatchTap {
    const uint8_t* patch;
    int S, P;
    __device__ __forceinline__ float at(int r, int c) const { return (float)patch[(P + r) * S + P + c]; }
    __device__ __forceinline__ int iat(int r, int c) const { return patch[(P + r) * S + P + c]; }
};

struct GlobalTap {
    const uint8_t* g;
    int H, W, pitch, y, x;
    __device__ __forceinline__ int iat(int r, int c) const
    {
        const int yy = min(max(y + r, 0), H - 1), xx = min(max(x + c, 0), W - 1);
        return __ldg(g + (size_t)yy * pitch + xx);
    }
    __device__ __forceinline__ float at(int r, int c) const { return (float)iat(r, c); }
};

// Bilinear intensity at (row, col) offsets relative to the point.
template <class Tap>
__device__ __forceinline__ float bilinear(const Tap& t, float r, float c)
{
    const float r0 = floorf(r), c0 = floorf(c);
    const float fr = r - r0, fc = c - c0;
    const int y = (int)r0, x = (int)c0;
    const float v00 = t.at(y, x), v01 = t.at(y, x + 1), v10 = t.at(y + 1, x), v11 = t.at(y + 1, x + 1);
    const float top = v00 + fc * (v01 - v00);
    const float bot = v10 + fc * (v11 - v10);
    return top + fr * (bot - top);
}

template <class Tap>
__device__ __forceinline__ void describe_point(const DescParams& p, const Tap& tap, long long k, int ws,
                                               unsigned long long* hist, float* acc, int lane)
{
    const int R = 2 * ws;
    int best = 0;
    if (!p.upright) {
        for (int j = lane; j < 36; j += 32) hist[j] = 0ull;
        __syncwarp();
        const int n = 2 * R + 1;
        for (int e = lane; e < n * n; e += 32) {
            const int u = e / n - R, v = e - (e / n) * n - R;
            const int a = tap.iat(u + 1, v) - tap.iat(u - 1, v);
            const int b = tap.iat(u, v + 1) - tap.iat(u, v - 1);
            const int s = a * a + b * b;
            if (s) atomicAdd(&hist[orient_bin(a, b)], (unsigned long long)orient_weight(s));
        }
        __syncwarp();
        if (lane == 0) {
            unsigned long long bv = hist[0];
            for (int j = 1; j < 36; ++j)
                if (hist[j] > bv) { bv = hist[j]; best = j; }
        }
        best = __shfl_sync(0xFFFFFFFFu, best, 0);
    }
    const float c = p.upright ? 1.f : p.cs[best][0];
    const float s = p.upright ? 0.f : p.cs[best][1];

    float* mine = acc + lane * kAccStride;
#pragma unroll
    for (int q = 0; q < 8; ++q) mine[q] = 0.f;
    const int cell = lane >> 1, cr = cell >> 2, cc = cell & 3;
    const int u0 = -R + cr * ws, v0 = -R + cc * ws;
    int iu = 0, iv = lane & 1;
    while (iv >= ws) { iv -= ws; ++iu; }
    for (; iu < ws;) {
        const float fu = (float)(u0 + iu), fv = (float)(v0 + iv);
        const float dy = fu * c - fv * s;
        const float dx = fu * s + fv * c;
        const float a = bilinear(tap, dy + c, dx + s) - bilinear(tap, dy - c, dx - s);
        const float b = bilinear(tap, dy - s, dx + c) - bilinear(tap, dy + s, dx - c);
        const float m = sqrtf(a * a + b * b);
        if (m > 0.f) {
            float o = atan2f(b, a) * 1.27323954473516268615f;   // 8 / (2 pi)
            if (o < 0.f) o += 8.f;
            if (o >= 8.f) o -= 8.f;
            const int b0 = (int)o;
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
    const float n = sqrtf(ss);
    const bool ok = n > 0.f;
    float ss2 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = ok ? fminf(v[q] / n, 0.2f) : 0.f;
        ss2 += v[q] * v[q];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss2 += __shfl_xor_sync(0xFFFFFFFFu, ss2, o);
    const float n2 = sqrtf(ss2);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = ok ? v[q] / n2 : 0.f;
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

template <bool PATCH>
__global__ void __launch_bounds__(kWarps * 32) k_describe(const DescParams p)
{
    extern __shared__ __align__(16) uint8_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t* base = sm + warp * p.warp_bytes;
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(base);
    float* acc = reinterpret_cast<float*>(base + kHistBytes);
    const long long k = p.K - 1 - ((long long)blockIdx.x * kWarps + warp);
    if (k < 0) return;
    int l = 0;
    while (l + 1 < p.nL && k >= p.off[l + 1]) ++l;
    const int ws = p.ws[l];
    const uint32_t id = __ldg(p.kp + k);
    const int y = (int)(id / (uint32_t)p.W), x = (int)(id - (uint32_t)y * (uint32_t)p.W);
    if (PATCH) {
        uint8_t* patch = base + kHistBytes + kAccBytes;
        const int P = p.pr[l], S = 2 * P + 1;
        for (int r = 0; r < S; ++r) {
            const int yy = min(max(y - P + r, 0), p.H - 1);
            const uint8_t* row = p.gray + (size_t)yy * p.pitch;
            for (int c = lane; c < S; c += 32) {
                const int xx = min(max(x - P + c, 0), p.W - 1);
                patch[r * S + c] = __ldg(row + xx);
            }
        }
        __syncwarp();
        PatchTap t{patch, S, P};
        describe_point(p, t, k, ws, hist, acc, lane);
    } else {
        GlobalTap t{p.gray, p.H, p.W, p.pitch, y, x};
        describe_point(p, t, k, ws, hist, acc, lane);
    }
}

__global__ void k_diag_orient(int32_t* bins, uint32_t* weights)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (bins && i < 511 * 511) {
        const int a = i / 511 - 255, b = i % 511 - 255;
        bins[i] = (a == 0 && b == 0) ? 0 : orient_bin(a, b);
    }
    if (weights && i <= 2 * 255 * 255) weights[i] = orient_weight(i);
}

}  // namespace

cudaError_t launch_describe(const uint8_t* gray, int H, int W, int pitch, const uint32_t* kp,
                            const ScaleTable& st, int upright, uint8_t* ori, float* desc,
                            uint16_t* desc_bf16, uint8_t* valid, cudaStream_t s)
{
    DescParams p;
    p.gray = gray; p.H = H; p.W = W; p.pitch = pitch; p.kp = kp; p.K = st.off[st.nL]; p.nL = st.nL;
    int pmax = 0;
    for (int l = 0; l <= st.nL; ++l) p.off[l] = st.off[l];
    for (int l = 0; l < st.nL; ++l) {
        p.ws[l] = st.ws[l];
        p.pr[l] = st.pr[l];
        pmax = pmax > st.pr[l] ? pmax : st.pr[l];
    }
    for (int k = 0; k < 36; ++k) {
        const double th = (k + 0.5) * 10.0 * 3.14159265358979323846 / 180.0;
        p.cs[k][0] = (float)cos(th);
        p.cs[k][1] = (float)sin(th);
    }
    p.upright = upright;
    p.ori = ori; p.desc = desc; p.desc16 = reinterpret_cast<__nv_bfloat16*>(desc_bf16); p.valid = valid;
    if (p.K == 0) return cudaSuccess;
    const int S = 2 * pmax + 1;
    const bool patch = (size_t)S * S <= 12 * 1024;
    p.warp_bytes = kHistBytes + kAccBytes + (patch ? ((S * S + 15) / 16) * 16 : 0);
    const size_t smem = (size_t)kWarps * p.warp_bytes;
    const unsigned grid = (unsigned)((p.K + kWarps - 1) / kWarps);
    if (patch) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_describe<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_describe<true><<<grid, kWarps * 32, smem, s>>>(p);
    } else {
        k_describe<false><<<grid, kWarps * 32, smem, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_diag_orient(int32_t* bins, uint32_t* weights, cudaStream_t s)
{
    k_diag_orient<<<(511 * 511 + 255) / 256, 256, 0, s>>>(bins, weights);
    return cudaGetLastError();
}

}  // namespace lp
