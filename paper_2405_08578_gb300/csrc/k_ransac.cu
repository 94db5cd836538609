// Matched-pair compaction and RANSAC homography estimation (Sec. 2.4-2.5,
// Eq. 7) for sm_103a.
//
//  k_compact      one CTA: stable prefix sum of accepted rows -> (xA, yA, xB, yB)
//  k_ransac_hyp   one thread per iteration t: Philox4x32-10 draw of 4 distinct
//                 matches, collinearity test, Hartley-normalised 4-point DLT
//                 solved in FP64 (8x8 Gaussian elimination, partial pivoting)
//  k_ransac_score one CTA per hypothesis: FP32 reprojection errors; counts of
//                 points certainly inside (e^2 < t^2 - eps) and possibly inside
//                 (e^2 < t^2 + eps)
//  k_ransac_select one CTA: the largest certain count c*; every hypothesis whose
//                 possible count reaches c* and that has points in the band is
//                 recounted in FP64, so the winner (most inliers, earliest t) is
//                 the FP64 winner
//  k_ransac_refit one CTA: FP64 inlier mask of the winner, Hartley
//                 normalisation, A^T A (9x9) by block reduction, cyclic Jacobi
//                 smallest eigenvector, denormalisation, final FP64 mask.
#include <math.h>

#include <algorithm>

#include "lp_internal.cuh"

namespace lp {
namespace {

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; each round
// multiplies words 0 and 2 by fixed odd constants (high/low halves), xors the
// high halves with words 1/3 and the round key; the key advances by the Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__global__ void k_diag_philox(const uint4* ctr, long long n, uint32_t k0, uint32_t k1, uint4* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox(ctr[i], k0, k1);
}

// ---------------------------------------------------------------- compaction
constexpr int kCompactThreads = 1024;

__global__ void __launch_bounds__(kCompactThreads)
k_compact(const uint32_t* kpA, int WA, const uint32_t* kpB, int WB, const int32_t* match, long long NA,
          float4* pts, int32_t* rows, int32_t* dM)
{
    __shared__ int warp_tot[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long chunk = (NA + kCompactThreads - 1) / kCompactThreads;
    const long long b = tid * chunk, e = min(NA, b + chunk);
    int cnt = 0;
    for (long long i = b; i < e; ++i) cnt += match[i] >= 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += v;
        }
        warp_tot[lane] = wi - w;   // exclusive
        if (lane == 31) *dM = wi;
    }
    __syncthreads();
    int pos = warp_tot[warp] + incl - cnt;
    for (long long i = b; i < e; ++i) {
        const int j = match[i];
        if (j < 0) continue;
        const uint32_t ia = kpA[i], ib = kpB[j];
        const uint32_t ya = ia / (uint32_t)WA, yb = ib / (uint32_t)WB;
        pts[pos] = make_float4((float)(ia - ya * WA), (float)ya, (float)(ib - yb * WB), (float)yb);
        if (rows) rows[pos] = (int32_t)i;
        ++pos;
    }
}

// ---------------------------------------------------------------- FP64 model
__device__ __forceinline__ long long m_count(const int32_t* dM, long long M_cap)
{
    if (!dM) return M_cap;
    const long long m = *dM;
    return m < 0 ? 0 : (m > M_cap ? M_cap : m);
}

// |cross(q - p, r - p)| small relative to the spread: the three are on a line.
__device__ __forceinline__ bool collinear(double px, double py, double qx, double qy, double rx, double ry)
{
    const double ux = qx - px, uy = qy - py, vx = rx - px, vy = ry - py;
    return fabs(ux * vy - uy * vx) <= 1e-9 * (ux * ux + uy * uy + vx * vx + vy * vy);
}

struct Norm2D { double s, cx, cy; };

// centroid to the origin, mean distance sqrt(2)
__device__ bool hartley4(const double* x, const double* y, Norm2D& n)
{
    double cx = 0, cy = 0;
    for (int i = 0; i < 4; ++i) { cx += x[i]; cy += y[i]; }
    cx /= 4; cy /= 4;
    double md = 0;
    for (int i = 0; i < 4; ++i) md += sqrt((x[i] - cx) * (x[i] - cx) + (y[i] - cy) * (y[i] - cy));
    md /= 4;
    if (!(md > 0)) return false;
    n.s = sqrt(2.0) / md; n.cx = cx; n.cy = cy;
    return true;
}

// H = Tb^-1 * Hn * Ta with T = [[s, 0, -s cx], [0, s, -s cy], [0, 0, 1]], h33 -> 1.
__device__ bool denorm(const Norm2D& na, const Norm2D& nb, const double* hn, double* H)
{
    // Hn * Ta
    double t[9];
    for (int r = 0; r < 3; ++r) {
        t[3 * r + 0] = hn[3 * r + 0] * na.s;
        t[3 * r + 1] = hn[3 * r + 1] * na.s;
        t[3 * r + 2] = hn[3 * r + 2] - hn[3 * r + 0] * na.s * na.cx - hn[3 * r + 1] * na.s * na.cy;
    }
    // Tb^-1 = [[1/s, 0, cx], [0, 1/s, cy], [0, 0, 1]]
    const double is = 1.0 / nb.s;
    for (int c = 0; c < 3; ++c) {
        H[0 + c] = is * t[0 + c] + nb.cx * t[6 + c];
        H[3 + c] = is * t[3 + c] + nb.cy * t[6 + c];
        H[6 + c] = t[6 + c];
    }
    double mx = 0;
    for (int i = 0; i < 9; ++i) mx = fmax(mx, fabs(H[i]));
    if (!(fabs(H[8]) > 1e-12 * mx)) return false;
    const double h = H[8];
    for (int i = 0; i < 9; ++i) H[i] /= h;
    return true;
}

// prefix == nullptr: uniform draw; otherwise word w picks the match whose
// interval of the inclusive prefix sums of integer weights contains
// floor(w * total / 2^32) (probability proportional to the weight).
__global__ void k_ransac_hyp(const float4* pts, long long M_cap, const int32_t* dM, int T, uint32_t k0, uint32_t k1,
                             const unsigned long long* prefix, const int32_t* skip, double* Hs, int8_t* hok)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T || (skip && *skip)) return;
    hok[t] = 0;
    const long long M = m_count(dM, M_cap);
    if (M < 4) return;
    int idx[4];
    int n = 0;
    uint4 blk = make_uint4(0, 0, 0, 0);
    for (int j = 0; j < 64 && n < 4; ++j) {
        if ((j & 3) == 0) blk = philox(make_uint4((uint32_t)t, (uint32_t)(j >> 2), 0u, 0u), k0, k1);
        const uint32_t w = (j & 3) == 0 ? blk.x : (j & 3) == 1 ? blk.y : (j & 3) == 2 ? blk.z : blk.w;
        int i;
        if (!prefix) {
            i = (int)(((unsigned long long)w * (unsigned long long)M) >> 32);
        } else {
            const unsigned long long total = prefix[M - 1];
            const unsigned long long target = __umul64hi((unsigned long long)w << 32, total);
            long long lo = 0, hi = M - 1;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (prefix[mid] > target) hi = mid; else lo = mid + 1;
            }
            i = (int)lo;
        }
        bool dup = false;
        for (int q = 0; q < n; ++q) dup |= idx[q] == i;
        if (!dup) idx[n++] = i;
    }
    if (n < 4) return;
    double xa[4], ya[4], xb[4], yb[4];
    for (int q = 0; q < 4; ++q) {
        const float4 p = pts[idx[q]];
        xa[q] = p.x; ya[q] = p.y; xb[q] = p.z; yb[q] = p.w;
    }
    for (int a = 0; a < 4; ++a) {
        const int i0 = (a + 1) & 3, i1 = (a + 2) & 3, i2 = (a + 3) & 3;
        if (collinear(xa[i0], ya[i0], xa[i1], ya[i1], xa[i2], ya[i2])) return;
        if (collinear(xb[i0], yb[i0], xb[i1], yb[i1], xb[i2], yb[i2])) return;
    }
    Norm2D na, nb;
    if (!hartley4(xa, ya, na) || !hartley4(xb, yb, nb)) return;
    double A[8][9];
    for (int q = 0; q < 4; ++q) {
        const double x = na.s * (xa[q] - na.cx), y = na.s * (ya[q] - na.cy);
        const double u = nb.s * (xb[q] - nb.cx), v = nb.s * (yb[q] - nb.cy);
        double* r0 = A[2 * q];
        double* r1 = A[2 * q + 1];
        r0[0] = x; r0[1] = y; r0[2] = 1; r0[3] = 0; r0[4] = 0; r0[5] = 0; r0[6] = -x * u; r0[7] = -y * u; r0[8] = u;
        r1[0] = 0; r1[1] = 0; r1[2] = 0; r1[3] = x; r1[4] = y; r1[5] = 1; r1[6] = -x * v; r1[7] = -y * v; r1[8] = v;
    }
    for (int c = 0; c < 8; ++c) {
        int p = c;
        for (int r = c + 1; r < 8; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (!(fabs(A[p][c]) > 1e-10)) return;
        if (p != c)
            for (int j = 0; j < 9; ++j) { const double tmp = A[c][j]; A[c][j] = A[p][j]; A[p][j] = tmp; }
        const double ip = 1.0 / A[c][c];
        for (int r = c + 1; r < 8; ++r) {
            const double f = A[r][c] * ip;
            for (int j = c; j < 9; ++j) A[r][j] -= f * A[c][j];
        }
    }
    double h[9];
    for (int r = 7; r >= 0; --r) {
        double s = A[r][8];
        for (int j = r + 1; j < 8; ++j) s -= A[r][j] * h[j];
        h[r] = s / A[r][r];
    }
    h[8] = 1.0;
    double H[9];
    if (!denorm(na, nb, h, H)) return;
    for (int i = 0; i < 9; ++i) Hs[9ll * t + i] = H[i];
    hok[t] = 1;
}

// ---------------------------------------------------------------- scoring
constexpr int kScoreThreads = 256;

__device__ __forceinline__ int block_sum(int v, int* red)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

__global__ void __launch_bounds__(kScoreThreads)
k_ransac_score(const float4* pts, long long M_cap, const int32_t* dM, const double* Hs, const int8_t* hok,
               float t2, float eps, const int32_t* skip, int32_t* lo, int32_t* hi)
{
    __shared__ int red[32];
    const int t = blockIdx.x;
    if ((skip && *skip) || !hok[t]) {
        if (threadIdx.x == 0) { lo[t] = -1; hi[t] = -1; }
        return;
    }
    const long long M = m_count(dM, M_cap);
    float h[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = (float)Hs[9ll * t + i];
    int clo = 0, chi = 0;
    for (long long i = threadIdx.x; i < M; i += kScoreThreads) {
        const float4 p = pts[i];
        // e^2 < t^2  <=>  |(u, v) - w p_B|^2 < t^2 w^2  for w > 0 (no division)
        const float w = fmaf(h[6], p.x, fmaf(h[7], p.y, h[8]));
        if (w > 0.f) {
            const float du = fmaf(-p.z, w, fmaf(h[0], p.x, fmaf(h[1], p.y, h[2])));
            const float dv = fmaf(-p.w, w, fmaf(h[3], p.x, fmaf(h[4], p.y, h[5])));
            const float d2 = du * du + dv * dv, w2 = w * w;
            clo += d2 < (t2 - eps) * w2;
            chi += d2 < (t2 + eps) * w2;
        }
    }
    clo = block_sum(clo, red);
    chi = block_sum(chi, red);
    if (threadIdx.x == 0) { lo[t] = clo; hi[t] = chi; }
}

// FP64 inlier test of one correspondence (Eq. 7, one-sided error in B):
// |pi(H p_A) - p_B|^2 < t^2, written for w > 0 as |(u, v) - w p_B|^2 < t^2 w^2,
// which needs no division.
__device__ __forceinline__ bool inlier64(const double* H, const float4& p, double t2)
{
    const double x = p.x, y = p.y;
    const double w = H[6] * x + H[7] * y + H[8];
    if (!(w > 0)) return false;
    const double du = H[0] * x + H[1] * y + H[2] - (double)p.z * w;
    const double dv = H[3] * x + H[4] * y + H[5] - (double)p.w * w;
    return du * du + dv * dv < t2 * (w * w);
}

constexpr int kSelThreads = 1024;

__global__ void __launch_bounds__(kSelThreads)
k_ransac_select(const float4* pts, long long M_cap, const int32_t* dM, int T, const double* Hs,
                const int32_t* lo, const int32_t* hi, double t2, const int32_t* skip, int t_off, int32_t* best_out)
{
    if (skip && *skip) return;
    __shared__ int red[32];
    __shared__ unsigned long long bestkey;
    __shared__ int cand[kSelThreads];
    __shared__ int ncand;
    const long long M = m_count(dM, M_cap);
    int cmax = -1;
    for (int t = threadIdx.x; t < T; t += kSelThreads) cmax = max(cmax, lo[t]);
#pragma unroll
    for (int o = 16; o; o >>= 1) cmax = max(cmax, __shfl_xor_sync(0xFFFFFFFFu, cmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cmax;
    if (threadIdx.x == 0) { bestkey = 0ull; ncand = 0; }
    __syncthreads();
    cmax = -1;
    for (int w = 0; w < kSelThreads / 32; ++w) cmax = max(cmax, red[w]);
    if (cmax < 0) {
        if (threadIdx.x == 0) { best_out[0] = -1; best_out[1] = -1; }
        return;
    }
    // key = (count + 1) << 32 | (0xFFFFFFFF - t): the max key is the most
    // inliers at the earliest iteration.  Iterations are visited in chunks of
    // one CTA width; in-band candidates of a chunk are recounted in FP64.
    for (int t0 = 0; t0 < T; t0 += kSelThreads) {
        const int t = t0 + threadIdx.x;
        if (t < T) {
            const int l = lo[t], h = hi[t];
            if (l >= 0 && h >= cmax) {
                if (h == l) {
                    atomicMax(&bestkey, ((unsigned long long)(l + 1) << 32) | (0xFFFFFFFFull - (unsigned)t));
                } else {
                    cand[atomicAdd(&ncand, 1)] = t;
                }
            }
        }
        __syncthreads();
        const int nc = ncand;
        for (int k = 0; k < nc; ++k) {
            const int tc = cand[k];
            double H[9];
            for (int i = 0; i < 9; ++i) H[i] = Hs[9ll * tc + i];
            int n = 0;
            for (long long i = threadIdx.x; i < M; i += kSelThreads) n += inlier64(H, pts[i], t2);
            n = block_sum(n, red);
            if (threadIdx.x == 0)
                atomicMax(&bestkey, ((unsigned long long)(n + 1) << 32) | (0xFFFFFFFFull - (unsigned)tc));
        }
        __syncthreads();
        if (threadIdx.x == 0) ncand = 0;
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        best_out[0] = t_off + (int)(0xFFFFFFFFull - (bestkey & 0xFFFFFFFFull));
        best_out[1] = (int)(bestkey >> 32) - 1;
    }
}

// Stop test of the guided phase.  w = (prior weight of the guided winner's
// FP64 inliers) / (total weight) is the chance that one guided draw is an
// inlier; the phase stops when (1 - w^4)^Tg <= 0.01, the standard bound
// T >= log(0.01) / log(1 - w^4) without logarithms.  Every operation is a
// single IEEE-rounded one (no contraction), powers by binary exponentiation.
// flags[2] = stop, flags[3] = iterations used.
__global__ void __launch_bounds__(kSelThreads)
k_guided_decide(const float4* pts, long long M_cap, const int32_t* dM, const double* Hs,
                const unsigned long long* prefix, int Tg, int T, double t2, int32_t* flags)
{
    __shared__ unsigned long long part[kSelThreads / 32];
    const int tb = flags[0];
    const long long M = m_count(dM, M_cap);
    if (tb < 0 || M < 4) {
        if (threadIdx.x == 0) { flags[2] = 0; flags[3] = Tg + T; }
        return;
    }
    double H[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) H[i] = Hs[9ll * tb + i];
    unsigned long long sw = 0;
    for (long long i = threadIdx.x; i < M; i += kSelThreads)
        if (inlier64(H, pts[i], t2)) sw += prefix[i] - (i ? prefix[i - 1] : 0ull);
#pragma unroll
    for (int o = 16; o; o >>= 1) sw += __shfl_xor_sync(0xFFFFFFFFu, sw, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sw;
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned long long s_in = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) s_in += part[w];
    const double w = __ddiv_rn((double)s_in, (double)prefix[M - 1]);
    const double w2 = __dmul_rn(w, w);
    double b = __dsub_rn(1.0, __dmul_rn(w2, w2)), r = 1.0;
    for (int e = Tg; e; e >>= 1) {
        if (e & 1) r = __dmul_rn(r, b);
        b = __dmul_rn(b, b);
    }
    const int stop = r <= 0.01;
    flags[2] = stop;
    flags[3] = stop ? Tg : Tg + T;
}

// ---------------------------------------------------------------- refit
// Least-squares refit of the winner's inliers (Eq. 7), spread over kRefitCTAs
// CTAs.  Each pass writes per-CTA partial sums; the next pass reduces them in
// a fixed order, so results do not depend on scheduling.
constexpr int kRefitThreads = 256;
constexpr int kRefitWarps = kRefitThreads / 32;
constexpr int kRefitCTAs = 32;
constexpr int kPartStride = 64;   // doubles per CTA partial row

struct RefitWS {
    double* part;     // [kRefitCTAs][kPartStride]
    double* Hf;       // [9] refitted homography
};

template <int N>
__device__ void block_sum_n(double* v, double (*part)[N], double* tot)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < N; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        v[q] = x;
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) part[warp][q] = v[q];
    __syncthreads();
    for (int q = threadIdx.x; q < N; q += kRefitThreads) {
        double s = 0;
        for (int w = 0; w < kRefitWarps; ++w) s += part[w][q];
        tot[q] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void cta_range(long long M, long long& b, long long& e)
{
    const long long chunk = (M + kRefitCTAs - 1) / kRefitCTAs;
    b = min(M, (long long)blockIdx.x * chunk);
    e = min(M, b + chunk);
}

// fixed-order sum of the CTAs' partials, columns [c0, c0 + n)
__device__ void sum_parts(const double* part, int c0, int n, double* out)
{
    for (int q = 0; q < n; ++q) {
        double s = 0;
        for (int c = 0; c < kRefitCTAs; ++c) s += part[c * kPartStride + c0 + q];
        out[q] = s;
    }
}

// pass 1: inlier mask of the winning hypothesis, count and coordinate sums
__global__ void __launch_bounds__(kRefitThreads)
k_refit_p1(const float4* pts, long long M_cap, const int32_t* dM, const double* Hs, const int32_t* best_in,
           double t2, uint8_t* inl, RefitWS ws)
{
    __shared__ double part[kRefitWarps][5];
    __shared__ double tot[5];
    const int best = *best_in;
    if (best < 0) return;
    const long long M = m_count(dM, M_cap);
    long long b, e;
    cta_range(M, b, e);
    double Hb[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Hb[i] = Hs[9ll * best + i];
    double v5[5] = {0, 0, 0, 0, 0};
    for (long long i = b + threadIdx.x; i < e; i += kRefitThreads) {
        const float4 p = pts[i];
        const bool in = inlier64(Hb, p, t2);
        inl[i] = in;
        if (in) { v5[0] += 1; v5[1] += p.x; v5[2] += p.y; v5[3] += p.z; v5[4] += p.w; }
    }
    block_sum_n<5>(v5, part, tot);
    if (threadIdx.x < 5) ws.part[blockIdx.x * kPartStride + threadIdx.x] = tot[threadIdx.x];
}

// pass 2: mean distances to the centroids (Hartley normalisation)
__global__ void __launch_bounds__(kRefitThreads)
k_refit_p2(const float4* pts, long long M_cap, const int32_t* dM, const int32_t* best_in, const uint8_t* inl,
           RefitWS ws)
{
    __shared__ double part[kRefitWarps][2];
    __shared__ double tot[2];
    __shared__ double c5[5];
    if (*best_in < 0) return;
    const long long M = m_count(dM, M_cap);
    if (threadIdx.x == 0) sum_parts(ws.part, 0, 5, c5);
    __syncthreads();
    const double n = c5[0];
    const double cxa = c5[1] / n, cya = c5[2] / n, cxb = c5[3] / n, cyb = c5[4] / n;
    long long b, e;
    cta_range(M, b, e);
    double v2[2] = {0, 0};
    for (long long i = b + threadIdx.x; i < e; i += kRefitThreads) {
        if (!inl[i]) continue;
        const float4 p = pts[i];
        v2[0] += sqrt((p.x - cxa) * (p.x - cxa) + (p.y - cya) * (p.y - cya));
        v2[1] += sqrt((p.z - cxb) * (p.z - cxb) + (p.w - cyb) * (p.w - cyb));
    }
    block_sum_n<2>(v2, part, tot);
    if (threadIdx.x < 2) ws.part[blockIdx.x * kPartStride + 5 + threadIdx.x] = tot[threadIdx.x];
}

__device__ void norms_from_parts(const double* part, Norm2D& na, Norm2D& nb, double& n, bool& good)
{
    double c7[7];
    sum_parts(part, 0, 7, c7);
    n = c7[0];
    const double cxa = c7[1] / n, cya = c7[2] / n, cxb = c7[3] / n, cyb = c7[4] / n;
    const double da = c7[5] / n, db = c7[6] / n;
    na = Norm2D{sqrt(2.0) / da, cxa, cya};
    nb = Norm2D{sqrt(2.0) / db, cxb, cyb};
    good = n >= 4 && da > 0 && db > 0;
}

// pass 3: upper triangle of A^T A (45 entries) in normalised coordinates
__global__ void __launch_bounds__(kRefitThreads)
k_refit_p3(const float4* pts, long long M_cap, const int32_t* dM, const int32_t* best_in, const uint8_t* inl,
           RefitWS ws)
{
    __shared__ double part[kRefitWarps][45];
    __shared__ double tot[45];
    __shared__ double nrm[6];
    __shared__ int good_s;
    if (*best_in < 0) return;
    const long long M = m_count(dM, M_cap);
    if (threadIdx.x == 0) {
        Norm2D na, nb;
        double n;
        bool good;
        norms_from_parts(ws.part, na, nb, n, good);
        nrm[0] = na.s; nrm[1] = na.cx; nrm[2] = na.cy; nrm[3] = nb.s; nrm[4] = nb.cx; nrm[5] = nb.cy;
        good_s = good;
    }
    __syncthreads();
    const Norm2D na{nrm[0], nrm[1], nrm[2]}, nb{nrm[3], nrm[4], nrm[5]};
    long long b, e;
    cta_range(M, b, e);
    double acc[45];
#pragma unroll
    for (int q = 0; q < 45; ++q) acc[q] = 0;
    if (good_s) {
        for (long long i = b + threadIdx.x; i < e; i += kRefitThreads) {
            if (!inl[i]) continue;
            const float4 p = pts[i];
            const double x = na.s * (p.x - na.cx), y = na.s * (p.y - na.cy);
            const double u = nb.s * (p.z - nb.cx), v = nb.s * (p.w - nb.cy);
            const double r0[9] = {-x, -y, -1, 0, 0, 0, x * u, y * u, u};
            const double r1[9] = {0, 0, 0, -x, -y, -1, x * v, y * v, v};
            int q = 0;
#pragma unroll
            for (int j = 0; j < 9; ++j)
#pragma unroll
                for (int k = j; k < 9; ++k) acc[q++] += r0[j] * r0[k] + r1[j] * r1[k];
        }
    }
    block_sum_n<45>(acc, part, tot);
    if (threadIdx.x < 45) ws.part[blockIdx.x * kPartStride + 8 + threadIdx.x] = tot[threadIdx.x];
}

// Smallest eigenvector of the symmetric positive semi-definite 9x9 matrix S by
// shifted inverse iteration: Cholesky of S + mu I (mu = 1e-12 trace S), then
// repeated solves.  The shift keeps the factorisation positive definite for
// exact data and leaves the eigenvectors unchanged.  Returns false if the
// factorisation fails.
__device__ bool smallest_eigvec9(const double (*S)[9], double* h)
{
    double L[9][9];
    double tr = 0;
    for (int i = 0; i < 9; ++i) tr += S[i][i];
    const double mu = 1e-12 * tr;
    double inv_d[9];
    for (int j = 0; j < 9; ++j) {
        double d = S[j][j] + mu;
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0)) return false;
        L[j][j] = sqrt(d);
        inv_d[j] = 1.0 / L[j][j];
        for (int i = j + 1; i < 9; ++i) {
            double sum = S[i][j];
            for (int k = 0; k < j; ++k) sum -= L[i][k] * L[j][k];
            L[i][j] = sum * inv_d[j];
        }
    }
    double x[9];
    for (int i = 0; i < 9; ++i) x[i] = 1.0;
    for (int it = 0; it < 24; ++it) {
        double y[9];
        for (int i = 0; i < 9; ++i) {   // L y = x
            double sum = x[i];
            for (int k = 0; k < i; ++k) sum -= L[i][k] * y[k];
            y[i] = sum * inv_d[i];
        }
        double z[9];
        for (int i = 8; i >= 0; --i) {  // L^T z = y
            double sum = y[i];
            for (int k = i + 1; k < 9; ++k) sum -= L[k][i] * z[k];
            z[i] = sum * inv_d[i];
        }
        double nz = 0;
        for (int i = 0; i < 9; ++i) nz += z[i] * z[i];
        const double inv = 1.0 / sqrt(nz);
        double diff = 0;
        // align the sign with the previous iterate before comparing
        double dot = 0;
        for (int i = 0; i < 9; ++i) dot += z[i] * x[i];
        const double sg = dot < 0 ? -inv : inv;
        for (int i = 0; i < 9; ++i) {
            const double xn = z[i] * sg;
            diff = fmax(diff, fabs(xn - x[i]));
            x[i] = xn;
        }
        if (it >= 2 && diff < 1e-15) break;
    }
    for (int i = 0; i < 9; ++i) h[i] = x[i];
    return true;
}

__global__ void k_refit_solve(const double* Hs, const int32_t* best_in, RefitWS ws, double* Hout, int32_t* n_in,
                              int32_t* best_t)
{
    if (threadIdx.x != 0) return;
    const int best = *best_in;
    if (best_t) *best_t = best;
    *n_in = 0;
    if (best < 0) {
        for (int i = 0; i < 9; ++i) { Hout[i] = 0.0; ws.Hf[i] = 0.0; }
        return;
    }
    Norm2D na, nb;
    double n;
    bool good;
    norms_from_parts(ws.part, na, nb, n, good);
    double H[9];
    bool ok = good;
    if (ok) {
        double t[45];
        sum_parts(ws.part, 8, 45, t);
        double S[9][9];
        int q = 0;
        for (int j = 0; j < 9; ++j)
            for (int k = j; k < 9; ++k) { S[j][k] = t[q]; S[k][j] = t[q]; ++q; }
        double h[9];
        ok = smallest_eigvec9(S, h) && denorm(na, nb, h, H);
    }
    for (int i = 0; i < 9; ++i) {
        const double v = ok ? H[i] : Hs[9ll * best + i];
        ws.Hf[i] = v;
        Hout[i] = v;
    }
}

// final inlier set of the refitted H
__global__ void __launch_bounds__(kRefitThreads)
k_refit_final(const float4* pts, long long M_cap, const int32_t* dM, RefitWS ws, double t2, uint8_t* inl,
              int32_t* n_in)
{
    __shared__ int red[kRefitWarps];
    const long long M = m_count(dM, M_cap);
    double H[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) H[i] = ws.Hf[i];
    const bool have = H[8] != 0.0;
    const long long chunk = (M_cap + gridDim.x - 1) / gridDim.x;
    const long long b = min(M_cap, (long long)blockIdx.x * chunk), e = min(M_cap, b + chunk);
    int n = 0;
    for (long long i = b + threadIdx.x; i < e; i += kRefitThreads) {
        const bool in = have && i < M && inlier64(H, pts[i], t2);
        inl[i] = in;
        n += in;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kRefitWarps; ++w) s += red[w];
        if (s) atomicAdd(n_in, s);
    }
}

}  // namespace

cudaError_t launch_compact(const uint32_t* kpA, int WA, const uint32_t* kpB, int WB, const int32_t* match,
                           int64_t NA, float* pts, int32_t* rows, int32_t* d_M, cudaStream_t s)
{
    k_compact<<<1, kCompactThreads, 0, s>>>(kpA, WA, kpB, WB, match, NA, reinterpret_cast<float4*>(pts), rows, d_M);
    return cudaGetLastError();
}

namespace {

struct RansacWS {
    double* Hs;       // [Ttot][9]
    int32_t* lo;      // [Ttot] certain FP32 counts (-1: no hypothesis)
    int32_t* hi;      // [Ttot] possible FP32 counts
    int32_t* flags;   // [4]: winner t, winner count, guided stop, iterations used
    int8_t* hok;      // [Ttot]
    RefitWS rw;
};

RansacWS carve(void* ws, int Ttot)
{
    RansacWS r;
    uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) & ~uintptr_t(255));
    r.Hs = reinterpret_cast<double*>(w);
    r.lo = reinterpret_cast<int32_t*>(r.Hs + 9ll * Ttot);
    r.hi = r.lo + Ttot;
    r.flags = r.hi + Ttot;
    r.hok = reinterpret_cast<int8_t*>(r.flags + 4);
    r.rw.part = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(r.hok + Ttot) + 255) & ~uintptr_t(255));
    r.rw.Hf = r.rw.part + kRefitCTAs * kPartStride + 1;
    return r;
}

void refit_launch(const float4* p4, int64_t M_cap, const int32_t* d_M, double t2, const RansacWS& w, double* H,
                  uint8_t* inlier, int32_t* n_in, int32_t* best_t, cudaStream_t s)
{
    k_refit_p1<<<kRefitCTAs, kRefitThreads, 0, s>>>(p4, M_cap, d_M, w.Hs, w.flags, t2, inlier, w.rw);
    k_refit_p2<<<kRefitCTAs, kRefitThreads, 0, s>>>(p4, M_cap, d_M, w.flags, inlier, w.rw);
    k_refit_p3<<<kRefitCTAs, kRefitThreads, 0, s>>>(p4, M_cap, d_M, w.flags, inlier, w.rw);
    k_refit_solve<<<1, 32, 0, s>>>(w.Hs, w.flags, w.rw, H, n_in, best_t);
    const unsigned gfin = (unsigned)std::max<long long>(1, std::min<long long>(kRefitCTAs, (M_cap + 1023) / 1024));
    k_refit_final<<<gfin, kRefitThreads, 0, s>>>(p4, M_cap, d_M, w.rw, t2, inlier, n_in);
}

// One batch of T hypotheses at rows [t_off, t_off + T) of the workspace,
// Philox counters 0..T-1; skipped entirely while *skip is non-zero.
void hyp_batch(const float4* p4, int64_t M_cap, const int32_t* d_M, const unsigned long long* prefix, int T,
               int t_off, uint32_t k0, uint32_t k1, float t2f, float eps, double t2, const int32_t* skip,
               const RansacWS& w, cudaStream_t s)
{
    k_ransac_hyp<<<(T + 15) / 16, 16, 0, s>>>(p4, M_cap, d_M, T, k0, k1, prefix, skip, w.Hs + 9ll * t_off,
                                              w.hok + t_off);
    k_ransac_score<<<T, kScoreThreads, 0, s>>>(p4, M_cap, d_M, w.Hs + 9ll * t_off, w.hok + t_off, t2f, eps, skip,
                                               w.lo + t_off, w.hi + t_off);
    k_ransac_select<<<1, kSelThreads, 0, s>>>(p4, M_cap, d_M, T, w.Hs + 9ll * t_off, w.lo + t_off, w.hi + t_off, t2,
                                              skip, t_off, w.flags);
}

}  // namespace

// Ttot = the number of hypotheses of one call (T, or Tg + T with a prior)
size_t ransac_workspace(int64_t M_cap, int Ttot)
{
    (void)M_cap;
    return 256 + (size_t)Ttot * (9 * sizeof(double) + 2 * sizeof(int32_t) + 1) + 256 +
           sizeof(double) * (kRefitCTAs * kPartStride + 16) + 256;
}

cudaError_t launch_ransac(const float* pts, int64_t M_cap, const int32_t* d_M, int T, float thresh,
                          uint64_t seed, uint32_t pair_id, double* H, uint8_t* inlier, int32_t* n_in,
                          int32_t* best_t, void* ws, size_t ws_bytes, int32_t* status, cudaStream_t s)
{
    (void)status;
    if (ws_bytes < ransac_workspace(M_cap, T)) return cudaErrorInvalidValue;
    const RansacWS w = carve(ws, T);
    const float4* p4 = reinterpret_cast<const float4*>(pts);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ pair_id;
    const double t2 = (double)thresh * (double)thresh;
    const float t2f = (float)t2;
    const float eps = fmaxf(0.05f, 0.01f * t2f);
    hyp_batch(p4, M_cap, d_M, nullptr, T, 0, k0, k1, t2f, eps, t2, nullptr, w, s);
    refit_launch(p4, M_cap, d_M, t2, w, H, inlier, n_in, best_t, s);
    return cudaGetLastError();
}

// Guided phase (Tg hypotheses drawn by the prior's prefix sums), the stop test,
// then the uniform fallback (T hypotheses, the plain RANSAC stream), skipped on
// the device when the guided phase stopped.  Hypothesis rows: guided [0, Tg),
// uniform [Tg, Tg + T).
cudaError_t launch_ransac_prior(const float* pts, int64_t M_cap, const int32_t* d_M, const unsigned long long* prefix,
                                int Tg, int T, float thresh, uint64_t seed, uint32_t pair_id, double* H,
                                uint8_t* inlier, int32_t* n_in, int32_t* best_t, int32_t* iters, void* ws,
                                size_t ws_bytes, cudaStream_t s)
{
    if (ws_bytes < ransac_workspace(M_cap, Tg + T)) return cudaErrorInvalidValue;
    const RansacWS w = carve(ws, Tg + T);
    const float4* p4 = reinterpret_cast<const float4*>(pts);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ pair_id;
    const double t2 = (double)thresh * (double)thresh;
    const float t2f = (float)t2;
    const float eps = fmaxf(0.05f, 0.01f * t2f);
    hyp_batch(p4, M_cap, d_M, prefix, Tg, 0, k0, k1, t2f, eps, t2, nullptr, w, s);
    k_guided_decide<<<1, kSelThreads, 0, s>>>(p4, M_cap, d_M, w.Hs, prefix, Tg, T, t2, w.flags);
    hyp_batch(p4, M_cap, d_M, nullptr, T, Tg, k0, k1, t2f, eps, t2, w.flags + 2, w, s);
    refit_launch(p4, M_cap, d_M, t2, w, H, inlier, n_in, best_t, s);
    if (iters) {
        cudaError_t e = cudaMemcpyAsync(iters, w.flags + 3, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Certain inlier counts of the last RANSAC's hypotheses (-1: none or skipped).
cudaError_t ransac_counts(void* ws, int Ttot, int32_t* host_counts, cudaStream_t s)
{
    const RansacWS w = carve(ws, Ttot);
    cudaError_t e = cudaMemcpyAsync(host_counts, w.lo, sizeof(int32_t) * (size_t)Ttot, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_diag_philox(const uint32_t* ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_diag_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(reinterpret_cast<const uint4*>(ctr), n, k0, k1,
                                                              reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

}  // namespace lp
