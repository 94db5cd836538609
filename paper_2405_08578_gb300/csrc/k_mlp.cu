// Learned RANSAC proposal (not part of the paper's method): match features, a
// 8-64-64-1 network (BF16-rounded weights, FP32 accumulation), its
// mean-BCE gradient and Adam, trained and evaluated by these kernels only.
//
//   k_mlp_features   one thread per matched pair: ratio, Delta1, scale of the
//                    reference point, orientation difference, four positions
//   k_mlp_forward    one thread per match, weights in shared memory
//   k_mlp_grad       64 samples per CTA: forward with stored activations,
//                    back-propagation, then the CTA's gradient as fixed-order
//                    sums over its samples (one partial row per CTA)
//   k_mlp_adam       one thread per parameter: fixed-order sum of the CTA
//                    partials, Adam on FP32 master weights, BF16 shadow copy
//   k_guided_prefix  one CTA: integer sampling weights of the prior and their
//                    inclusive prefix sums for RANSAC's guided draw
#include <cuda_bf16.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kNP = kMlpParams;
constexpr int kW1 = 0, kB1 = 512, kW2 = 576, kB2 = 4672, kW3 = 4736, kB3 = 4800;
constexpr int kFwdThreads = 128;
constexpr int kGradSamples = 64;
constexpr int kGradThreads = 128;

__device__ __forceinline__ float sigmoidf_stable(float z)
{
    if (z >= 0.f) return 1.f / (1.f + __expf(-z));
    const float e = __expf(z);
    return e / (1.f + e);
}

__global__ void k_mlp_features(const uint32_t* kpA, const uint8_t* oriA, int HA, int WA, const uint32_t* kpB,
                               const uint8_t* oriB, int HB, int WB, const int32_t* match, const float* d1,
                               const float* d2, const int32_t* rows, const int32_t* dM, long long M_cap,
                               MlpScales sc, float* feat)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long M = dM ? min((long long)*dM, M_cap) : M_cap;
    if (r >= M) return;
    const int i = rows[r];
    const int j = match[i];
    int l = 0;
    while (l + 1 < sc.nL && i >= sc.off[l + 1]) ++l;
    const uint32_t ia = kpA[i], ib = kpB[j];
    const uint32_t ya = ia / (uint32_t)WA, yb = ib / (uint32_t)WB;
    int dk = ((int)oriB[j] - (int)oriA[i]) % 36;
    if (dk < 0) dk += 36;
    float dth = 10.f * (float)dk;
    if (dth >= 180.f) dth -= 360.f;
    float* f = feat + 8 * r;
    f[0] = d2[i] > 0.f ? d1[i] / d2[i] : 1.f;
    f[1] = d1[i];
    f[2] = sc.log2L[l] / sc.log2Lmax;
    f[3] = dth / 180.f;
    f[4] = (float)(ia - ya * WA) / (float)WA;
    f[5] = (float)ya / (float)HA;
    f[6] = (float)(ib - yb * WB) / (float)WB;
    f[7] = (float)yb / (float)HB;
}

__device__ __forceinline__ float mlp_forward1(const float* P, const float* x, float* h1)
{
    for (int i = 0; i < 64; ++i) {
        float s = P[kB1 + i];
#pragma unroll
        for (int k = 0; k < 8; ++k) s = fmaf(P[kW1 + 8 * i + k], x[k], s);
        h1[i] = fmaxf(s, 0.f);
    }
    float z = P[kB3];
    for (int i = 0; i < 64; ++i) {
        float s = P[kB2 + i];
#pragma unroll 16
        for (int k = 0; k < 64; ++k) s = fmaf(P[kW2 + 64 * i + k], h1[k], s);
        z = fmaf(P[kW3 + i], fmaxf(s, 0.f), z);
    }
    return z;
}

__global__ void __launch_bounds__(kFwdThreads)
k_mlp_forward(const float* shadow, const float* feat, long long M_cap, const int32_t* dM, float* prob, float* logit)
{
    __shared__ float P[kNP];
    for (int e = threadIdx.x; e < kNP; e += kFwdThreads) P[e] = shadow[e];
    __syncthreads();
    const long long r = (long long)blockIdx.x * kFwdThreads + threadIdx.x;
    const long long M = dM ? min((long long)*dM, M_cap) : M_cap;
    if (r >= M) return;
    float x[8], h1[64];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = feat[8 * r + k];
    const float z = mlp_forward1(P, x, h1);
    if (logit) logit[r] = z;
    if (prob) prob[r] = sigmoidf_stable(z);
}

__global__ void __launch_bounds__(kGradThreads)
k_mlp_grad(const float* shadow, const float* feat, const uint8_t* label, long long B, float* part, float* lossp)
{
    extern __shared__ __align__(16) float smg[];
    float* P = smg;                                   // [kNP]
    float* X = P + kNP + 3;                           // [64][8]
    float* H1 = X + kGradSamples * 8;                 // [64][64]
    float* H2 = H1 + kGradSamples * 64;               // [64][64]
    float* D2 = H2 + kGradSamples * 64;               // [64][64]
    float* D1 = D2 + kGradSamples * 64;               // [64][64]
    float* DZ = D1 + kGradSamples * 64;               // [64]
    float* LS = DZ + kGradSamples;                    // [64]
    const int tid = threadIdx.x;
    for (int e = tid; e < kNP; e += kGradThreads) P[e] = shadow[e];
    const long long s0 = (long long)blockIdx.x * kGradSamples;
    const int ns = (int)min((long long)kGradSamples, B - s0);
    for (int e = tid; e < kGradSamples * 8; e += kGradThreads) X[e] = e < ns * 8 ? feat[8 * s0 + e] : 0.f;
    __syncthreads();
    // forward + back-propagation, one thread per sample
    if (tid < kGradSamples) {
        float* h1 = H1 + 64 * tid;
        float* h2 = H2 + 64 * tid;
        float* d2 = D2 + 64 * tid;
        float* d1 = D1 + 64 * tid;
        const bool live = tid < ns;
        if (live) {
            const float* x = X + 8 * tid;
            for (int i = 0; i < 64; ++i) {
                float s = P[kB1 + i];
#pragma unroll
                for (int k = 0; k < 8; ++k) s = fmaf(P[kW1 + 8 * i + k], x[k], s);
                h1[i] = fmaxf(s, 0.f);
            }
            float z = P[kB3];
            for (int i = 0; i < 64; ++i) {
                float s = P[kB2 + i];
                for (int k = 0; k < 64; ++k) s = fmaf(P[kW2 + 64 * i + k], h1[k], s);
                h2[i] = fmaxf(s, 0.f);
                z = fmaf(P[kW3 + i], h2[i], z);
            }
            const float y = label[s0 + tid] ? 1.f : 0.f;
            LS[tid] = fmaxf(z, 0.f) - z * y + log1pf(__expf(-fabsf(z)));
            const float dz = (sigmoidf_stable(z) - y) / (float)B;
            DZ[tid] = dz;
            for (int i = 0; i < 64; ++i) d2[i] = h2[i] > 0.f ? dz * P[kW3 + i] : 0.f;
            for (int k = 0; k < 64; ++k) {
                float s = 0.f;
                for (int i = 0; i < 64; ++i) s = fmaf(P[kW2 + 64 * i + k], d2[i], s);
                d1[k] = h1[k] > 0.f ? s : 0.f;
            }
        } else {
            LS[tid] = 0.f;
            DZ[tid] = 0.f;
            for (int i = 0; i < 64; ++i) { h1[i] = 0.f; h2[i] = 0.f; d2[i] = 0.f; d1[i] = 0.f; }
        }
    }
    __syncthreads();
    // this CTA's gradient: fixed-order sums over its samples
    float* out = part + (long long)blockIdx.x * kNP;
    for (int e = tid; e < kNP; e += kGradThreads) {
        float g = 0.f;
        if (e < kB1) {                       // W1[i][k] += d1[s][i] x[s][k]
            const int i = e / 8, k = e % 8;
            for (int s = 0; s < kGradSamples; ++s) g = fmaf(D1[64 * s + i], X[8 * s + k], g);
        } else if (e < kW2) {                // b1[i]
            const int i = e - kB1;
            for (int s = 0; s < kGradSamples; ++s) g += D1[64 * s + i];
        } else if (e < kB2) {                // W2[i][k] += d2[s][i] h1[s][k]
            const int i = (e - kW2) / 64, k = (e - kW2) % 64;
            for (int s = 0; s < kGradSamples; ++s) g = fmaf(D2[64 * s + i], H1[64 * s + k], g);
        } else if (e < kW3) {                // b2[i]
            const int i = e - kB2;
            for (int s = 0; s < kGradSamples; ++s) g += D2[64 * s + i];
        } else if (e < kB3) {                // w3[k] += dz[s] h2[s][k]
            const int k = e - kW3;
            for (int s = 0; s < kGradSamples; ++s) g = fmaf(DZ[s], H2[64 * s + k], g);
        } else {                             // b3
            for (int s = 0; s < kGradSamples; ++s) g += DZ[s];
        }
        out[e] = g;
    }
    if (tid == 0) {
        float l = 0.f;
        for (int s = 0; s < kGradSamples; ++s) l += LS[s];
        lossp[blockIdx.x] = l;
    }
}

__global__ void k_mlp_adam(float* master, float* m, float* v, float* shadow, const float* part, int nparts,
                           const float* lossp, long long B, float lr, float b1, float b2, float eps, float c1,
                           float c2, float* loss_out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e == 0 && loss_out) {
        float l = 0.f;
        for (int c = 0; c < nparts; ++c) l += lossp[c];
        *loss_out = l / (float)B;
    }
    if (e >= kNP) return;
    float g = 0.f;
    for (int c = 0; c < nparts; ++c) g += part[(long long)c * kNP + e];
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    const float w = master[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    master[e] = w;
    shadow[e] = __bfloat162float(__float2bfloat16_rn(w));
}

__global__ void k_shadow(const float* master, float* shadow)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kNP) shadow[e] = __bfloat162float(__float2bfloat16_rn(master[e]));
}

// q_i = floor(65536 * max(p_i, 1e-3) + 1/2) (NaN takes the floor), inclusive
// prefix sums in 64 bits.  The product is exact in FP32 (a power-of-two
// scaling); the half is added to its exact fractional part, so no rounding
// step can carry the sum across an integer.
constexpr int kPrefixThreads = 1024;

__global__ void __launch_bounds__(kPrefixThreads)
k_guided_prefix(const float* prob, long long M_cap, const int32_t* dM, unsigned long long* prefix)
{
    __shared__ unsigned long long wsum[32];
    const long long M = dM ? min((long long)*dM, M_cap) : M_cap;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long chunk = (M + kPrefixThreads - 1) / kPrefixThreads;
    const long long b = tid * chunk, e = min(M, b + chunk);
    auto q = [&](long long i) -> unsigned long long {
        float p = prob[i];
        if (!(p > 1e-3f)) p = 1e-3f;
        const float x = p * 65536.f, f = floorf(x);
        return (unsigned long long)f + (x - f >= 0.5f ? 1ull : 0ull);
    };
    unsigned long long s = 0;
    for (long long i = b; i < e; ++i) s += q(i);
    unsigned long long incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = wsum[lane];
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += v;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    unsigned long long run = wsum[warp] + incl - s;
    for (long long i = b; i < e; ++i) {
        run += q(i);
        prefix[i] = run;
    }
}

}  // namespace

size_t mlp_grad_smem() { return sizeof(float) * (kNP + 3 + kGradSamples * (8 + 4 * 64 + 2)); }
int mlp_grad_ctas(long long B) { return (int)((B + kGradSamples - 1) / kGradSamples); }

cudaError_t launch_mlp_features(const uint32_t* kpA, const uint8_t* oriA, int HA, int WA, const uint32_t* kpB,
                                const uint8_t* oriB, int HB, int WB, const int32_t* match, const float* d1,
                                const float* d2, const int32_t* rows, const int32_t* dM, long long M_cap,
                                const MlpScales& sc, float* feat, cudaStream_t s)
{
    if (M_cap <= 0) return cudaSuccess;
    k_mlp_features<<<(unsigned)((M_cap + 255) / 256), 256, 0, s>>>(kpA, oriA, HA, WA, kpB, oriB, HB, WB, match, d1,
                                                                  d2, rows, dM, M_cap, sc, feat);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* shadow, const float* feat, long long M_cap, const int32_t* dM, float* prob,
                               float* logit, cudaStream_t s)
{
    if (M_cap <= 0) return cudaSuccess;
    k_mlp_forward<<<(unsigned)((M_cap + kFwdThreads - 1) / kFwdThreads), kFwdThreads, 0, s>>>(shadow, feat, M_cap, dM,
                                                                                           prob, logit);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_step(float* master, float* m, float* v, float* shadow, const float* feat,
                                  const uint8_t* label, long long B, float* part, float* lossp, float lr, int t,
                                  float* loss_out, cudaStream_t s)
{
    const int n = mlp_grad_ctas(B);
    const size_t smem = mlp_grad_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_grad<<<n, kGradThreads, smem, s>>>(shadow, feat, label, B, part, lossp);
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, t)), c2 = (float)(1.0 - pow(b2, t));
    k_mlp_adam<<<(kNP + 255) / 256, 256, 0, s>>>(master, m, v, shadow, part, n, lossp, B, lr, (float)b1, (float)b2,
                                                 1e-8f, c1, c2, loss_out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_shadow(const float* master, float* shadow, cudaStream_t s)
{
    k_shadow<<<(kNP + 255) / 256, 256, 0, s>>>(master, shadow);
    return cudaGetLastError();
}

cudaError_t launch_guided_prefix(const float* prob, long long M_cap, const int32_t* dM, unsigned long long* prefix,
                                 cudaStream_t s)
{
    if (M_cap <= 0) return cudaSuccess;
    k_guided_prefix<<<1, kPrefixThreads, 0, s>>>(prob, M_cap, dM, prefix);
    return cudaGetLastError();
}

}  // namespace lp
