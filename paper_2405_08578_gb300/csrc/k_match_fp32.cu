// Nearest-neighbour matching with Eq. 6 distances (Sec. 2.4), plain FP32 form.
//
// Delta^2(i, j) = |a_i|^2 + |b_j|^2 - 2 a_i . b_j, the dot products by a
// register-blocked SIMT GEMM (FP32 FMA): a CTA keeps its 128 A rows (64 KB,
// transposed) resident in shared memory and streams 128-column B tiles in
// 32-deep K chunks (double-buffered).  Each thread owns an 8 x 8 block of
// distances and keeps, per row, the two smallest |b_j|^2 - 2 a.b seen so far
// (lowest j on ties, because columns are visited in increasing order).  The
// B range is split S ways so that the grid fills whole waves; a finishing
// kernel merges the S partial top-2 lists, adds |a_i|^2 and applies the ratio
// test and Delta_s.  No distance matrix is ever written.
#include "lp_internal.cuh"

namespace lp {

// Shared with the BF16 path (k_match_tc.cu).
__global__ void k_row_norms(const float* d, const uint8_t* v, long long n, float* out, float invalid_value);
__global__ void k_match_finish(const float4* part, int S, long long NA, const float* na, const uint8_t* vA,
                               float ratio2, float delta_s2, int32_t* match, float* d1, float* d2);

namespace {

constexpr int kTile = 128;     // rows and columns per CTA tile
constexpr int kKc = 32;        // K chunk
constexpr int kThreads = 256;  // 16 x 16 threads, 8 x 8 outputs each
constexpr int kPadA = 4;       // AsT row pad (floats)

struct Top2 {
    float b1, b2;
    int j1, j2;
};

__device__ __forceinline__ void top2_push(Top2& t, float d, int j)
{
    if (d < t.b2) {
        if (d < t.b1) {
            t.b2 = t.b1; t.j2 = t.j1;
            t.b1 = d; t.j1 = j;
        } else {
            t.b2 = d; t.j2 = j;
        }
    }
}

// (d, j) lexicographic order: smaller distance first, lower index on ties.
__device__ __forceinline__ bool lex_less(float d, int j, float e, int k)
{
    return d < e || (d == e && (unsigned)j < (unsigned)k);
}

__device__ __forceinline__ void top2_merge(Top2& t, float d, int j)
{
    if (j < 0) return;
    if (lex_less(d, j, t.b1, t.j1)) {
        t.b2 = t.b1; t.j2 = t.j1;
        t.b1 = d; t.j1 = j;
    } else if (lex_less(d, j, t.b2, t.j2)) {
        t.b2 = d; t.j2 = j;
    }
}

__global__ void __launch_bounds__(kThreads, 2)
k_match_fp32_main(const float* __restrict__ A, long long NA, const int32_t* __restrict__ d_rows,
                  const float* __restrict__ B, const float* __restrict__ nb, long long NB, int S,
                  long long cols_per_split, float4* __restrict__ part)
{
    extern __shared__ __align__(16) float smf[];
    float* AsT = smf;                                 // [128 k][128 + pad rows]
    float* BsT = AsT + 128 * (kTile + kPadA);         // 2 x [32 k][128 cols]
    float* nbs = BsT + 2 * kKc * kTile;               // [128]

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const long long row0 = (long long)blockIdx.x * kTile;
    // rows beyond a device-side count (queued re-scan rows) have nothing to do;
    // the partial layout keeps NA as its row capacity
    const long long n_rows = d_rows ? min(NA, (long long)*d_rows) : NA;
    if (row0 >= n_rows) return;
    const int split = blockIdx.y;
    const long long c_begin = (long long)split * cols_per_split;
    const long long c_end = min(NB, c_begin + cols_per_split);

    // A block, transposed: AsT[k][r]
    for (int e = tid; e < kTile * 32; e += kThreads) {
        const int r = e >> 5, q = e & 31;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row0 + r < n_rows) v = __ldg(reinterpret_cast<const float4*>(A + (row0 + r) * 128) + q);
        AsT[(4 * q + 0) * (kTile + kPadA) + r] = v.x;
        AsT[(4 * q + 1) * (kTile + kPadA) + r] = v.y;
        AsT[(4 * q + 2) * (kTile + kPadA) + r] = v.z;
        AsT[(4 * q + 3) * (kTile + kPadA) + r] = v.w;
    }

    Top2 best[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) best[i] = Top2{INFINITY, INFINITY, -1, -1};

    auto load_chunk = [&](long long c0, int kc, float* dst) {
        // 128 columns x 32 k = 1024 float4 -> 4 per thread; stored [k][col]
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            const int e = tid + it * kThreads;
            const int col = e & 127, q = e >> 7;        // q in [0, 8)
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c0 + col < c_end) v = __ldg(reinterpret_cast<const float4*>(B + (c0 + col) * 128 + kc) + q);
            dst[(4 * q + 0) * kTile + col] = v.x;
            dst[(4 * q + 1) * kTile + col] = v.y;
            dst[(4 * q + 2) * kTile + col] = v.z;
            dst[(4 * q + 3) * kTile + col] = v.w;
        }
    };

    for (long long c0 = c_begin; c0 < c_end; c0 += kTile) {
        __syncthreads();   // previous tile fully consumed (and A staged on the first pass)
        if (tid < kTile) nbs[tid] = (c0 + tid < c_end) ? __ldg(nb + c0 + tid) : INFINITY;
        load_chunk(c0, 0, BsT);
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 1
        for (int kc = 0; kc < 128; kc += kKc) {
            __syncthreads();
            float* cur = BsT + ((kc / kKc) & 1) * kKc * kTile;
            if (kc + kKc < 128) load_chunk(c0, kc + kKc, BsT + (((kc / kKc) + 1) & 1) * kKc * kTile);
#pragma unroll 4
            for (int k = 0; k < kKc; ++k) {
                const float* ak = AsT + (kc + k) * (kTile + kPadA) + ty * 8;
                const float* bk = cur + k * kTile + tx * 8;
                const float4 a0 = *reinterpret_cast<const float4*>(ak);
                const float4 a1 = *reinterpret_cast<const float4*>(ak + 4);
                const float4 b0 = *reinterpret_cast<const float4*>(bk);
                const float4 b1 = *reinterpret_cast<const float4*>(bk + 4);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float nbj = nbs[tx * 8 + j];
            const int col = (int)(c0 + tx * 8 + j);
#pragma unroll
            for (int i = 0; i < 8; ++i) top2_push(best[i], fmaf(-2.f, acc[i][j], nbj), col);
        }
    }
    // merge the 16 column-owners of each row (a half-warp) in fixed order
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const float ob1 = __shfl_xor_sync(0xFFFFFFFFu, best[i].b1, o);
            const float ob2 = __shfl_xor_sync(0xFFFFFFFFu, best[i].b2, o);
            const int oj1 = __shfl_xor_sync(0xFFFFFFFFu, best[i].j1, o);
            const int oj2 = __shfl_xor_sync(0xFFFFFFFFu, best[i].j2, o);
            top2_merge(best[i], ob1, oj1);
            top2_merge(best[i], ob2, oj2);
        }
        const long long r = row0 + ty * 8 + i;
        if (tx == 0 && r < n_rows)
            part[(long long)split * NA + r] =
                make_float4(best[i].b1, best[i].b2, __int_as_float(best[i].j1), __int_as_float(best[i].j2));
    }
}

int pick_splits(long long rowblocks, long long NB, int slots)
{
    long long maxS = (NB + kTile - 1) / kTile;
    int bestS = 1;
    double bestEff = -1;
    for (int S = 1; S <= 32 && S <= maxS; ++S) {
        const double waves = (double)(rowblocks * S) / slots;
        const double eff = waves / ceil(waves) - (S - 1) * 0.002;   // small cost per extra split
        if (waves >= 1.0 && eff > bestEff + 1e-9) { bestEff = eff; bestS = S; }
        if (waves < 1.0 && bestEff < 0) bestS = S;
    }
    return bestS;
}

size_t smem_bytes() { return sizeof(float) * (128 * (kTile + kPadA) + 2 * kKc * kTile + kTile); }

}  // namespace

// |d_i|^2 per row (fixed summation order); rows with v == 0 get invalid_value.
__global__ void k_row_norms(const float* d, const uint8_t* v, long long n, float* out, float invalid_value)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const float4 x = reinterpret_cast<const float4*>(d + w * 128)[lane];
    float s = x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) out[w] = v[w] ? s : invalid_value;
}

// Merge S partial top-2 lists (split order = column order), then Eq. 6 and the
// ratio test (ratio2 = 0: no ratio test, any valid nearest neighbour passes to
// the Delta_s test).  part rows hold (b1, b2, j1, j2) with b = |b|^2 - 2 a.b.
__global__ void k_match_finish(const float4* part, int S, long long NA, const float* na, const uint8_t* vA,
                               float ratio2, float delta_s2, int32_t* match, float* d1, float* d2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NA) return;
    Top2 t{INFINITY, INFINITY, -1, -1};
    for (int s = 0; s < S; ++s) {
        const float4 p = part[(long long)s * NA + i];
        top2_merge(t, p.x, __float_as_int(p.z));
        top2_merge(t, p.y, __float_as_int(p.w));
    }
    const float a2 = na[i];
    const float e1 = fmaxf(a2 + t.b1, 0.f), e2 = fmaxf(a2 + t.b2, 0.f);
    const bool ratio_ok = ratio2 > 0.f ? (t.j2 >= 0 && isfinite(t.b2) && e1 < ratio2 * e2) : (t.j1 >= 0 && isfinite(t.b1));
    const bool ok = vA[i] && ratio_ok && e1 < delta_s2;
    match[i] = ok ? t.j1 : -1;
    d1[i] = (vA[i] && t.j1 >= 0) ? sqrtf(e1) : INFINITY;
    d2[i] = (vA[i] && t.j2 >= 0) ? sqrtf(e2) : INFINITY;
}

size_t match_fp32_workspace(int64_t NA, int64_t NB, int num_sms)
{
    const long long rowblocks = (NA + kTile - 1) / kTile;
    const int S = pick_splits(rowblocks, NB, 2 * num_sms);
    return 256 + sizeof(float) * (size_t)(NA + NB) + sizeof(float4) * (size_t)S * (size_t)NA;
}

cudaError_t launch_match_fp32(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s)
{
    const long long rowblocks = (a.NA + kTile - 1) / kTile;
    const int S = pick_splits(rowblocks, a.NB, 2 * num_sms);
    if (ws_bytes < match_fp32_workspace(a.NA, a.NB, num_sms)) return cudaErrorInvalidValue;
    float* na = reinterpret_cast<float*>(ws);
    float* nb = na + a.NA;
    float4* part = reinterpret_cast<float4*>(reinterpret_cast<uintptr_t>(nb + a.NB + 3) & ~uintptr_t(15));
    if (a.NA == 0) return cudaSuccess;
    k_row_norms<<<(unsigned)((a.NA * 32 + 255) / 256), 256, 0, s>>>(a.dA, a.vA, a.NA, na, 0.f);
    if (a.NB > 0) k_row_norms<<<(unsigned)((a.NB * 32 + 255) / 256), 256, 0, s>>>(a.dB, a.vB, a.NB, nb, INFINITY);
    const long long tiles = (a.NB + kTile - 1) / kTile;
    const long long cps = ((tiles + S - 1) / S) * kTile;
    const size_t smem = smem_bytes();
    cudaFuncSetAttribute(k_match_fp32_main, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (a.NB > 0) {
        dim3 grid((unsigned)rowblocks, (unsigned)S);
        if (a.ev0) cudaEventRecord(a.ev0, s);
        k_match_fp32_main<<<grid, kThreads, smem, s>>>(a.dA, a.NA, nullptr, a.dB, nb, a.NB, S, cps, part);
        if (a.ev1) cudaEventRecord(a.ev1, s);
    }
    const int Sused = a.NB > 0 ? S : 0;
    k_match_finish<<<(unsigned)((a.NA + 255) / 256), 256, 0, s>>>(part, Sused, a.NA, na, a.vA, a.ratio2, a.delta_s2,
                                                                  a.match, a.d1, a.d2);
    return cudaGetLastError();
}

}  // namespace lp
