// Internal declarations of liblp (GB300 / sm_103a).  Not part of the C ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lp.h"

namespace lp {

// ---- device status word (written by kernels, read by lp_sync_status) ----
enum : int32_t { DEV_OK = 0, DEV_TIMEOUT = 4, DEV_INCONSISTENT = 8 };

__device__ __forceinline__ void set_status(int32_t* st, int32_t code)
{
    if (st) atomicCAS(st, 0, code);
}

// ---- scale table: canonical keypoint ranges per window size ----
struct ScaleTable {
    int nL;
    int L[LP_MAX_SCALES];        // ascending
    int ws[LP_MAX_SCALES];       // sub-region side w_s (Eq. 3-4)
    int pr[LP_MAX_SCALES];       // patch radius for the describe kernel
    int nwx[LP_MAX_SCALES];      // windows per row
    int nwy[LP_MAX_SCALES];
    int64_t off[LP_MAX_SCALES + 1];  // first keypoint of each scale; off[nL] = K
};

// Host-side construction (lp_api.cu).
int make_scale_table(const int* Ls, int nL, double beta0, int H, int W, ScaleTable* st);

// 2-D tiled TMA descriptor of a row-major array: `inner` elements per row,
// `outer` rows, `row_bytes` between rows, box {box_inner, box_outer}; no
// interleave, out-of-range elements read as zero.  false when the driver
// entry point is missing or rejects the arguments (k_match_tc.cu).
bool encode_tiled_2d(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                     uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swizzle);

// ---- kernel launchers (each .cu file owns its kernels) ----
// Two auxiliary streams a launcher may fork independent launches onto; it
// joins them back to its own stream before returning (graph capture follows).
struct Fork {
    cudaStream_t aux[2];
    cudaEvent_t fork_ev, join_ev[2];
};

// k_detect.cu
// alpha > 0: Eq. 1's literal FP64 ramp (one launch per scale); 0: integer keys
// status: the device status word (bounded waits of the TMA path); num_sms: the device's SM count
cudaError_t launch_detect(const uint8_t* img, int H, int W, int pitch, int ch, const ScaleTable& st, double alpha,
                          uint32_t* kp, uint8_t* gray, int32_t* status, int num_sms, cudaStream_t s);
cudaError_t launch_diag_gray(const uint8_t* rgb, int64_t n, uint8_t* gray, cudaStream_t s);
// N images with the same scales and channels in launches of up to 12 on the
// fast path; *done = false (nothing launched) when the scales need the general
// path, which the caller then runs image by image
cudaError_t launch_detect_batch(const uint8_t* const* imgs, const int* Hs, const int* Ws, const int* pitches, int N,
                                int ch, const ScaleTable* sts, uint32_t* const* kps, uint8_t* const* grays,
                                int32_t* status, int num_sms, cudaStream_t s, bool* done);

// k_describe.cu
size_t describe_lut_bytes();
cudaError_t launch_build_luts(void* luts, cudaStream_t s);

// border = 1: points whose neighbourhood (radius st.pr) leaves the image are marked invalid.
// hard = 1: each sample's magnitude goes whole to its 45-degree sector (no linear split).
// fork (or nullptr): the scale groups run concurrently on s and the two auxiliary streams.
cudaError_t launch_describe(const uint8_t* gray, int H, int W, int pitch, const uint32_t* kp,
                            const ScaleTable& st, int upright, int border, int hard, const void* luts, uint8_t* ori,
                            float* desc, uint16_t* desc_bf16, uint8_t* valid, const Fork* fork, cudaStream_t s);
cudaError_t launch_diag_orient(int32_t* bins, uint32_t* weights, cudaStream_t s);

// k_match.cu

struct MatchArgs {
    const float* dA; const uint16_t* dA16; const uint8_t* vA; int64_t NA;
    const float* dB; const uint16_t* dB16; const uint8_t* vB; int64_t NB;
    float ratio2;        // ratio^2
    float delta_s2;      // Delta_s^2 or +inf
    int32_t* match; float* d1; float* d2;
    int32_t* status;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // recorded around the distance kernel when set
    const Fork* fork = nullptr;                 // BF16 form: row norms run on the auxiliary streams
    int splits = 0;                             // BF16 form: column splits (0: the built-in choice)
    int pass1_stride = 0;                       // BF16 form: pass-1 tile stride (0: the built-in 3)
    const float* normA = nullptr;               // batched BF16 form: row norms of A and of B (+inf for
    const float* normB = nullptr;               //   invalid rows), computed once per image
    int elem = 0;                               // tensor-core operands: 0 BF16 (dA16, dB16), 1 E4M3
                                                //   (converted from dA, dB into the workspace)
};
size_t match_fp32_workspace(int64_t NA, int64_t NB, int num_sms);
cudaError_t launch_match_fp32(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s);
// S: column splits (0: the built-in choice, match_bf16_default_splits)
size_t match_bf16_workspace(int64_t NA, int64_t NB, int num_sms, int S = 0, int elem = 0);
int match_bf16_default_splits(int64_t NA, int64_t NB, int num_sms);
cudaError_t launch_match_bf16(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s);
// Batched BF16 form: the distance passes of P pairs in persistent launches of
// up to 64 pairs (k_match_tc_batch, one atomic work queue per launch), then
// per pair launch_match_bf16_tail.  sync: device int32[match_bf16_batch_sync_words]
// (zeroed here); hold: extra pass-1 completions every pass-2 unit waits for
// (diagnostic, 0 normally: a hold makes the waits give up with LP_ERR_TIMEOUT).
size_t match_bf16_batch_sync_words(const MatchArgs* args, int P);
cudaError_t launch_match_bf16_batch(const MatchArgs* args, void* const* ws, const size_t* ws_bytes, int P,
                                    int32_t* sync, int hold, int num_sms, cudaStream_t s);
cudaError_t launch_match_bf16_tail(const MatchArgs& a, void* ws, size_t ws_bytes, int num_sms, cudaStream_t s);
cudaError_t launch_row_norms(const float* d, const uint8_t* v, int64_t n, float* out, cudaStream_t s);
int64_t match_bf16_rescans(const void* ws, int64_t NA, int64_t NB, int num_sms, int S, cudaStream_t s);

// k_ransac.cu
size_t compact_workspace(int64_t NA);
cudaError_t launch_compact(const uint32_t* kpA, int WA, const uint32_t* kpB, int WB, const int32_t* match,
                           int64_t NA, float* pts, int32_t* rows, int32_t* d_M, int32_t* tile_cnt, cudaStream_t s);
size_t ransac_workspace(int64_t M_cap, int Ttot);
// model: LP_MODEL_HOMOGRAPHY (Eq. 7) or LP_MODEL_RIGID (Eq. 8)
cudaError_t launch_ransac(const float* pts, int64_t M_cap, const int32_t* d_M, int T, int model, float thresh,
                          uint64_t seed, uint32_t pair_id, double* H, uint8_t* inlier, int32_t* n_in,
                          int32_t* best_t, void* ws, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_diag_philox(const uint32_t* ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* out,
                               cudaStream_t s);

// k_ransac.cu (guided phase, stop test, uniform fallback); Ttot = Tg + T; the
// guided winner ends the search only with at least min_support inliers
cudaError_t launch_ransac_prior(const float* pts, int64_t M_cap, const int32_t* d_M, const unsigned long long* prefix,
                                int Tg, int T, int model, float thresh, uint64_t seed, uint32_t pair_id,
                                int min_support, double* H,
                                uint8_t* inlier, int32_t* n_in, int32_t* best_t, int32_t* iters, void* ws,
                                size_t ws_bytes, cudaStream_t s);
cudaError_t ransac_counts(void* ws, int Ttot, int32_t* host_counts, cudaStream_t s);

// k_mosaic.cu (Sec. 4 canvas); *bad = 1: more than 64 images or a singular placement
cudaError_t launch_mosaic_render(const lp_image* imgs, int N, const double* G, const int32_t* round_of, uint8_t* canvas,
                                 int cw, int ch, int pitch, uint8_t* cover, cudaStream_t s, int* bad);

// k_mlp.cu (learned proposal)
constexpr int kMlpParams = 4801;
struct MlpScales {
    int nL;
    long long off[LP_MAX_SCALES + 1];
    float log2L[LP_MAX_SCALES];
    float log2Lmax;
};
size_t mlp_grad_smem();
int mlp_grad_ctas(long long B);
cudaError_t launch_mlp_features(const uint32_t* kpA, const uint8_t* oriA, int HA, int WA, const uint32_t* kpB,
                                const uint8_t* oriB, int HB, int WB, const int32_t* match, const float* d1,
                                const float* d2, const int32_t* rows, const int32_t* dM, long long M_cap,
                                const MlpScales& sc, float* feat, cudaStream_t s);
cudaError_t launch_mlp_forward(const float* shadow, const float* feat, long long M_cap, const int32_t* dM, float* prob,
                               float* logit, cudaStream_t s);
cudaError_t launch_mlp_train_step(float* master, float* m, float* v, float* shadow, const float* feat,
                                  const uint8_t* label, long long B, float* part, float* lossp, float lr, int t,
                                  float* loss_out, cudaStream_t s);
cudaError_t launch_mlp_shadow(const float* master, float* shadow, cudaStream_t s);
cudaError_t launch_guided_prefix(const float* prob, long long M_cap, const int32_t* dM, unsigned long long* prefix,
                                 cudaStream_t s);

}  // namespace lp
