// C ABI of liblp: argument validation, context, workspace and the stage
// sequence of the LP-SIFT path (Sec. 2 of the paper, Fig. 2 steps (b)-(f)).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lp_internal.cuh"

namespace {

struct DBuf {
    void* p = nullptr;
    size_t n = 0;
};

enum BufId {
    B_MATCH_WS, B_RANSAC_WS,
    B_IMG_A, B_IMG_B, B_GRAY_A, B_GRAY_B, B_KP_A, B_KP_B, B_ORI_A, B_ORI_B,
    B_DESC_A, B_DESC_B, B_D16_A, B_D16_B, B_VAL_A, B_VAL_B,
    B_MATCH, B_D1, B_D2, B_PTS, B_M, B_INL, B_H, B_NIN, B_BEST, B_LUTS, B_BATCH, B_PREFIX,
    B_ROWS, B_FEAT, B_PROB, B_COMPACT,
    B_IMG_A1, B_IMG_B1, B_HSTREAM,
    B_COUNT
};

}  // namespace

struct lp_mlp {
    int device = 0;
    float* master = nullptr;   // [LP_MLP_PARAMS] x 4: master, m, v, shadow (one block)
    float* m = nullptr;
    float* v = nullptr;
    float* shadow = nullptr;
    float* part = nullptr;     // per-CTA gradient partials
    float* lossp = nullptr;
    size_t part_ctas = 0;
    int step = 0;
};

struct lp_ctx {
    lp_config cfg;
    int64_t last_NA = 0, last_NB = 0;   // sizes of the last BF16 match (for diagnostics)
    bool luts_ready = false;            // orientation tables built on this context's device
    std::vector<long long> graph_key;   // lp_stitch_pairs: what the cached graph was captured for
    cudaGraphExec_t graph_exec = nullptr;
    int device = 0;
    int num_sms = 0;
    int32_t* d_status = nullptr;
    cudaStream_t last = nullptr;
    int last_ransac_hyps = 0;           // hypotheses of the last lp_ransac / lp_ransac_prior
    lp_mlp* proposal = nullptr;         // lp_set_proposal: network guiding the stitch calls' RANSAC
    cudaEvent_t prof_ev[2] = {nullptr, nullptr};   // lp_set_profiling: around the last distance kernel
    bool prof_recorded = false;
    int32_t guided_iters = 0;
    // lp_set_autotune: (S, pass-1 stride) of the BF16 matcher per size class
    // (ceil(log2 NA), ceil(log2 NB)), timed on the class's first eager call
    bool autotune = false;
    struct TuneEntry {
        int ba, bb, S, stride;
        float us, us_builtin;
    };
    std::vector<TuneEntry> tune;
    int last_S = 0;                     // column splits of the last BF16 match
    int batch_hold = 0;                 // lp_diag_set_batch_hold: extra pass-1 completions batch waits expect
    lp::Fork fork{};                    // auxiliary streams of lp_describe (created on first use)
    bool fork_ready = false;
    cudaStream_t img_stream = nullptr;  // lp_stitch_pair: image B's detect and describe;
                                        // lp_stitch_pairs: the pairs' RANSAC
    cudaEvent_t img_ev[2] = {nullptr, nullptr};
    cudaEvent_t pair_ev[4] = {nullptr, nullptr, nullptr, nullptr};   // lp_stitch_pairs: compacted, lane slot 0..2 free
    // lp_stitch_pairs_host: upload stream; per upload slot "uploaded" and
    // "free again" events, and the caller's start
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t up_ev[2] = {nullptr, nullptr}, free_ev[2] = {nullptr, nullptr}, start_ev = nullptr;
    DBuf buf[B_COUNT];
    char err[512];
};

namespace {

int fail(lp_ctx* c, int code, const char* fmt, ...);

// The context's auxiliary streams and events, created on first use.
int ensure_fork(lp_ctx* c)
{
    if (c->fork_ready) return LP_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&c->fork.aux[0], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->fork.aux[1], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork.fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork.join_ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork.join_ev[1], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LP_ERR_CUDA, "auxiliary streams: %s", cudaGetErrorString(e));
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->img_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->img_ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->img_ev[1], cudaEventDisableTiming);
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&c->pair_ev[q], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LP_ERR_CUDA, "auxiliary streams: %s", cudaGetErrorString(e));
    }
    c->fork_ready = true;
    return LP_OK;
}

int fail(lp_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof c->err, fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(lp_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, LP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LP_CUDA(ctx, call)                                    \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Grow-only device buffer owned by the context.  Growing waits for the
// context's last stream so that no queued kernel still uses the old block.
int ensure(lp_ctx* c, BufId id, size_t bytes)
{
    DBuf& b = c->buf[id];
    if (b.n >= bytes && b.p) return LP_OK;
    if (b.p) {
        if (c->last) cudaStreamSynchronize(c->last);
        cudaFree(b.p);
        b.p = nullptr;
        b.n = 0;
    }
    size_t n = std::max<size_t>(bytes, 256);
    n = (n + 4095) & ~size_t(4095);
    cudaError_t e = cudaMalloc(&b.p, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(c, LP_ERR_NOMEM, "workspace allocation of %zu bytes failed: %s", n, cudaGetErrorString(e));
    }
    b.n = n;
    return LP_OK;
}

int check_cfg(lp_ctx* c, const lp_config* cfg)
{
    if (!cfg) return fail(c, LP_ERR_ARG, "null config");
    if (cfg->nL < 1 || cfg->nL > LP_MAX_SCALES) return fail(c, LP_ERR_ARG, "nL=%d outside 1..%d", cfg->nL, LP_MAX_SCALES);
    for (int l = 0; l < cfg->nL; ++l) {
        if (cfg->Ls[l] < 2 || cfg->Ls[l] > 4096) return fail(c, LP_ERR_ARG, "L=%d outside 2..4096", cfg->Ls[l]);
        for (int m = 0; m < l; ++m)
            if (cfg->Ls[m] == cfg->Ls[l]) return fail(c, LP_ERR_ARG, "window size %d repeated", cfg->Ls[l]);
    }
    if (!(cfg->ratio >= 0.f && cfg->ratio <= 1.f)) return fail(c, LP_ERR_ARG, "ratio must be in [0, 1]");
    if (!(cfg->alpha >= 0.0 && cfg->alpha < 1e300)) return fail(c, LP_ERR_ARG, "alpha must be finite and >= 0");
    if (cfg->border != 0 && cfg->border != 1) return fail(c, LP_ERR_ARG, "border must be 0 or 1");
    if (cfg->hard_bins != 0 && cfg->hard_bins != 1) return fail(c, LP_ERR_ARG, "hard_bins must be 0 or 1");
    if (cfg->ransac_iters < 1 || cfg->ransac_iters > 65536) return fail(c, LP_ERR_ARG, "ransac_iters outside 1..65536");
    if (!(cfg->thresh_px > 0.f)) return fail(c, LP_ERR_ARG, "thresh_px must be > 0");
    if (cfg->precision != LP_PREC_FP32 && cfg->precision != LP_PREC_BF16 && cfg->precision != LP_PREC_FP8)
        return fail(c, LP_ERR_ARG, "unknown precision %d", cfg->precision);
    if (cfg->model != LP_MODEL_HOMOGRAPHY && cfg->model != LP_MODEL_RIGID)
        return fail(c, LP_ERR_ARG, "unknown model %d", cfg->model);
    return LP_OK;
}

int check_image(lp_ctx* c, const uint8_t* img, int H, int W, int pitch, int ch)
{
    if (!img) return fail(c, LP_ERR_ARG, "null image");
    if (H <= 0 || W <= 0) return fail(c, LP_ERR_ARG, "image %dx%d is empty", W, H);
    if ((long long)H * W > (1ll << 24)) return fail(c, LP_ERR_UNSUPPORTED, "H*W=%lld above 2^24", (long long)H * W);
    if (ch != 1 && ch != 3) return fail(c, LP_ERR_ARG, "channels=%d (1 or 3)", ch);
    if (pitch < W * ch) return fail(c, LP_ERR_ARG, "pitch %d < W*channels %d", pitch, W * ch);
    if (pitch % 16 || !aligned(img, 16)) return fail(c, LP_ERR_ALIGN, "image base and pitch must be 16-byte aligned");
    return LP_OK;
}

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

int build_luts(lp_ctx* c, cudaStream_t s)
{
    int r = ensure(c, B_LUTS, lp::describe_lut_bytes());
    if (r) return r;
    LP_CUDA(c, lp::launch_build_luts(c->buf[B_LUTS].p, s));
    c->luts_ready = true;
    return LP_OK;
}

size_t al256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

namespace lp {

int make_scale_table(const int* Ls_in, int nL, double beta0, int H, int W, ScaleTable* st)
{
    if (nL < 1 || nL > LP_MAX_SCALES) return LP_ERR_ARG;
    int Ls[LP_MAX_SCALES];
    // ascending (insertion sort of at most LP_MAX_SCALES values)
    for (int l = 0; l < nL; ++l) {
        int k = l;
        for (; k > 0 && Ls[k - 1] > Ls_in[l]; --k) Ls[k] = Ls[k - 1];
        Ls[k] = Ls_in[l];
    }
    const int Lmin = Ls[0], Lmax = Ls[nL - 1];
    // Eq. 3-4: w_s = beta*L, beta = beta0*(L/Lmax)^(-1/2); the default beta0 is
    // the largest value that keeps w = 4 w_s <= L for every L
    if (beta0 <= 0) beta0 = sqrt((double)Lmin / (double)Lmax) / 4.0;
    st->nL = nL;
    int64_t off = 0;
    for (int l = 0; l < nL; ++l) {
        st->L[l] = Ls[l];
        const double beta = beta0 * pow((double)Ls[l] / (double)Lmax, -0.5);
        const int w = (int)floor(beta * Ls[l] + 0.5);
        st->ws[l] = w < 1 ? 1 : w;
        // neighbourhood radius: turned-grid points reach sqrt(2) (2 w_s + 1);
        // bilinear taps add one pixel
        st->pr[l] = (int)ceil(2.0 * sqrt(2.0) * st->ws[l] + 1.5) + 1;
        st->nwx[l] = W / Ls[l];
        st->nwy[l] = H / Ls[l];
        st->off[l] = off;
        off += 2ll * st->nwx[l] * st->nwy[l];
    }
    st->off[nL] = off;
    return LP_OK;
}

}  // namespace lp

extern "C" {

int lp_config_default(lp_config* cfg)
{
    if (!cfg) return LP_ERR_ARG;
    memset(cfg, 0, sizeof *cfg);
    cfg->nL = 4;
    cfg->Ls[0] = 16; cfg->Ls[1] = 32; cfg->Ls[2] = 64; cfg->Ls[3] = 128;
    cfg->beta0 = 0.0;
    cfg->ratio = 0.8f;
    cfg->delta_s = INFINITY;
    cfg->ransac_iters = 1000;
    cfg->thresh_px = 3.0f;
    cfg->seed = 0;
    cfg->min_inliers = 8;
    cfg->precision = LP_PREC_FP32;
    cfg->upright = 0;
    cfg->model = LP_MODEL_HOMOGRAPHY;
    cfg->alpha = 0.0;
    cfg->border = 0;
    cfg->hard_bins = 0;
    return LP_OK;
}

int lp_create(lp_ctx** out, const lp_config* cfg)
{
    if (!out) return LP_ERR_ARG;
    *out = nullptr;
    lp_ctx* c = new lp_ctx();
    c->err[0] = 0;
    int r = check_cfg(c, cfg);
    if (r) { delete c; return r; }
    c->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        return LP_ERR_CUDA;
    }
    *out = c;
    return LP_OK;
}

int lp_destroy(lp_ctx* c)
{
    if (!c) return LP_ERR_ARG;
    cudaDeviceSynchronize();
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    for (auto& b : c->buf)
        if (b.p) cudaFree(b.p);
    if (c->d_status) cudaFree(c->d_status);
    for (auto& e : c->prof_ev)
        if (e) cudaEventDestroy(e);
    if (c->fork_ready) {
        for (auto& a : c->fork.aux) cudaStreamDestroy(a);
        cudaEventDestroy(c->fork.fork_ev);
        for (auto& e : c->fork.join_ev) cudaEventDestroy(e);
        cudaStreamDestroy(c->img_stream);
        for (auto& e : c->img_ev) cudaEventDestroy(e);
        for (auto& e : c->pair_ev) cudaEventDestroy(e);
    }
    if (c->copy_stream) {
        cudaStreamDestroy(c->copy_stream);
        for (auto& e : c->up_ev) cudaEventDestroy(e);
        for (auto& e : c->free_ev) cudaEventDestroy(e);
        cudaEventDestroy(c->start_ev);
    }
    delete c;
    return LP_OK;
}

int64_t lp_num_keypoints(int H, int W, const int* Ls, int nL)
{
    if (!Ls || nL < 1 || H < 0 || W < 0) return -1;
    int64_t K = 0;
    for (int l = 0; l < nL; ++l) {
        if (Ls[l] < 2) return -1;
        K += 2ll * (H / Ls[l]) * (W / Ls[l]);
    }
    return K;
}

int lp_detect(lp_ctx* c, const uint8_t* img, int H, int W, int pitch, int channels, uint32_t* kp_idx,
              uint8_t* gray, void* stream)
{
    if (!c) return LP_ERR_ARG;
    int r = check_image(c, img, H, W, pitch, channels);
    if (r) return r;
    const int64_t K = lp_num_keypoints(H, W, c->cfg.Ls, c->cfg.nL);
    if (K > 0 && !kp_idx) return fail(c, LP_ERR_ARG, "null kp_idx");
    if (kp_idx && !aligned(kp_idx, 8)) return fail(c, LP_ERR_ALIGN, "kp_idx must be 8-byte aligned");
    if (channels == 3 && !gray) return fail(c, LP_ERR_ARG, "RGB input needs the gray output buffer");
    if (channels == 3 && (W % 16 == 0) && !aligned(gray, 16)) return fail(c, LP_ERR_ALIGN, "gray must be 16-byte aligned");
    lp::ScaleTable st;
    lp::make_scale_table(c->cfg.Ls, c->cfg.nL, c->cfg.beta0, H, W, &st);
    c->last = S(stream);
    LP_CUDA(c, lp::launch_detect(img, H, W, pitch, channels, st, c->cfg.alpha, kp_idx, gray, c->d_status, c->num_sms,
                                 S(stream)));
    return LP_OK;
}

int lp_detect_batch(lp_ctx* c, const lp_image* imgs, int N, uint32_t* const* kp_idx, uint8_t* const* gray,
                    void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (N < 1 || !imgs || !kp_idx || !gray) return fail(c, LP_ERR_ARG, "need N >= 1 images and their outputs");
    const int ch = imgs[0].channels;
    for (int i = 0; i < N; ++i) {
        int r = check_image(c, imgs[i].data, imgs[i].H, imgs[i].W, imgs[i].pitch, imgs[i].channels);
        if (r) return r;
        if (imgs[i].channels != ch) return fail(c, LP_ERR_ARG, "images differ in channel count");
        const int64_t K = lp_num_keypoints(imgs[i].H, imgs[i].W, c->cfg.Ls, c->cfg.nL);
        if (K > 0 && !kp_idx[i]) return fail(c, LP_ERR_ARG, "null kp_idx[%d]", i);
        if (kp_idx[i] && !aligned(kp_idx[i], 8)) return fail(c, LP_ERR_ALIGN, "kp_idx[%d] must be 8-byte aligned", i);
        if (ch == 3 && !gray[i]) return fail(c, LP_ERR_ARG, "RGB input needs gray[%d]", i);
        if (ch == 3 && (imgs[i].W % 16 == 0) && !aligned(gray[i], 16))
            return fail(c, LP_ERR_ALIGN, "gray[%d] must be 16-byte aligned", i);
    }
    c->last = S(stream);
    bool done = false;
    if (c->cfg.alpha == 0.0) {
        std::vector<lp::ScaleTable> st((size_t)N);
        std::vector<const uint8_t*> src((size_t)N);
        std::vector<int> Hs((size_t)N), Ws((size_t)N), ps((size_t)N);
        for (int i = 0; i < N; ++i) {
            lp::make_scale_table(c->cfg.Ls, c->cfg.nL, c->cfg.beta0, imgs[i].H, imgs[i].W, &st[i]);
            src[i] = imgs[i].data; Hs[i] = imgs[i].H; Ws[i] = imgs[i].W; ps[i] = imgs[i].pitch;
        }
        LP_CUDA(c, lp::launch_detect_batch(src.data(), Hs.data(), Ws.data(), ps.data(), N, ch, st.data(), kp_idx,
                                           gray, c->d_status, c->num_sms, S(stream), &done));
    }
    for (int i = 0; i < N && !done; ++i) {
        int r = lp_detect(c, imgs[i].data, imgs[i].H, imgs[i].W, imgs[i].pitch, ch, kp_idx[i], gray[i], stream);
        if (r) return r;
    }
    return LP_OK;
}

int lp_describe(lp_ctx* c, const uint8_t* gray, int H, int W, int gray_pitch, const uint32_t* kp_idx, int64_t K,
                uint8_t* ori, float* desc, uint16_t* desc_bf16, uint8_t* valid, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (!gray || H <= 0 || W <= 0 || gray_pitch < W) return fail(c, LP_ERR_ARG, "bad intensity image");
    if ((long long)H * W > (1ll << 24)) return fail(c, LP_ERR_UNSUPPORTED, "H*W above 2^24");
    const int64_t Kexp = lp_num_keypoints(H, W, c->cfg.Ls, c->cfg.nL);
    if (K != Kexp) return fail(c, LP_ERR_ARG, "K=%lld but the image has %lld feature points", (long long)K, (long long)Kexp);
    if (K == 0) return LP_OK;
    if (!kp_idx || !ori || !desc || !valid) return fail(c, LP_ERR_ARG, "null output");
    if (!aligned(desc, 16) || (desc_bf16 && !aligned(desc_bf16, 8))) return fail(c, LP_ERR_ALIGN, "descriptor alignment");
    lp::ScaleTable st;
    lp::make_scale_table(c->cfg.Ls, c->cfg.nL, c->cfg.beta0, H, W, &st);
    c->last = S(stream);
    if (!c->luts_ready) {
        int r = build_luts(c, S(stream));
        if (r) return r;
    }
    if (int r = ensure_fork(c)) return r;
    LP_CUDA(c, lp::launch_describe(gray, H, W, gray_pitch, kp_idx, st, c->cfg.upright, c->cfg.border,
                                   c->cfg.hard_bins, c->buf[B_LUTS].p, ori, desc, desc_bf16, valid, &c->fork,
                                   S(stream)));
    return LP_OK;
}

namespace {

int log2_bucket(int64_t n)
{
    int b = 0;
    while (b < 62 && (int64_t(1) << b) < n) ++b;
    return b;
}

// The BF16 matcher's (column splits, pass-1 stride) for a's size class: the
// cached choice, or -- on the class's first call outside stream capture --
// the fastest of a few candidates around the built-in choice, each timed once
// after a warm-up run on the caller's own inputs.  Every candidate gives the
// same outputs (each is certified against the FP32 form), so tuning on live
// data changes nothing but the time.  Under capture the built-in choice runs.
int tune_match(lp_ctx* c, lp::MatchArgs& a, cudaStream_t s)
{
    const int ba = log2_bucket(a.NA), bb = log2_bucket(a.NB);
    for (const auto& e : c->tune)
        if (e.ba == ba && e.bb == bb) {
            a.splits = e.S;
            a.pass1_stride = e.stride;
            return LP_OK;
        }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return LP_OK;
    const int S0 = lp::match_bf16_default_splits(a.NA, a.NB, c->num_sms);
    std::vector<std::pair<int, int>> cand = {{S0, 3}, {S0, 2}, {S0, 4}, {std::max(1, S0 / 2), 3},
                                             {std::min(16, 2 * S0), 3}, {std::min(16, S0 + 1), 3}};
    std::sort(cand.begin() + 1, cand.end());
    cand.erase(std::unique(cand.begin() + 1, cand.end()), cand.end());
    size_t ws = 0;
    for (const auto& q : cand) ws = std::max(ws, lp::match_bf16_workspace(a.NA, a.NB, c->num_sms, q.first, a.elem));
    int r = ensure(c, B_MATCH_WS, ws);
    if (r) return r;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LP_CUDA(c, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(c, ce, "cudaEventCreate");
    }
    lp::MatchArgs t = a;
    t.ev0 = t.ev1 = nullptr;
    float best = INFINITY, builtin = INFINITY;
    int bS = S0, bst = 3;
    for (size_t k = 0; k < cand.size() && ce == cudaSuccess; ++k) {
        t.splits = cand[k].first;
        t.pass1_stride = cand[k].second;
        float ms = 0.f;
        if ((ce = lp::launch_match_bf16(t, c->buf[B_MATCH_WS].p, c->buf[B_MATCH_WS].n, c->num_sms, s)) != cudaSuccess ||
            (ce = cudaEventRecord(e0, s)) != cudaSuccess ||
            (ce = lp::launch_match_bf16(t, c->buf[B_MATCH_WS].p, c->buf[B_MATCH_WS].n, c->num_sms, s)) != cudaSuccess ||
            (ce = cudaEventRecord(e1, s)) != cudaSuccess || (ce = cudaEventSynchronize(e1)) != cudaSuccess ||
            (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
            break;
        if (k == 0) builtin = ms;
        if (ms < best) { best = ms; bS = cand[k].first; bst = cand[k].second; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "autotune");
    c->tune.push_back({ba, bb, bS, bst, 1e3f * best, 1e3f * builtin});
    a.splits = bS;
    a.pass1_stride = bst;
    return LP_OK;
}

// The tuned (splits, pass-1 stride) of a size class when the tuner is on and
// the class is in the table; 0 (the built-in choice) otherwise.
int tuned_splits(const lp_ctx* c, int64_t NA, int64_t NB, int* stride)
{
    *stride = 0;
    if (!c->autotune) return 0;
    const int ba = log2_bucket(NA), bb = log2_bucket(NB);
    for (const auto& e : c->tune)
        if (e.ba == ba && e.bb == bb) {
            *stride = e.stride;
            return e.S;
        }
    return 0;
}

}  // namespace

int lp_match(lp_ctx* c, const float* dA, const uint16_t* dA_bf16, const uint8_t* vA, int64_t NA, const float* dB,
             const uint16_t* dB_bf16, const uint8_t* vB, int64_t NB, int32_t* match, float* d1, float* d2,
             void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (NA < 0 || NB < 0 || NA > (1ll << 31) - 1 || NB > (1ll << 31) - 1) return fail(c, LP_ERR_ARG, "bad sizes");
    if (NA == 0) return LP_OK;
    if (!dA || !vA || !match || !d1 || !d2 || (NB > 0 && (!dB || !vB))) return fail(c, LP_ERR_ARG, "null argument");
    if (!aligned(dA, 16) || (dB && !aligned(dB, 16))) return fail(c, LP_ERR_ALIGN, "descriptors must be 16-byte aligned");
    lp::MatchArgs a;
    a.dA = dA; a.dA16 = dA_bf16; a.vA = vA; a.NA = NA;
    a.dB = dB; a.dB16 = dB_bf16; a.vB = vB; a.NB = NB;
    a.ratio2 = (float)((double)c->cfg.ratio * (double)c->cfg.ratio);
    const bool ds = c->cfg.delta_s > 0.f && isfinite(c->cfg.delta_s);
    a.delta_s2 = ds ? (float)((double)c->cfg.delta_s * (double)c->cfg.delta_s) : INFINITY;
    a.match = match; a.d1 = d1; a.d2 = d2; a.status = c->d_status;
    c->last = S(stream);
    if (c->prof_ev[0] && NB > 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(S(stream), &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            a.ev0 = c->prof_ev[0];
            a.ev1 = c->prof_ev[1];
            c->prof_recorded = true;
        }
    }
    if (c->cfg.precision == LP_PREC_BF16 || c->cfg.precision == LP_PREC_FP8) {
        const int f8 = c->cfg.precision == LP_PREC_FP8;
        if (!f8 && (!dA_bf16 || (NB > 0 && !dB_bf16)))
            return fail(c, LP_ERR_ARG, "BF16 matching needs the bf16 descriptors");
        if (!f8 && (!aligned(dA_bf16, 16) || (dB_bf16 && !aligned(dB_bf16, 16))))
            return fail(c, LP_ERR_ALIGN, "bf16 alignment");
        a.elem = f8;
        int r;
        if ((r = ensure_fork(c))) return r;
        a.fork = &c->fork;
        if (c->autotune && NB > 0 && (r = tune_match(c, a, S(stream)))) return r;
        r = ensure(c, B_MATCH_WS, lp::match_bf16_workspace(NA, NB, c->num_sms, a.splits, a.elem));
        if (r) return r;
        c->last_S = a.splits;
        c->last_NA = NA;
        c->last_NB = NB;
        LP_CUDA(c, lp::launch_match_bf16(a, c->buf[B_MATCH_WS].p, c->buf[B_MATCH_WS].n, c->num_sms, S(stream)));
        return LP_OK;
    }
    int r = ensure(c, B_MATCH_WS, lp::match_fp32_workspace(NA, NB, c->num_sms));
    if (r) return r;
    LP_CUDA(c, lp::launch_match_fp32(a, c->buf[B_MATCH_WS].p, c->buf[B_MATCH_WS].n, c->num_sms, S(stream)));
    return LP_OK;
}

int lp_compact(lp_ctx* c, const uint32_t* kpA, int WA, const uint32_t* kpB, int WB, const int32_t* match, int64_t NA,
               float* pts, int32_t* rows, int32_t* d_M, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (NA < 0 || WA <= 0 || WB <= 0) return fail(c, LP_ERR_ARG, "bad sizes");
    if (!d_M || (NA > 0 && (!kpA || !kpB || !match || !pts))) return fail(c, LP_ERR_ARG, "null argument");
    if (pts && !aligned(pts, 16)) return fail(c, LP_ERR_ALIGN, "pts must be 16-byte aligned");
    int r = ensure(c, B_COMPACT, lp::compact_workspace(NA));
    if (r) return r;
    c->last = S(stream);
    LP_CUDA(c, lp::launch_compact(kpA, WA, kpB, WB, match, NA, pts, rows, d_M, (int32_t*)c->buf[B_COMPACT].p,
                                  S(stream)));
    return LP_OK;
}

int lp_ransac(lp_ctx* c, const float* pts, int64_t M_cap, const int32_t* d_M, uint32_t pair_id, double* H,
              uint8_t* inlier, int32_t* n_inliers, int32_t* best_t, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (M_cap < 0 || M_cap > (1ll << 31) - 1) return fail(c, LP_ERR_ARG, "bad M_cap");
    if (!H || !n_inliers || (M_cap > 0 && (!pts || !inlier))) return fail(c, LP_ERR_ARG, "null argument");
    if (pts && !aligned(pts, 16)) return fail(c, LP_ERR_ALIGN, "pts must be 16-byte aligned");
    const int T = c->cfg.ransac_iters;
    int r = ensure(c, B_RANSAC_WS, lp::ransac_workspace(M_cap, T));
    if (r) return r;
    c->last = S(stream);
    c->last_ransac_hyps = T;
    LP_CUDA(c, lp::launch_ransac(pts, M_cap, d_M, T, c->cfg.model, c->cfg.thresh_px, c->cfg.seed, pair_id, H, inlier,
                                 n_inliers, best_t, c->buf[B_RANSAC_WS].p, c->buf[B_RANSAC_WS].n, S(stream)));
    return LP_OK;
}

namespace {

// features -> inlier probabilities -> guided RANSAC, for one compacted pair
int guided_tail(lp_ctx* c, const uint32_t* kpA, const uint8_t* oriA, int HA, int WA, const uint32_t* kpB,
                const uint8_t* oriB, int HB, int WB, const int32_t* match, const float* d1, const float* d2,
                const int32_t* rows, float* feat, float* prob, const float* pts, int64_t M_cap, const int32_t* dM,
                uint32_t pair_id, double* H, uint8_t* inl, int32_t* n_in, void* stream)
{
    int r = lp_mlp_features(c, kpA, oriA, HA, WA, kpB, oriB, HB, WB, match, d1, d2, rows, dM, M_cap, feat, stream);
    if (r) return r;
    if ((r = lp_mlp_forward(c->proposal, feat, M_cap, dM, prob, nullptr, stream)))
        return fail(c, r, "lp_mlp_forward failed");
    return lp_ransac_prior(c, pts, M_cap, dM, prob, c->guided_iters, pair_id, H, inl, n_in, nullptr, nullptr, stream);
}

}  // namespace

int lp_set_proposal(lp_ctx* c, lp_mlp* mlp, int32_t guided_iters)
{
    if (!c) return LP_ERR_ARG;
    if (mlp && (guided_iters < 1 || guided_iters > 65536)) return fail(c, LP_ERR_ARG, "guided_iters must be 1..65536");
    c->proposal = mlp;
    c->guided_iters = mlp ? guided_iters : 0;
    return LP_OK;
}

namespace {

// b_queued: image B's upload is already queued on the context's image stream,
// which is ordered after the caller's earlier work (lp_stitch_pair_host)
int stitch_pair_impl(lp_ctx* c, const uint8_t* imgA, int HA, int WA, int pitchA, const uint8_t* imgB, int HB, int WB,
                     int pitchB, int channels, uint32_t pair_id, double* H, int32_t* n_in, int32_t* M_out,
                     void* stream, bool b_queued)
{
    if (!c) return LP_ERR_ARG;
    int r = check_image(c, imgA, HA, WA, pitchA, channels);
    if (!r) r = check_image(c, imgB, HB, WB, pitchB, channels);
    if (r) return r;
    if (!H || !n_in) return fail(c, LP_ERR_ARG, "null output");
    const int64_t KA = lp_num_keypoints(HA, WA, c->cfg.Ls, c->cfg.nL);
    const int64_t KB = lp_num_keypoints(HB, WB, c->cfg.Ls, c->cfg.nL);
    const bool bf = c->cfg.precision == LP_PREC_BF16;
    struct { BufId id; size_t n; } need[] = {
        {B_GRAY_A, channels == 3 ? (size_t)HA * WA + 16 : 0}, {B_GRAY_B, channels == 3 ? (size_t)HB * WB + 16 : 0},
        {B_KP_A, 4 * (size_t)KA}, {B_KP_B, 4 * (size_t)KB}, {B_ORI_A, (size_t)KA}, {B_ORI_B, (size_t)KB},
        {B_DESC_A, 512 * (size_t)KA}, {B_DESC_B, 512 * (size_t)KB},
        {B_D16_A, bf ? 256 * (size_t)KA : 0}, {B_D16_B, bf ? 256 * (size_t)KB : 0},
        {B_VAL_A, (size_t)KA}, {B_VAL_B, (size_t)KB}, {B_MATCH, 4 * (size_t)KA}, {B_D1, 4 * (size_t)KA},
        {B_D2, 4 * (size_t)KA}, {B_PTS, 16 * (size_t)KA}, {B_M, 16}, {B_INL, (size_t)KA}, {B_BEST, 16},
        {B_ROWS, c->proposal ? 4 * (size_t)KA + 16 : 0}, {B_FEAT, c->proposal ? 32 * (size_t)KA + 32 : 0},
        {B_PROB, c->proposal ? 4 * (size_t)KA + 16 : 0}};
    for (auto& q : need)
        if (q.n && (r = ensure(c, q.id, q.n))) return r;
    auto P = [&](BufId id) { return c->buf[id].p; };
    const uint8_t* gA = channels == 3 ? (const uint8_t*)P(B_GRAY_A) : imgA;
    const uint8_t* gB = channels == 3 ? (const uint8_t*)P(B_GRAY_B) : imgB;
    const int gpA = channels == 3 ? WA : pitchA, gpB = channels == 3 ? WB : pitchB;
    // both images' peaks in one launch on the caller's stream (after image B's
    // upload when that is queued on the image stream); then image B's
    // description on the context's image stream beside image A's, joined back
    // before matching
    if ((r = ensure_fork(c))) return r;
    void* sB = c->img_stream;
    if (b_queued) {
        LP_CUDA(c, cudaEventRecord(c->img_ev[0], c->img_stream));
        LP_CUDA(c, cudaStreamWaitEvent(S(stream), c->img_ev[0], 0));
    }
    {
        const lp_image ims[2] = {{imgA, HA, WA, pitchA, channels}, {imgB, HB, WB, pitchB, channels}};
        uint32_t* const kps[2] = {(uint32_t*)P(B_KP_A), (uint32_t*)P(B_KP_B)};
        uint8_t* const grs[2] = {(uint8_t*)P(B_GRAY_A), (uint8_t*)P(B_GRAY_B)};
        if ((r = lp_detect_batch(c, ims, 2, kps, grs, stream))) return r;
    }
    LP_CUDA(c, cudaEventRecord(c->img_ev[0], S(stream)));
    LP_CUDA(c, cudaStreamWaitEvent(c->img_stream, c->img_ev[0], 0));
    if ((r = lp_describe(c, gA, HA, WA, gpA, (const uint32_t*)P(B_KP_A), KA, (uint8_t*)P(B_ORI_A), (float*)P(B_DESC_A),
                         bf ? (uint16_t*)P(B_D16_A) : nullptr, (uint8_t*)P(B_VAL_A), stream)))
        return r;
    if ((r = lp_describe(c, gB, HB, WB, gpB, (const uint32_t*)P(B_KP_B), KB, (uint8_t*)P(B_ORI_B), (float*)P(B_DESC_B),
                         bf ? (uint16_t*)P(B_D16_B) : nullptr, (uint8_t*)P(B_VAL_B), sB)))
        return r;
    LP_CUDA(c, cudaEventRecord(c->img_ev[1], c->img_stream));
    LP_CUDA(c, cudaStreamWaitEvent(S(stream), c->img_ev[1], 0));
    if ((r = lp_match(c, (const float*)P(B_DESC_A), (const uint16_t*)P(B_D16_A), (const uint8_t*)P(B_VAL_A), KA,
                      (const float*)P(B_DESC_B), (const uint16_t*)P(B_D16_B), (const uint8_t*)P(B_VAL_B), KB,
                      (int32_t*)P(B_MATCH), (float*)P(B_D1), (float*)P(B_D2), stream)))
        return r;
    int32_t* dM = M_out ? M_out : (int32_t*)P(B_M);
    if (KA == 0) {
        LP_CUDA(c, cudaMemsetAsync(dM, 0, sizeof(int32_t), S(stream)));
    } else if ((r = lp_compact(c, (const uint32_t*)P(B_KP_A), WA, (const uint32_t*)P(B_KP_B), WB,
                               (const int32_t*)P(B_MATCH), KA, (float*)P(B_PTS),
                               c->proposal ? (int32_t*)P(B_ROWS) : nullptr, dM, stream))) {
        return r;
    }
    if (c->proposal && KA > 0)
        return guided_tail(c, (const uint32_t*)P(B_KP_A), (const uint8_t*)P(B_ORI_A), HA, WA, (const uint32_t*)P(B_KP_B),
                           (const uint8_t*)P(B_ORI_B), HB, WB, (const int32_t*)P(B_MATCH), (const float*)P(B_D1),
                           (const float*)P(B_D2), (int32_t*)P(B_ROWS), (float*)P(B_FEAT), (float*)P(B_PROB),
                           (const float*)P(B_PTS), KA, dM, pair_id, H, (uint8_t*)P(B_INL), n_in, stream);
    return lp_ransac(c, (const float*)P(B_PTS), KA, dM, pair_id, H, (uint8_t*)P(B_INL), n_in, nullptr, stream);
}

}  // namespace

int lp_stitch_pair(lp_ctx* c, const uint8_t* imgA, int HA, int WA, int pitchA, const uint8_t* imgB, int HB, int WB,
                   int pitchB, int channels, uint32_t pair_id, double* H, int32_t* n_in, int32_t* M_out, void* stream)
{
    return stitch_pair_impl(c, imgA, HA, WA, pitchA, imgB, HB, WB, pitchB, channels, pair_id, H, n_in, M_out, stream,
                            false);
}

int lp_stitch_pair_host(lp_ctx* c, const uint8_t* hA, int HA, int WA, int pitchA, const uint8_t* hB, int HB, int WB,
                        int pitchB, int channels, uint32_t pair_id, double* H_host, int32_t* n_in_host,
                        int32_t* M_host, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (!hA || !hB || !H_host || !n_in_host) return fail(c, LP_ERR_ARG, "null argument");
    if (HA <= 0 || HB <= 0 || pitchA % 16 || pitchB % 16) return fail(c, LP_ERR_ALIGN, "pitch must be a multiple of 16");
    int r;
    const size_t nA = (size_t)HA * pitchA, nB = (size_t)HB * pitchB;
    if ((r = ensure(c, B_IMG_A, nA)) || (r = ensure(c, B_IMG_B, nB)) || (r = ensure(c, B_H, 128)) ||
        (r = ensure(c, B_NIN, 64)))
        return r;
    if ((r = ensure_fork(c))) return r;
    cudaStream_t s = S(stream);
    c->last = s;
    // A uploads on the caller's stream, B on the image stream (after the
    // caller's earlier work): the two copies and image A's detection overlap
    LP_CUDA(c, cudaEventRecord(c->img_ev[0], s));
    LP_CUDA(c, cudaStreamWaitEvent(c->img_stream, c->img_ev[0], 0));
    LP_CUDA(c, cudaMemcpyAsync(c->buf[B_IMG_A].p, hA, nA, cudaMemcpyHostToDevice, s));
    LP_CUDA(c, cudaMemcpyAsync(c->buf[B_IMG_B].p, hB, nB, cudaMemcpyHostToDevice, c->img_stream));
    double* dH = (double*)c->buf[B_H].p;
    int32_t* dn = (int32_t*)c->buf[B_NIN].p;
    if ((r = stitch_pair_impl(c, (const uint8_t*)c->buf[B_IMG_A].p, HA, WA, pitchA, (const uint8_t*)c->buf[B_IMG_B].p,
                              HB, WB, pitchB, channels, pair_id, dH, dn, dn + 1, stream, true)))
        return r;
    int32_t tmp[2];
    LP_CUDA(c, cudaMemcpyAsync(H_host, dH, 9 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LP_CUDA(c, cudaMemcpyAsync(tmp, dn, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LP_CUDA(c, cudaStreamSynchronize(s));
    *n_in_host = tmp[0];
    if (M_host) *M_host = tmp[1];
    return LP_OK;
}

int lp_stitch_pairs_host(lp_ctx* c, const lp_host_pair* pairs, int P, int channels, uint32_t pair_id0,
                         double* H_host, int32_t* n_in_host, int32_t* M_host, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (P < 0 || (P > 0 && (!pairs || !H_host || !n_in_host))) return fail(c, LP_ERR_ARG, "null argument or P < 0");
    if (P == 0) return LP_OK;
    size_t nA = 16, nB = 16;
    for (int q = 0; q < P; ++q) {
        const lp_host_pair& h = pairs[q];
        if (!h.A || !h.B) return fail(c, LP_ERR_ARG, "null image of pair %d", q);
        if (h.HA <= 0 || h.HB <= 0 || h.pitchA % 16 || h.pitchB % 16)
            return fail(c, LP_ERR_ALIGN, "pair %d: pitch must be a multiple of 16", q);
        nA = std::max(nA, (size_t)h.HA * h.pitchA);
        nB = std::max(nB, (size_t)h.HB * h.pitchB);
    }
    int r;
    if ((r = ensure(c, B_IMG_A, nA)) || (r = ensure(c, B_IMG_B, nB)) || (r = ensure(c, B_IMG_A1, nA)) ||
        (r = ensure(c, B_IMG_B1, nB)) || (r = ensure(c, B_HSTREAM, (size_t)P * (9 * sizeof(double) + 8) + 64)) ||
        (r = ensure_fork(c)))
        return r;
    if (!c->copy_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaEventCreateWithFlags(&c->up_ev[k], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->free_ev[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->start_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LP_ERR_CUDA, "upload stream: %s", cudaGetErrorString(e));
        }
    }
    cudaStream_t s = S(stream), cs = c->copy_stream;
    c->last = s;
    double* dH = (double*)c->buf[B_HSTREAM].p;
    int32_t* dn = (int32_t*)(dH + 9 * (size_t)P);
    void* slotA[2] = {c->buf[B_IMG_A].p, c->buf[B_IMG_A1].p};
    void* slotB[2] = {c->buf[B_IMG_B].p, c->buf[B_IMG_B1].p};
    // uploads start after the caller's earlier work on its stream
    LP_CUDA(c, cudaEventRecord(c->start_ev, s));
    LP_CUDA(c, cudaStreamWaitEvent(cs, c->start_ev, 0));
    for (int q = 0; q < P; ++q) {
        const lp_host_pair& h = pairs[q];
        const int k = q & 1;
        // slot k is free once pair q - 2 is done
        if (q >= 2) LP_CUDA(c, cudaStreamWaitEvent(cs, c->free_ev[k], 0));
        LP_CUDA(c, cudaMemcpyAsync(slotA[k], h.A, (size_t)h.HA * h.pitchA, cudaMemcpyHostToDevice, cs));
        LP_CUDA(c, cudaMemcpyAsync(slotB[k], h.B, (size_t)h.HB * h.pitchB, cudaMemcpyHostToDevice, cs));
        LP_CUDA(c, cudaEventRecord(c->up_ev[k], cs));
        LP_CUDA(c, cudaStreamWaitEvent(s, c->up_ev[k], 0));
        if ((r = stitch_pair_impl(c, (const uint8_t*)slotA[k], h.HA, h.WA, h.pitchA, (const uint8_t*)slotB[k], h.HB,
                                  h.WB, h.pitchB, channels, pair_id0 + (uint32_t)q, dH + 9 * (size_t)q,
                                  dn + 2 * (size_t)q, dn + 2 * (size_t)q + 1, stream, false)))
            return r;
        LP_CUDA(c, cudaEventRecord(c->free_ev[k], s));
    }
    std::vector<int32_t> tmp(2 * (size_t)P);
    LP_CUDA(c, cudaMemcpyAsync(H_host, dH, 9 * sizeof(double) * (size_t)P, cudaMemcpyDeviceToHost, s));
    LP_CUDA(c, cudaMemcpyAsync(tmp.data(), dn, 2 * sizeof(int32_t) * (size_t)P, cudaMemcpyDeviceToHost, s));
    LP_CUDA(c, cudaStreamSynchronize(s));
    for (int q = 0; q < P; ++q) {
        n_in_host[q] = tmp[2 * (size_t)q];
        if (M_host) M_host[q] = tmp[2 * (size_t)q + 1];
    }
    return LP_OK;
}

namespace {

__global__ void k_pair_valid(const int32_t* n_in, int P, int min_inl, uint8_t* valid)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) valid[p] = n_in[p] >= min_inl ? 1 : 0;
}

struct ImgBufs {
    size_t gray, kp, ori, desc, d16, val;
    int64_t K;
};

}  // namespace

int lp_stitch_pairs(lp_ctx* c, const lp_image* imgs, int N, const int32_t* pairs, int P, double* HM, int32_t* n_in,
                    uint8_t* valid, int32_t* M_out, void* stream)
{
    return lp_stitch_pairs_ids(c, imgs, N, pairs, nullptr, P, HM, n_in, valid, M_out, stream);
}

int lp_stitch_pairs_ids(lp_ctx* c, const lp_image* imgs, int N, const int32_t* pairs, const uint32_t* pair_ids, int P,
                        double* HM, int32_t* n_in, uint8_t* valid, int32_t* M_out, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (pair_ids && !pairs) return fail(c, LP_ERR_ARG, "pair_ids need an explicit pair list");
    if (!imgs || N < 2) return fail(c, LP_ERR_ARG, "need at least two images");
    if (!HM || !n_in || !valid) return fail(c, LP_ERR_ARG, "null output");
    const int ch = imgs[0].channels;
    for (int i = 0; i < N; ++i) {
        int r = check_image(c, imgs[i].data, imgs[i].H, imgs[i].W, imgs[i].pitch, imgs[i].channels);
        if (r) return r;
        if (imgs[i].channels != ch) return fail(c, LP_ERR_ARG, "images differ in channel count");
    }
    std::vector<int32_t> pl;
    if (!pairs) {
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) { pl.push_back(i); pl.push_back(j); }
        P = N * (N - 1) / 2;
    } else {
        if (P < 1) return fail(c, LP_ERR_ARG, "P=%d", P);
        pl.assign(pairs, pairs + 2 * (size_t)P);
        for (int q = 0; q < 2 * P; ++q)
            if (pl[q] < 0 || pl[q] >= N) return fail(c, LP_ERR_ARG, "pair index %d outside 0..%d", pl[q], N - 1);
    }
    // ---- plan: per-image feature buffers in one block, per-pair scratch reused
    const bool bf = c->cfg.precision == LP_PREC_BF16;
    std::vector<ImgBufs> ib(N);
    size_t o = 0;
    int64_t Kmax = 0;
    for (int i = 0; i < N; ++i) {
        const int64_t K = lp_num_keypoints(imgs[i].H, imgs[i].W, c->cfg.Ls, c->cfg.nL);
        ib[i].K = K;
        Kmax = std::max(Kmax, K);
        ib[i].gray = o; o += ch == 3 ? al256((size_t)imgs[i].H * imgs[i].W + 16) : 0;
        ib[i].kp = o; o += al256(4 * (size_t)K + 8);
        ib[i].ori = o; o += al256((size_t)K + 8);
        ib[i].desc = o; o += al256(512 * (size_t)K + 16);
        ib[i].d16 = o; o += bf ? al256(256 * (size_t)K + 16) : 0;
        ib[i].val = o; o += al256((size_t)K + 8);
    }
    // kLanes slots of match outputs, compacted points, inlier masks and RANSAC
    // workspace: pair q's RANSAC (and, with the learned proposal, its features,
    // forward pass and guided RANSAC) runs on lane q % kLanes -- the context's
    // image stream and its two auxiliary streams -- beside the next pairs'
    // matching tails and each other's RANSAC
    constexpr int kLanes = 3;
    const bool guided = c->proposal != nullptr;
    const int Ttot = c->cfg.ransac_iters + (guided ? c->guided_iters : 0);
    const size_t row_slot = al256(4 * (size_t)Kmax + 8);
    const size_t o_match = o; o += kLanes * row_slot;
    const size_t o_d1 = o; o += kLanes * row_slot;
    const size_t o_d2 = o; o += kLanes * row_slot;
    const size_t pts_slot = al256(16 * (size_t)Kmax + 16), inl_slot = al256((size_t)Kmax + 8);
    const size_t o_pts = o; o += kLanes * pts_slot;
    const size_t o_inl = o; o += kLanes * inl_slot;
    const size_t o_M = o; o += al256(4 * (size_t)P + 8);
    const size_t o_rows = o; o += guided ? kLanes * row_slot : 0;
    const size_t feat_slot = guided ? al256(32 * (size_t)Kmax + 32) : 0;
    const size_t o_feat = o; o += kLanes * feat_slot;
    const size_t o_prob = o; o += guided ? kLanes * row_slot : 0;
    const size_t rws_slot = al256(lp::ransac_workspace(Kmax, Ttot));
    const size_t o_rws = o; o += kLanes * rws_slot;
    const size_t pre_slot = guided ? al256(sizeof(unsigned long long) * (size_t)(Kmax + 1)) : 0;
    const size_t o_pre = o; o += kLanes * pre_slot;
    // BF16: the distance passes of every pair run first, in persistent launches
    // over all pairs (k_match_tc_batch); each pair then keeps its thresholds and
    // candidate lists in a workspace of its own until its tail (re-rank,
    // re-scan, finish) runs in the pair loop.  Row norms once per image.
    std::vector<lp::MatchArgs> margs(bf ? (size_t)P : 0);
    std::vector<size_t> o_pws(bf ? (size_t)P : 0), pws_bytes(bf ? (size_t)P : 0);
    std::vector<size_t> o_norm(bf ? (size_t)N : 0);
    size_t o_sync = 0;
    if (bf) {
        for (int i = 0; i < N; ++i) { o_norm[i] = o; o += al256(4 * (size_t)ib[i].K + 8); }
        for (int q = 0; q < P; ++q) {
            const ImgBufs &A = ib[pl[2 * q]], &B = ib[pl[2 * q + 1]];
            lp::MatchArgs& a = margs[q];
            a.NA = A.K;
            a.NB = B.K;
            a.splits = tuned_splits(c, A.K, B.K, &a.pass1_stride);
            pws_bytes[q] = lp::match_bf16_workspace(A.K, B.K, c->num_sms, a.splits);
            o_pws[q] = o;
            o += al256(pws_bytes[q]);
        }
        o_sync = o;
        o += al256(4 * lp::match_bf16_batch_sync_words(margs.data(), P) + 8);
    }
    int r = ensure(c, B_BATCH, o + 256);
    if (r) return r;
    if ((r = ensure_fork(c))) return r;
    size_t mws = 0;
    for (int q = 0; q < P; ++q) {
        const int64_t KA = ib[pl[2 * q]].K, KB = ib[pl[2 * q + 1]].K;
        if (!bf)
            mws = std::max(mws, c->cfg.precision == LP_PREC_FP8 ? lp::match_bf16_workspace(KA, KB, c->num_sms, 0, 1)
                                                                 : lp::match_fp32_workspace(KA, KB, c->num_sms));
    }
    if ((r = ensure(c, B_MATCH_WS, std::max<size_t>(mws, 256))) ||
        (r = ensure(c, B_COMPACT, lp::compact_workspace(Kmax))))
        return r;
    cudaStream_t s = S(stream);
    if (!c->luts_ready && (r = build_luts(c, s))) return r;
    uint8_t* base = reinterpret_cast<uint8_t*>(al256(reinterpret_cast<uintptr_t>(c->buf[B_BATCH].p)));
    int32_t* Mbuf = M_out ? M_out : reinterpret_cast<int32_t*>(base + o_M);

    std::vector<long long> key = {N, P, ch, c->batch_hold, c->autotune ? (long long)c->tune.size() : -1ll,
                                  (long long)(uintptr_t)HM, (long long)(uintptr_t)n_in,
                                  (long long)(uintptr_t)valid, (long long)(uintptr_t)Mbuf,
                                  (long long)(uintptr_t)c->buf[B_BATCH].p, (long long)(uintptr_t)c->buf[B_MATCH_WS].p,
                                  (long long)(uintptr_t)c->buf[B_RANSAC_WS].p,
                                  (long long)(uintptr_t)c->proposal, c->guided_iters,
                                  (long long)(uintptr_t)c->buf[B_PREFIX].p,
                                  (long long)(uintptr_t)c->buf[B_COMPACT].p};
    for (int i = 0; i < N; ++i) {
        key.push_back((long long)(uintptr_t)imgs[i].data);
        key.push_back(imgs[i].H); key.push_back(imgs[i].W); key.push_back(imgs[i].pitch);
    }
    key.insert(key.end(), pl.begin(), pl.end());
    std::vector<uint32_t> pid((size_t)P);
    for (int q = 0; q < P; ++q) pid[q] = pair_ids ? pair_ids[q] : (uint32_t)q;
    key.insert(key.end(), pid.begin(), pid.end());
    c->last = s;
    if (s && c->graph_exec && key == c->graph_key) {
        LP_CUDA(c, cudaGraphLaunch(c->graph_exec, s));
        return LP_OK;
    }

    auto enqueue = [&]() -> int {
        int rr;
        {
            std::vector<uint32_t*> kps((size_t)N);
            std::vector<uint8_t*> grays((size_t)N);
            for (int i = 0; i < N; ++i) {
                kps[i] = (uint32_t*)(base + ib[i].kp);
                grays[i] = ch == 3 ? base + ib[i].gray : nullptr;
            }
            if ((rr = lp_detect_batch(c, imgs, N, kps.data(), grays.data(), stream))) return rr;
        }
        for (int i = 0; i < N; ++i) {
            uint8_t* g = ch == 3 ? base + ib[i].gray : nullptr;
            const uint8_t* gsrc = ch == 3 ? g : imgs[i].data;
            const int gp = ch == 3 ? imgs[i].W : imgs[i].pitch;
            if ((rr = lp_describe(c, gsrc, imgs[i].H, imgs[i].W, gp, (const uint32_t*)(base + ib[i].kp), ib[i].K,
                                  base + ib[i].ori, (float*)(base + ib[i].desc),
                                  bf ? (uint16_t*)(base + ib[i].d16) : nullptr, base + ib[i].val, stream)))
                return rr;
        }
        if (bf) {
            // row norms once per image, then the distance passes of every pair
            const float ratio2 = (float)((double)c->cfg.ratio * (double)c->cfg.ratio);
            const bool ds = c->cfg.delta_s > 0.f && isfinite(c->cfg.delta_s);
            const float delta_s2 = ds ? (float)((double)c->cfg.delta_s * (double)c->cfg.delta_s) : INFINITY;
            for (int i = 0; i < N; ++i)
                LP_CUDA(c, lp::launch_row_norms((const float*)(base + ib[i].desc), base + ib[i].val, ib[i].K,
                                                (float*)(base + o_norm[i]), s));
            std::vector<void*> wsp((size_t)P);
            for (int q = 0; q < P; ++q) {
                const int a_ = pl[2 * q], b_ = pl[2 * q + 1];
                lp::MatchArgs& a = margs[q];
                a.dA = (const float*)(base + ib[a_].desc);
                a.dA16 = (const uint16_t*)(base + ib[a_].d16);
                a.vA = base + ib[a_].val;
                a.dB = (const float*)(base + ib[b_].desc);
                a.dB16 = (const uint16_t*)(base + ib[b_].d16);
                a.vB = base + ib[b_].val;
                a.ratio2 = ratio2;
                a.delta_s2 = delta_s2;
                a.status = c->d_status;
                a.normA = (const float*)(base + o_norm[a_]);
                a.normB = (const float*)(base + o_norm[b_]);
                wsp[q] = base + o_pws[q];
            }
            LP_CUDA(c, lp::launch_match_bf16_batch(margs.data(), wsp.data(), pws_bytes.data(), P,
                                                   (int32_t*)(base + o_sync), c->batch_hold, c->num_sms, s));
        }
        // lanes: pair q's RANSAC on stream rs[q % kLanes]; the lane's slot of
        // buffers is reused by pair q + kLanes only after that RANSAC ended
        cudaStream_t rs[kLanes] = {c->img_stream, c->fork.aux[0], c->fork.aux[1]};
        LP_CUDA(c, cudaEventRecord(c->pair_ev[0], s));
        for (int k = 0; k < kLanes; ++k) {
            LP_CUDA(c, cudaStreamWaitEvent(rs[k], c->pair_ev[0], 0));
            LP_CUDA(c, cudaEventRecord(c->pair_ev[1 + k], s));
        }
        for (int q = 0; q < P; ++q) {
            const int a = pl[2 * q], b = pl[2 * q + 1];
            const ImgBufs &A = ib[a], &B = ib[b];
            const int slot = q % kLanes;
            cudaStream_t sr = rs[slot];
            float* pts = (float*)(base + o_pts + slot * pts_slot);
            uint8_t* inl = base + o_inl + slot * inl_slot;
            float* feat = (float*)(base + o_feat + slot * feat_slot);
            int32_t* mt = (int32_t*)(base + o_match + slot * row_slot);
            float* d1 = (float*)(base + o_d1 + slot * row_slot);
            float* d2 = (float*)(base + o_d2 + slot * row_slot);
            int32_t* rows = guided ? (int32_t*)(base + o_rows + slot * row_slot) : nullptr;
            float* prob = guided ? (float*)(base + o_prob + slot * row_slot) : nullptr;
            void* rws = base + o_rws + slot * rws_slot;
            auto* pre = guided ? reinterpret_cast<unsigned long long*>(base + o_pre + slot * pre_slot) : nullptr;
            // the slot's previous RANSAC (pair q - kLanes) has finished reading it
            LP_CUDA(c, cudaStreamWaitEvent(s, c->pair_ev[1 + slot], 0));
            if (A.K == 0) {
                LP_CUDA(c, cudaMemsetAsync(Mbuf + q, 0, sizeof(int32_t), s));
            } else {
                if (bf) {
                    lp::MatchArgs ma = margs[q];
                    ma.match = mt;
                    ma.d1 = d1;
                    ma.d2 = d2;
                    LP_CUDA(c, lp::launch_match_bf16_tail(ma, base + o_pws[q], pws_bytes[q], c->num_sms, s));
                } else if ((rr = lp_match(c, (const float*)(base + A.desc), nullptr, base + A.val, A.K,
                                          (const float*)(base + B.desc), nullptr, base + B.val, B.K, mt, d1, d2,
                                          stream))) {
                    return rr;
                }
                if ((rr = lp_compact(c, (const uint32_t*)(base + A.kp), imgs[a].W, (const uint32_t*)(base + B.kp),
                                     imgs[b].W, mt, A.K, pts, rows, Mbuf + q, stream)))
                    return rr;
            }
            LP_CUDA(c, cudaEventRecord(c->pair_ev[0], s));
            LP_CUDA(c, cudaStreamWaitEvent(sr, c->pair_ev[0], 0));
            if (guided && A.K > 0) {
                if ((rr = lp_mlp_features(c, (const uint32_t*)(base + A.kp), base + A.ori, imgs[a].H, imgs[a].W,
                                          (const uint32_t*)(base + B.kp), base + B.ori, imgs[b].H, imgs[b].W, mt, d1,
                                          d2, rows, Mbuf + q, A.K, feat, sr)))
                    return rr;
                if ((rr = lp_mlp_forward(c->proposal, feat, A.K, Mbuf + q, prob, nullptr, sr)))
                    return fail(c, rr, "lp_mlp_forward failed");
                LP_CUDA(c, lp::launch_guided_prefix(prob, A.K, Mbuf + q, pre, sr));
                LP_CUDA(c, lp::launch_ransac_prior(pts, A.K, Mbuf + q, pre, c->guided_iters, c->cfg.ransac_iters,
                                                   c->cfg.model, c->cfg.thresh_px, c->cfg.seed, pid[q],
                                                   c->cfg.min_inliers, HM + 9 * (size_t)q, inl, n_in + q, nullptr,
                                                   nullptr, rws, rws_slot, sr));
            } else {
                LP_CUDA(c, lp::launch_ransac(pts, A.K, Mbuf + q, c->cfg.ransac_iters, c->cfg.model, c->cfg.thresh_px,
                                             c->cfg.seed, pid[q], HM + 9 * (size_t)q, inl, n_in + q, nullptr, rws,
                                             rws_slot, sr));
            }
            LP_CUDA(c, cudaEventRecord(c->pair_ev[1 + slot], sr));
        }
        for (int k = 0; k < kLanes; ++k) LP_CUDA(c, cudaStreamWaitEvent(s, c->pair_ev[1 + k], 0));
        c->last = s;
        k_pair_valid<<<(P + 127) / 128, 128, 0, s>>>(n_in, P, c->cfg.min_inliers, valid);
        LP_CUDA(c, cudaGetLastError());
        return LP_OK;
    };
    // first call for this key: run eagerly, then record the same sequence as a
    // graph for later calls (not on the legacy default stream)
    if ((r = enqueue())) return r;
    if (bf && c->autotune) {
        // a size class met for the first time is tuned on this call's own
        // descriptors, which stay in the batch buffer after the call; the next
        // call lays its pairs out with the tuned choice (and records its graph)
        const size_t n0 = c->tune.size();
        for (int q = 0; q < P; ++q) {
            int st = 0;
            if (margs[q].NA == 0 || margs[q].NB == 0 || tuned_splits(c, margs[q].NA, margs[q].NB, &st)) continue;
            lp::MatchArgs a = margs[q];
            a.match = (int32_t*)(base + o_match);
            a.d1 = (float*)(base + o_d1);
            a.d2 = (float*)(base + o_d2);
            a.normA = a.normB = nullptr;
            a.fork = &c->fork;
            a.ev0 = a.ev1 = nullptr;
            a.splits = a.pass1_stride = 0;
            if ((r = tune_match(c, a, s))) return r;
        }
        if (c->tune.size() != n0) return LP_OK;
    }
    if (s) {
        if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
        c->graph_key.clear();
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int er = enqueue();
            const cudaError_t ee = cudaStreamEndCapture(s, &g);
            if (er == LP_OK && ee == cudaSuccess && g) {
                if (cudaGraphInstantiate(&c->graph_exec, g, 0) == cudaSuccess) c->graph_key = key;
                else c->graph_exec = nullptr;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    return LP_OK;
}

int lp_ransac_prior(lp_ctx* c, const float* pts, int64_t M_cap, const int32_t* d_M, const float* prior,
                    int32_t guided_iters, uint32_t pair_id, double* H, uint8_t* inlier, int32_t* n_inliers,
                    int32_t* best_t, int32_t* iters_used, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (M_cap < 0 || M_cap > (1ll << 31) - 1) return fail(c, LP_ERR_ARG, "bad M_cap");
    if (guided_iters < 1 || guided_iters > 65536) return fail(c, LP_ERR_ARG, "guided_iters must be 1..65536");
    if (!H || !n_inliers || (M_cap > 0 && (!pts || !inlier || !prior))) return fail(c, LP_ERR_ARG, "null argument");
    if (pts && !aligned(pts, 16)) return fail(c, LP_ERR_ALIGN, "pts must be 16-byte aligned");
    const int T = c->cfg.ransac_iters, Ttot = guided_iters + T;
    int r = ensure(c, B_RANSAC_WS, lp::ransac_workspace(M_cap, Ttot));
    if (!r) r = ensure(c, B_PREFIX, sizeof(unsigned long long) * (size_t)(M_cap + 1));
    if (r) return r;
    c->last = S(stream);
    c->last_ransac_hyps = Ttot;
    auto* pre = static_cast<unsigned long long*>(c->buf[B_PREFIX].p);
    LP_CUDA(c, lp::launch_guided_prefix(prior, M_cap, d_M, pre, S(stream)));
    LP_CUDA(c, lp::launch_ransac_prior(pts, M_cap, d_M, pre, guided_iters, T, c->cfg.model, c->cfg.thresh_px,
                                       c->cfg.seed, pair_id, c->cfg.min_inliers, H, inlier, n_inliers, best_t,
                                       iters_used,
                                       c->buf[B_RANSAC_WS].p,
                                       c->buf[B_RANSAC_WS].n, S(stream)));
    return LP_OK;
}

int lp_diag_last_ransac_counts(lp_ctx* c, int32_t* host_counts, int n)
{
    if (!c || !host_counts || n != c->last_ransac_hyps || n <= 0 || !c->buf[B_RANSAC_WS].p) return LP_ERR_ARG;
    LP_CUDA(c, lp::ransac_counts(c->buf[B_RANSAC_WS].p, n, host_counts, c->last));
    return LP_OK;
}

int lp_mlp_features(lp_ctx* c, const uint32_t* kpA, const uint8_t* oriA, int HA, int WA, const uint32_t* kpB,
                    const uint8_t* oriB, int HB, int WB, const int32_t* match, const float* d1, const float* d2,
                    const int32_t* rows, const int32_t* d_M, int64_t M_cap, float* feat, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (M_cap < 0 || HA <= 0 || WA <= 0 || HB <= 0 || WB <= 0) return fail(c, LP_ERR_ARG, "bad sizes");
    if (M_cap > 0 && (!kpA || !oriA || !kpB || !oriB || !match || !d1 || !d2 || !rows || !feat))
        return fail(c, LP_ERR_ARG, "null argument");
    lp::ScaleTable st;
    lp::make_scale_table(c->cfg.Ls, c->cfg.nL, c->cfg.beta0, HA, WA, &st);
    lp::MlpScales sc;
    sc.nL = st.nL;
    for (int l = 0; l <= st.nL; ++l) sc.off[l] = st.off[l];
    for (int l = 0; l < st.nL; ++l) sc.log2L[l] = (float)log2((double)st.L[l]);
    sc.log2Lmax = (float)log2((double)st.L[st.nL - 1]);
    c->last = S(stream);
    LP_CUDA(c, lp::launch_mlp_features(kpA, oriA, HA, WA, kpB, oriB, HB, WB, match, d1, d2, rows, d_M, M_cap, sc,
                                       feat, S(stream)));
    return LP_OK;
}

int lp_mosaic_render(lp_ctx* c, const lp_image* imgs, int N, const double* G, const int32_t* round_of,
                     uint8_t* canvas, int canvas_w, int canvas_h, int canvas_pitch, uint8_t* cover, void* stream)
{
    if (!c) return LP_ERR_ARG;
    if (!imgs || N < 1 || !G || !round_of || canvas_w < 0 || canvas_h < 0) return fail(c, LP_ERR_ARG, "bad arguments");
    const int ch = imgs[0].channels;
    for (int i = 0; i < N; ++i) {
        if (round_of[i] < 0) continue;
        int r = check_image(c, imgs[i].data, imgs[i].H, imgs[i].W, imgs[i].pitch, imgs[i].channels);
        if (r) return r;
        if (imgs[i].channels != ch) return fail(c, LP_ERR_ARG, "images differ in channel count");
    }
    if (canvas_w > 0 && canvas_h > 0 && (!canvas || canvas_pitch < canvas_w * ch))
        return fail(c, LP_ERR_ARG, "canvas pointer or pitch");
    c->last = S(stream);
    int bad = 0;
    LP_CUDA(c, lp::launch_mosaic_render(imgs, N, G, round_of, canvas, canvas_w, canvas_h, canvas_pitch, cover,
                                        S(stream), &bad));
    if (bad) return fail(c, LP_ERR_ARG, "more than 64 images or a singular placement");
    return LP_OK;
}

int lp_diag_set_batch_hold(lp_ctx* c, int32_t hold)
{
    if (!c) return LP_ERR_ARG;
    if (hold < 0) return fail(c, LP_ERR_ARG, "hold must be >= 0");
    c->batch_hold = hold;
    return LP_OK;
}

int lp_set_autotune(lp_ctx* c, int32_t on)
{
    if (!c) return LP_ERR_ARG;
    c->autotune = on != 0;
    return LP_OK;
}

int lp_autotune_table(lp_ctx* c, int32_t* rows, int32_t cap, int32_t* n)
{
    if (!c) return LP_ERR_ARG;
    if (!n || cap < 0 || (cap > 0 && !rows)) return fail(c, LP_ERR_ARG, "null argument");
    *n = (int32_t)c->tune.size();
    for (int32_t k = 0; k < cap && k < *n; ++k) {
        const auto& e = c->tune[(size_t)k];
        int32_t* r = rows + 6 * (size_t)k;
        r[0] = e.ba; r[1] = e.bb; r[2] = e.S; r[3] = e.stride;
        r[4] = (int32_t)lrintf(e.us); r[5] = (int32_t)lrintf(e.us_builtin);
    }
    return LP_OK;
}

int lp_set_profiling(lp_ctx* c, int on)
{
    if (!c) return LP_ERR_ARG;
    if (on && !c->prof_ev[0]) {
        if (cudaEventCreate(&c->prof_ev[0]) != cudaSuccess || cudaEventCreate(&c->prof_ev[1]) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, LP_ERR_CUDA, "cudaEventCreate failed");
        }
    } else if (!on && c->prof_ev[0]) {
        cudaEventSynchronize(c->prof_ev[1]);
        cudaEventDestroy(c->prof_ev[0]);
        cudaEventDestroy(c->prof_ev[1]);
        c->prof_ev[0] = c->prof_ev[1] = nullptr;
    }
    c->prof_recorded = false;
    return LP_OK;
}

int lp_diag_last_match_kernel_ms(lp_ctx* c, float* ms)
{
    if (!c || !ms) return LP_ERR_ARG;
    if (!c->prof_ev[0] || !c->prof_recorded) return fail(c, LP_ERR_ARG, "no profiled lp_match call");
    LP_CUDA(c, cudaEventSynchronize(c->prof_ev[1]));
    LP_CUDA(c, cudaEventElapsedTime(ms, c->prof_ev[0], c->prof_ev[1]));
    return LP_OK;
}

int lp_sync_status(lp_ctx* c)
{
    if (!c) return LP_ERR_ARG;
    if (c->last) LP_CUDA(c, cudaStreamSynchronize(c->last));
    else LP_CUDA(c, cudaDeviceSynchronize());
    int32_t st = 0;
    LP_CUDA(c, cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost));
    LP_CUDA(c, cudaMemset(c->d_status, 0, sizeof st));
    return st;
}

const char* lp_last_error(lp_ctx* c) { return c ? c->err : "null context"; }

int lp_diag_last_rescans(lp_ctx* c, int64_t* out)
{
    if (!c || !out) return LP_ERR_ARG;
    *out = 0;
    if ((c->cfg.precision != LP_PREC_BF16 && c->cfg.precision != LP_PREC_FP8) || !c->buf[B_MATCH_WS].p ||
        c->last_NA == 0)
        return LP_OK;
    *out = lp::match_bf16_rescans(c->buf[B_MATCH_WS].p, c->last_NA, c->last_NB, c->num_sms, c->last_S, c->last);
    return *out < 0 ? LP_ERR_CUDA : LP_OK;
}

int lp_diag_orient_bins(int32_t* out, void* stream)
{
    if (!out) return LP_ERR_ARG;
    return lp::launch_diag_orient(out, nullptr, S(stream)) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

int lp_diag_orient_weights(uint32_t* out, void* stream)
{
    if (!out) return LP_ERR_ARG;
    return lp::launch_diag_orient(nullptr, out, S(stream)) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

int lp_diag_philox(const uint32_t* ctr, int64_t n, uint32_t key0, uint32_t key1, uint32_t* out, void* stream)
{
    if ((n > 0 && (!ctr || !out)) || n < 0) return LP_ERR_ARG;
    if (!aligned(ctr, 16) || !aligned(out, 16)) return LP_ERR_ALIGN;
    return lp::launch_diag_philox(ctr, n, key0, key1, out, S(stream)) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

int lp_diag_gray(const uint8_t* rgb, int64_t n, uint8_t* gray, void* stream)
{
    if (n < 0 || (n > 0 && (!rgb || !gray))) return LP_ERR_ARG;
    if (n == 0) return LP_OK;
    return lp::launch_diag_gray(rgb, n, gray, S(stream)) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}


namespace {

uint64_t splitmix64(uint64_t& x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int mlp_upload(lp_mlp* m, const float* host)
{
    std::vector<float> zero(LP_MLP_PARAMS, 0.f);
    if (cudaMemcpy(m->master, host, sizeof(float) * LP_MLP_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->m, zero.data(), sizeof(float) * LP_MLP_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->v, zero.data(), sizeof(float) * LP_MLP_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess ||
        lp::launch_mlp_shadow(m->master, m->shadow, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return LP_ERR_CUDA;
    m->step = 0;
    return LP_OK;
}

}  // namespace

int lp_mlp_create(lp_mlp** out, uint64_t seed)
{
    if (!out) return LP_ERR_ARG;
    *out = nullptr;
    lp_mlp* m = new lp_mlp();
    if (cudaGetDevice(&m->device) != cudaSuccess || cudaMalloc(&m->master, sizeof(float) * 4 * LP_MLP_PARAMS) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return LP_ERR_CUDA;
    }
    m->m = m->master + LP_MLP_PARAMS;
    m->v = m->m + LP_MLP_PARAMS;
    m->shadow = m->v + LP_MLP_PARAMS;
    // He-uniform: U(-sqrt(6 / fan_in), +sqrt(6 / fan_in)), zero biases
    std::vector<float> h(LP_MLP_PARAMS, 0.f);
    uint64_t st = seed;
    auto uni = [&](double a) { return (float)(a * (2.0 * ((splitmix64(st) >> 11) * 0x1.0p-53) - 1.0)); };
    for (int i = 0; i < 512; ++i) h[i] = uni(sqrt(6.0 / 8.0));
    for (int i = 576; i < 4672; ++i) h[i] = uni(sqrt(6.0 / 64.0));
    for (int i = 4736; i < 4800; ++i) h[i] = uni(sqrt(6.0 / 64.0));
    int r = mlp_upload(m, h.data());
    if (r) { cudaFree(m->master); delete m; return r; }
    *out = m;
    return LP_OK;
}

int lp_mlp_destroy(lp_mlp* m)
{
    if (!m) return LP_ERR_ARG;
    cudaDeviceSynchronize();
    cudaFree(m->master);
    if (m->part) cudaFree(m->part);
    delete m;
    return LP_OK;
}

int lp_mlp_set_params(lp_mlp* m, const float* host)
{
    if (!m || !host) return LP_ERR_ARG;
    return mlp_upload(m, host);
}

int lp_mlp_get_params(lp_mlp* m, float* host)
{
    if (!m || !host) return LP_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(host, m->master, sizeof(float) * LP_MLP_PARAMS, cudaMemcpyDeviceToHost) != cudaSuccess)
        return LP_ERR_CUDA;
    return LP_OK;
}

int lp_mlp_get_state(lp_mlp* m, float* host, int32_t* step)
{
    if (!m || !host) return LP_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(host, m->master, sizeof(float) * 3 * LP_MLP_PARAMS, cudaMemcpyDeviceToHost) != cudaSuccess)
        return LP_ERR_CUDA;
    if (step) *step = m->step;
    return LP_OK;
}

int lp_mlp_save(lp_mlp* m, const char* path)
{
    if (!m || !path) return LP_ERR_ARG;
    std::vector<float> h(3 * LP_MLP_PARAMS);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h.data(), m->master, sizeof(float) * 3 * LP_MLP_PARAMS, cudaMemcpyDeviceToHost) != cudaSuccess)
        return LP_ERR_CUDA;
    FILE* f = fopen(path, "wb");
    if (!f) return LP_ERR_ARG;
    const char magic[8] = {'L', 'P', 'M', 'L', 'P', '0', '0', '1'};
    const int32_t hdr[2] = {LP_MLP_PARAMS, m->step};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof hdr, 1, f) == 1 &&
              fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? LP_OK : LP_ERR_ARG;
}

int lp_mlp_load(lp_mlp* m, const char* path)
{
    if (!m || !path) return LP_ERR_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return LP_ERR_ARG;
    char magic[8];
    int32_t hdr[2];
    std::vector<float> h(3 * LP_MLP_PARAMS);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "LPMLP001", 8) == 0 && fread(hdr, sizeof hdr, 1, f) == 1 &&
              hdr[0] == LP_MLP_PARAMS && fread(h.data(), sizeof(float), h.size(), f) == h.size();
    fclose(f);
    if (!ok) return LP_ERR_ARG;
    if (cudaMemcpy(m->master, h.data(), sizeof(float) * 3 * LP_MLP_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess ||
        lp::launch_mlp_shadow(m->master, m->shadow, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return LP_ERR_CUDA;
    m->step = hdr[1];
    return LP_OK;
}

int lp_mlp_forward(lp_mlp* m, const float* feat, int64_t M_cap, const int32_t* d_M, float* prob, float* logit,
                   void* stream)
{
    if (!m || M_cap < 0 || (M_cap > 0 && !feat)) return LP_ERR_ARG;
    return lp::launch_mlp_forward(m->shadow, feat, M_cap, d_M, prob, logit, S(stream)) == cudaSuccess ? LP_OK
                                                                                                      : LP_ERR_CUDA;
}

int lp_mlp_train_step(lp_mlp* m, const float* feat, const uint8_t* label, int64_t B, float lr, float* loss,
                      void* stream)
{
    if (!m || B <= 0 || !feat || !label || !(lr > 0.f)) return LP_ERR_ARG;
    const size_t n = (size_t)lp::mlp_grad_ctas(B);
    if (n > m->part_ctas) {
        cudaStreamSynchronize(S(stream));
        if (m->part) cudaFree(m->part);
        m->part = nullptr;
        if (cudaMalloc(&m->part, sizeof(float) * n * (LP_MLP_PARAMS + 1)) != cudaSuccess) {
            cudaGetLastError();
            m->part_ctas = 0;
            return LP_ERR_NOMEM;
        }
        m->lossp = m->part + n * LP_MLP_PARAMS;
        m->part_ctas = n;
    }
    m->step += 1;
    return lp::launch_mlp_train_step(m->master, m->m, m->v, m->shadow, feat, label, B, m->part, m->lossp, lr, m->step,
                                     loss, S(stream)) == cudaSuccess
               ? LP_OK
               : LP_ERR_CUDA;
}

}  // extern "C"
