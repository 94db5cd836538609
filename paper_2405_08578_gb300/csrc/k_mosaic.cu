// Sec. 4 mosaic: reference rounds over the homography matrix H_M (host) and
// the warp of every placed image onto one canvas (device).
//
//  lp_mosaic_plan    host: image degrees from the valid H_M entries; round 1
//                    takes the image of largest degree as reference (identity)
//                    and places its matched images through their entries;
//                    each later round takes, among unmatched images linked to a
//                    placed one, the one of largest degree, places it through
//                    its link (to the placed image of lowest index) and then
//                    its unmatched neighbours through it.  Ties: lowest index.
//                    Placements map image pixels to the canvas (the integer
//                    bounding box of the placed corner pixels).
//  k_mosaic_render   one thread per canvas pixel: every placed image whose
//                    inverse placement maps the pixel inside the image adds
//                    its bilinear sample; the pixel is the mean (rounded half
//                    up), 0 where no image covers it; `cover` counts them.  A
//                    CTA skips the images whose canvas bounding box (from the
//                    placed corners, with a margin) misses its 32 x 8 tile.
#include <math.h>
#include <string.h>

#include <vector>

#include "lp_internal.cuh"

namespace {

constexpr int kMaxMosaic = 64;

struct MosaicImage {
    const uint8_t* data;
    int H, W, pitch;
    float m[9];   // canvas pixel -> image pixel
    int bx0, by0, bx1, by1;   // canvas pixels the image can cover (inclusive)
};

struct MosaicParams {
    int n, C, cw, ch, pitch;
    uint8_t* canvas;
    uint8_t* cover;
    MosaicImage im[kMaxMosaic];
};

__global__ void __launch_bounds__(256) k_mosaic_render(const __grid_constant__ MosaicParams p)
{
    const int tx0 = blockIdx.x * 32, ty0 = blockIdx.y * 8;
    const int x = tx0 + (threadIdx.x & 31);
    const int y = ty0 + (threadIdx.x >> 5);
    if (x >= p.cw || y >= p.ch) return;
    const float fx = (float)x, fy = (float)y;
    float sum[3] = {0.f, 0.f, 0.f};
    int n = 0;
    for (int i = 0; i < p.n; ++i) {
        const MosaicImage& I = p.im[i];
        if (I.bx1 < tx0 || I.bx0 > tx0 + 31 || I.by1 < ty0 || I.by0 > ty0 + 7) continue;   // CTA-uniform
        const float w = fmaf(I.m[6], fx, fmaf(I.m[7], fy, I.m[8]));
        if (!(w > 0.f)) continue;
        const float u = fmaf(I.m[0], fx, fmaf(I.m[1], fy, I.m[2])) / w;
        const float v = fmaf(I.m[3], fx, fmaf(I.m[4], fy, I.m[5])) / w;
        if (!(u >= 0.f && v >= 0.f && u <= (float)(I.W - 1) && v <= (float)(I.H - 1))) continue;
        const int u0 = (int)floorf(u), v0 = (int)floorf(v);
        const int u1 = u0 + 1 < I.W ? u0 + 1 : u0, v1 = v0 + 1 < I.H ? v0 + 1 : v0;
        const float fu = u - (float)u0, fv = v - (float)v0;
        const uint8_t* r0 = I.data + (size_t)v0 * I.pitch;
        const uint8_t* r1 = I.data + (size_t)v1 * I.pitch;
        for (int c = 0; c < p.C; ++c) {
            const float p00 = __ldg(r0 + u0 * p.C + c), p01 = __ldg(r0 + u1 * p.C + c);
            const float p10 = __ldg(r1 + u0 * p.C + c), p11 = __ldg(r1 + u1 * p.C + c);
            const float top = p00 + fu * (p01 - p00), bot = p10 + fu * (p11 - p10);
            sum[c] += top + fv * (bot - top);
        }
        ++n;
    }
    uint8_t* out = p.canvas + (size_t)y * p.pitch + (size_t)x * p.C;
    for (int c = 0; c < p.C; ++c) out[c] = n ? (uint8_t)floorf(sum[c] / (float)n + 0.5f) : (uint8_t)0;
    if (p.cover) p.cover[(size_t)y * p.cw + x] = (uint8_t)n;
}

void mul3(const double* A, const double* B, double* Cm)
{
    double t[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) t[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
    memcpy(Cm, t, sizeof t);
}

bool inverse3(const double* M, double* R)
{
    const double a = M[0], b = M[1], c = M[2], d = M[3], e = M[4], f = M[5], g = M[6], h = M[7], i = M[8];
    const double A = e * i - f * h, B = f * g - d * i, Cc = d * h - e * g;
    const double det = a * A + b * B + c * Cc;
    if (!(fabs(det) > 0)) return false;
    const double s = 1.0 / det;
    R[0] = A * s; R[1] = (c * h - b * i) * s; R[2] = (b * f - c * e) * s;
    R[3] = B * s; R[4] = (a * i - c * g) * s; R[5] = (c * d - a * f) * s;
    R[6] = Cc * s; R[7] = (b * g - a * h) * s; R[8] = (a * e - b * d) * s;
    return true;
}

}  // namespace

extern "C" {

int lp_mosaic_plan(int N, const int32_t* pairs, int P, const double* HM, const uint8_t* valid, const int32_t* Hs,
                   const int32_t* Ws, double* G, int32_t* round_of, int32_t* ref_of, int32_t* canvas_w,
                   int32_t* canvas_h)
{
    if (N < 1 || N > kMaxMosaic || P < 0 || (P > 0 && (!pairs || !HM || !valid)) || !Hs || !Ws || !G || !round_of ||
        !ref_of || !canvas_w || !canvas_h)
        return LP_ERR_ARG;
    for (int q = 0; q < 2 * P; ++q)
        if (pairs[q] < 0 || pairs[q] >= N) return LP_ERR_ARG;
    for (int i = 0; i < N; ++i)
        if (Hs[i] < 1 || Ws[i] < 1) return LP_ERR_ARG;
    std::vector<int> degree(N, 0);
    for (int q = 0; q < P; ++q)
        if (valid[q]) { ++degree[pairs[2 * q]]; ++degree[pairs[2 * q + 1]]; }
    auto other = [&](int q, int i) { return pairs[2 * q] == i ? pairs[2 * q + 1] : (pairs[2 * q + 1] == i ? pairs[2 * q] : -1); };
    // map from image `from` to the other image of entry q
    auto map_from = [&](int q, int from, double* M) {
        if (pairs[2 * q] == from) { memcpy(M, HM + 9 * (size_t)q, sizeof(double) * 9); return true; }
        return inverse3(HM + 9 * (size_t)q, M);
    };
    std::vector<double> W((size_t)N * 9, 0.0);   // image -> frame of the first reference
    for (int i = 0; i < N; ++i) { round_of[i] = -1; ref_of[i] = -1; }
    int placed = 0;
    for (int rnd = 0; placed < N; ++rnd) {
        int ref = -1, via = -1;
        for (int i = 0; i < N; ++i) {
            if (round_of[i] >= 0) continue;
            int link = -1, link_img = -1;
            if (rnd > 0) {
                for (int q = 0; q < P; ++q) {
                    const int o = valid[q] ? other(q, i) : -1;
                    if (o >= 0 && round_of[o] >= 0 && (link < 0 || o < link_img)) { link = q; link_img = o; }
                }
                if (link < 0) continue;
            }
            if (ref < 0 || degree[i] > degree[ref]) { ref = i; via = link; }
        }
        if (ref < 0) break;
        if (rnd == 0) {
            for (int k = 0; k < 9; ++k) W[9 * (size_t)ref + k] = k % 4 == 0 ? 1.0 : 0.0;
        } else {
            double M[9];
            if (!map_from(via, ref, M)) break;
            mul3(&W[9 * (size_t)other(via, ref)], M, &W[9 * (size_t)ref]);
        }
        round_of[ref] = rnd;
        ref_of[ref] = ref;
        ++placed;
        for (int q = 0; q < P; ++q) {
            const int j = valid[q] ? other(q, ref) : -1;
            if (j < 0 || round_of[j] >= 0) continue;
            double M[9];
            if (!map_from(q, j, M)) continue;
            mul3(&W[9 * (size_t)ref], M, &W[9 * (size_t)j]);
            round_of[j] = rnd;
            ref_of[j] = ref;
            ++placed;
        }
    }
    double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
    for (int i = 0; i < N; ++i) {
        if (round_of[i] < 0) continue;
        const double* g = &W[9 * (size_t)i];
        for (int c = 0; c < 4; ++c) {
            const double cx = (c & 1) ? Ws[i] - 1.0 : 0.0, cy = (c & 2) ? Hs[i] - 1.0 : 0.0;
            const double w = g[6] * cx + g[7] * cy + g[8];
            const double x = (g[0] * cx + g[1] * cy + g[2]) / w, y = (g[3] * cx + g[4] * cy + g[5]) / w;
            x0 = fmin(x0, x); x1 = fmax(x1, x); y0 = fmin(y0, y); y1 = fmax(y1, y);
        }
    }
    if (!placed) { *canvas_w = 0; *canvas_h = 0; return LP_OK; }
    const double sx = floor(x0), sy = floor(y0);
    const double cwd = ceil(x1) - sx + 1.0, chd = ceil(y1) - sy + 1.0;
    if (!(cwd >= 1 && chd >= 1 && cwd <= 32768 && chd <= 32768)) return LP_ERR_UNSUPPORTED;
    *canvas_w = (int32_t)cwd;
    *canvas_h = (int32_t)chd;
    const double shift[9] = {1, 0, -sx, 0, 1, -sy, 0, 0, 1};
    for (int i = 0; i < N; ++i) {
        if (round_of[i] < 0) { memset(G + 9 * (size_t)i, 0, sizeof(double) * 9); continue; }
        mul3(shift, &W[9 * (size_t)i], G + 9 * (size_t)i);
    }
    return LP_OK;
}

}  // extern "C"

namespace lp {

cudaError_t launch_mosaic_render(const lp_image* imgs, int N, const double* G, const int32_t* round_of, uint8_t* canvas,
                                 int cw, int ch, int pitch, uint8_t* cover, cudaStream_t s, int* bad)
{
    *bad = 0;
    if (N < 1 || N > kMaxMosaic) { *bad = 1; return cudaSuccess; }
    MosaicParams p;
    memset(&p, 0, sizeof p);
    p.C = imgs[0].channels;
    p.cw = cw;
    p.ch = ch;
    p.pitch = pitch;
    p.canvas = canvas;
    p.cover = cover;
    for (int i = 0; i < N; ++i) {
        if (round_of[i] < 0) continue;
        double inv[9];
        if (!inverse3(G + 9 * (size_t)i, inv)) { *bad = 1; return cudaSuccess; }
        MosaicImage& m = p.im[p.n++];
        m.data = imgs[i].data;
        m.H = imgs[i].H;
        m.W = imgs[i].W;
        m.pitch = imgs[i].pitch;
        for (int k = 0; k < 9; ++k) m.m[k] = (float)inv[k];
        // canvas footprint: with w > 0 at the four corners (w is affine over
        // the image, so positive everywhere) the image maps onto the convex
        // quad of its corners; otherwise no culling
        const double* g = G + 9 * (size_t)i;
        double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
        bool bounded = true;
        for (int q = 0; q < 4; ++q) {
            const double cx = (q & 1) ? imgs[i].W - 1.0 : 0.0, cy = (q & 2) ? imgs[i].H - 1.0 : 0.0;
            const double w = g[6] * cx + g[7] * cy + g[8];
            if (!(w > 0)) { bounded = false; break; }
            const double u = (g[0] * cx + g[1] * cy + g[2]) / w, v = (g[3] * cx + g[4] * cy + g[5]) / w;
            x0 = fmin(x0, u); x1 = fmax(x1, u); y0 = fmin(y0, v); y1 = fmax(y1, v);
        }
        if (bounded && x1 - x0 < 1e9 && y1 - y0 < 1e9) {
            m.bx0 = (int)floor(x0) - 2; m.by0 = (int)floor(y0) - 2;
            m.bx1 = (int)ceil(x1) + 2;  m.by1 = (int)ceil(y1) + 2;
        } else {
            m.bx0 = m.by0 = -(1 << 30);
            m.bx1 = m.by1 = 1 << 30;
        }
    }
    if (cw <= 0 || ch <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((cw + 31) / 32), (unsigned)((ch + 7) / 8));
    k_mosaic_render<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace lp
