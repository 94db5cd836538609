"""LP-SIFT oracle -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.

Python view of the plain FP64 C oracle in ``lp_oracle.c`` (compiled with gcc,
no vectorisation flags).  Only the tests, ``__graft_entry__.smoke`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares nothing with
the CUDA library except the seeded input generator.

Functions follow the paper's Sec. 2 (two-image stitching) and Sec. 4 (the
all-pairs homography matrix H_M); each C function cites its passage.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lp_oracle.c")
_HDR = os.path.join(_HERE, "lp_oracle.h")
_LIB = os.path.join(_HERE, "liblp_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, strict IEEE FP64)."""
    stale = not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Run every oracle function against another build of the C source (the
    mutation tests compile copies of lp_oracle.c with one planted mistake)."""
    global _lib
    saved = lib()
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = saved


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile C source text (a copy of lp_oracle.c) with the oracle's flags."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
                           "-I", _HERE, "-o", out_path, c_path, "-lm"])
    return out_path


def _load(path: str):
    L = C.CDLL(path)
    P = C.c_void_p
    i32, i64, u32, f64 = C.c_int, C.c_int64, C.c_uint32, C.c_double
    sig = {
        "or_gray_from_rgb": (i32, [P, i32, i32, i32, P]),
        "or_num_keypoints": (i64, [i32, i32, P, i32]),
        "or_detect": (i32, [P, i32, i32, i32, P, i32, f64, P]),
        "or_region_ws": (i32, [P, i32, f64, i32, P]),
        "or_orient_bin": (i32, [i32, i32]),
        "or_orient_weight": (u32, [i32]),
        "or_orient": (i32, [P, i32, i32, i32, P, P, i64, P, P]),
        "or_describe": (i32, [P, i32, i32, i32, P, P, P, i64, P, P]),
        "or_octant": (i32, [f64, f64]),
        "or_describe_ex": (i32, [P, i32, i32, i32, P, P, P, i64, i32, P, P]),
        "or_turn_fx": (i32, [i32, P, P]),
        "or_match": (i32, [P, P, i64, P, P, i64, f64, f64, P, i64, P, P, P, P, P]),
        "or_philox4x32_10": (None, [P, P, P]),
        "or_ransac_sample": (i32, [i64, C.c_uint64, u32, i32, P]),
        "or_dlt4": (i32, [P, P, P]),
        "or_refit": (i32, [P, P, i64, P]),
        "or_eig_sym": (i32, [i32, P, P, P]),
        "or_score": (i64, [P, P, i64, f64, P]),
        "or_ransac": (i32, [P, i64, i32, f64, C.c_uint64, u32, P, P, P, P, P, P]),
        "or_ransac_model": (i32, [P, i64, i32, i32, f64, C.c_uint64, u32, P, P, P, P, P, P]),
        "or_ransac_sample_k": (i32, [i64, C.c_uint64, u32, i32, i32, P]),
        "or_rigid_fit": (i32, [P, P, i64, P]),
        "or_model_sample_size": (i32, [i32]),
        "or_mlp_features": (i32, [i64, P, P, P, i32, P, P, P, i32, i32, i32, i32, P]),
        "or_mlp_forward": (i32, [P, P, i64, P, P]),
        "or_mlp_loss_grad": (i32, [P, P, P, i64, P, P]),
        "or_mlp_adam": (i32, [P, P, P, P, i32, i32, f64, f64, f64, f64]),
        "or_guided_weights": (i32, [P, i64, P]),
        "or_ransac_sample_guided": (i32, [i64, P, C.c_uint64, u32, i32, P]),
        "or_ransac_prior": (i32, [P, i64, P, i32, i32, f64, C.c_uint64, u32, i32, P, P, P, P, P, P]),
        "or_ransac_prior_model": (i32, [P, i64, i32, P, i32, i32, f64, C.c_uint64, u32, i32, P, P, P, P, P, P]),
        "or_guided_stop": (i32, [C.c_uint64, C.c_uint64, i32]),
        "or_guided_stop_k": (i32, [C.c_uint64, C.c_uint64, i32, i32]),
        "or_ransac_sample_guided_k": (i32, [i64, P, C.c_uint64, u32, i32, i32, P]),
        "or_mosaic_plan": (i32, [i32, P, i32, P, P, P, P, P, P, P, P, P]),
        "or_border_valid": (i32, [P, P, i64, i32, i32, P]),
        "or_mosaic_render": (i32, [i32, P, P, P, P, i32, P, P, i32, i32, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
def gray(img: np.ndarray) -> np.ndarray:
    """uint8 (H, W) or (H, W, 3) -> uint8 (H, W) intensity (Sec. 2.1)."""
    if img.ndim == 2:
        return np.ascontiguousarray(img, np.uint8)
    H, W, _ = img.shape
    rgb = _c(img, np.uint8)
    out = np.empty((H, W), np.uint8)
    assert lib().or_gray_from_rgb(_p(rgb), H, W, 3 * W, _p(out)) == 0
    return out


def num_keypoints(H: int, W: int, Ls) -> int:
    Ls = _c(Ls, np.int32)
    return int(lib().or_num_keypoints(H, W, _p(Ls), len(Ls)))


def detect(g: np.ndarray, Ls, alpha: float = 0.0) -> np.ndarray:
    """Eq. 1-2 feature points as raster indices, canonical order."""
    g = _c(g, np.uint8)
    H, W = g.shape
    Ls = _c(Ls, np.int32)
    K = num_keypoints(H, W, Ls)
    idx = np.empty(K, np.uint32)
    assert lib().or_detect(_p(g), H, W, W, _p(Ls), len(Ls), float(alpha), _p(idx)) == 0
    return idx


def region_ws(Ls, beta0: float = 0.0, d: int = 4) -> np.ndarray:
    Ls = _c(Ls, np.int32)
    ws = np.empty(len(Ls), np.int32)
    assert lib().or_region_ws(_p(Ls), len(Ls), float(beta0), d, _p(ws)) == 0
    return ws


def keypoint_scales(H: int, W: int, Ls, beta0: float = 0.0):
    """Per-keypoint (L, w_s) arrays in canonical order (L ascending)."""
    Ls_sorted = sorted(int(x) for x in Ls)
    ws_map = dict(zip(Ls_sorted, region_ws(Ls_sorted, beta0).tolist()))
    Lk, wk = [], []
    for L in Ls_sorted:
        n = 2 * (H // L) * (W // L)
        Lk.append(np.full(n, L, np.int32))
        wk.append(np.full(n, ws_map[L], np.int32))
    return np.concatenate(Lk), np.concatenate(wk)


def orient_bin(a: int, b: int) -> int:
    return int(lib().or_orient_bin(int(a), int(b)))


def octant(a: float, b: float) -> int:
    """Hard 8-direction sector [45k, 45(k+1)) degrees of atan2(b, a)."""
    return int(lib().or_octant(float(a), float(b)))


def turn_fx(k: int) -> tuple[int, int]:
    """(round(2^11 cos th), round(2^11 sin th)), th = (k + 0.5) * 10 degrees."""
    cq, sq = C.c_int(), C.c_int()
    assert lib().or_turn_fx(int(k), C.byref(cq), C.byref(sq)) == 0
    return cq.value, sq.value


def orient_weight(s: int) -> int:
    return int(lib().or_orient_weight(int(s)))


def orient(g: np.ndarray, idx: np.ndarray, ws: np.ndarray, want_hist: bool = False):
    g = _c(g, np.uint8)
    H, W = g.shape
    idx = _c(idx, np.uint32)
    ws = _c(ws, np.int32)
    K = len(idx)
    ori = np.empty(K, np.uint8)
    hist = np.empty((K, 36), np.uint64) if want_hist else None
    assert lib().or_orient(_p(g), H, W, W, _p(idx), _p(ws), K, _p(ori), _p(hist)) == 0
    return (ori, hist) if want_hist else ori


def describe(g: np.ndarray, idx: np.ndarray, ws: np.ndarray, ori: np.ndarray | None, border: bool = False,
             hard: bool = False):
    """Sec. 2.3 descriptors: soft bins, or (hard=True) whole magnitudes in
    45-degree sectors on the exact fixed-point turned grid."""
    g = _c(g, np.uint8)
    H, W = g.shape
    idx = _c(idx, np.uint32)
    ws = _c(ws, np.int32)
    K = len(idx)
    o = None if ori is None else _c(ori, np.uint8)
    desc = np.empty((K, 128), np.float64)
    valid = np.empty(K, np.uint8)
    assert lib().or_describe_ex(_p(g), H, W, W, _p(idx), _p(ws), _p(o), K, int(bool(hard)), _p(desc),
                                _p(valid)) == 0
    if border:
        assert lib().or_border_valid(_p(idx), _p(ws), K, H, W, _p(valid)) == 0
    return desc, valid


def match(dA, vA, dB, vB, ratio: float = 0.8, delta_s: float = float("inf"), rows=None):
    """Eq. 6 nearest neighbour + ratio test; returns (match, d1, d2, j1, j2)."""
    dA = _c(dA, np.float64)
    dB = _c(dB, np.float64)
    vA = _c(vA, np.uint8)
    vB = _c(vB, np.uint8)
    NA, NB = len(dA), len(dB)
    r = None if rows is None else _c(rows, np.int64)
    n = NA if r is None else len(r)
    m = np.empty(n, np.int32)
    d1 = np.empty(n, np.float64)
    d2 = np.empty(n, np.float64)
    j1 = np.empty(n, np.int32)
    j2 = np.empty(n, np.int32)
    assert lib().or_match(_p(dA), _p(vA), NA, _p(dB), _p(vB), NB, float(ratio), float(delta_s),
                          _p(r), 0 if r is None else len(r), _p(m), _p(d1), _p(d2), _p(j1), _p(j2)) == 0
    return m, d1, d2, j1, j2


def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.empty(4, np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def ransac_sample(M: int, seed: int, pair_id: int, t: int, k: int = 4):
    s = np.empty(k, np.int32)
    r = lib().or_ransac_sample_k(M, seed, pair_id, t, k, _p(s))
    return None if r else s


# Sec. 2.5 models: Eq. 7 homography (4-match samples), Eq. 8 rigid (2-match samples)
MODEL_HOMOGRAPHY = 0
MODEL_RIGID = 1


def rigid_fit(pts, mask=None):
    """Least-squares Eq. 8 (rotation + translation) of the masked rows of pts."""
    p = _c(pts, np.float64).reshape(-1, 4)
    m = _c(np.ones(len(p), np.uint8) if mask is None else mask, np.uint8)
    H = np.empty(9, np.float64)
    r = lib().or_rigid_fit(_p(p), _p(m), len(p), _p(H))
    return None if r else H.reshape(3, 3)


def dlt4(src, dst):
    s = _c(src, np.float64)
    d = _c(dst, np.float64)
    H = np.empty(9, np.float64)
    r = lib().or_dlt4(_p(s), _p(d), _p(H))
    return None if r else H.reshape(3, 3)


def refit(pts, mask):
    p = _c(pts, np.float64)
    m = _c(mask, np.uint8)
    H = np.empty(9, np.float64)
    r = lib().or_refit(_p(p), _p(m), len(m), _p(H))
    return None if r else H.reshape(3, 3)


def eig_sym(A):
    A = _c(A, np.float64)
    n = A.shape[0]
    ev = np.empty(n, np.float64)
    V = np.empty((n, n), np.float64)
    assert lib().or_eig_sym(n, _p(A), _p(ev), _p(V)) == 0
    return ev, V


def score(H, pts, thresh: float = 3.0):
    Hh = _c(H, np.float64).reshape(9)
    p = _c(pts, np.float64)
    m = np.empty(len(p), np.uint8)
    n = lib().or_score(_p(Hh), _p(p), len(p), float(thresh), _p(m))
    return int(n), m


def ransac(pts, T: int = 1000, thresh: float = 3.0, seed: int = 0, pair_id: int = 0, want_all: bool = False,
           model: int = MODEL_HOMOGRAPHY):
    """Returns dict(H, inliers, n_in, best_t[, counts, Hs])."""
    p = _c(pts, np.float64).reshape(-1, 4)
    M = len(p)
    H = np.empty(9, np.float64)
    inl = np.empty(M, np.uint8)
    n_in = C.c_int32()
    bt = C.c_int32()
    counts = np.empty(T, np.int32) if want_all else None
    Hs = np.empty((T, 9), np.float64) if want_all else None
    lib().or_ransac_model(_p(p), M, int(model), T, float(thresh), seed, pair_id, _p(H), _p(inl), C.byref(n_in),
                          C.byref(bt), _p(counts), _p(Hs))
    out = dict(H=H.reshape(3, 3), inliers=inl, n_in=int(n_in.value), best_t=int(bt.value))
    if want_all:
        out["counts"] = counts
        out["Hs"] = Hs
    return out


def keypoint_xy(idx: np.ndarray, W: int) -> np.ndarray:
    idx = np.asarray(idx, np.int64)
    return np.stack([idx % W, idx // W], axis=1).astype(np.float64)


def match_points(idxA, idxB, m, WA: int, WB: int) -> tuple[np.ndarray, np.ndarray]:
    """Compact accepted matches into (xA, yA, xB, yB) rows, in row order of A."""
    rows = np.nonzero(np.asarray(m) >= 0)[0]
    pa = keypoint_xy(np.asarray(idxA)[rows], WA)
    pb = keypoint_xy(np.asarray(idxB)[np.asarray(m)[rows]], WB)
    return np.concatenate([pa, pb], axis=1), rows


def features(img: np.ndarray, Ls, beta0: float = 0.0, upright: bool = False, alpha: float = 0.0,
             border: bool = False):
    """Sec. 2.1-2.3 for one image: gray, peaks, orientation, descriptors."""
    g = gray(img)
    H, W = g.shape
    idx = detect(g, Ls, alpha)
    _, ws = keypoint_scales(H, W, Ls, beta0)
    ori = None if upright else orient(g, idx, ws)
    desc, valid = describe(g, idx, ws, ori, border)
    return dict(gray=g, idx=idx, ws=ws, ori=ori, desc=desc, valid=valid)


def stitch_pair(imgA, imgB, Ls, ratio=0.8, T=1000, thresh=3.0, seed=0, pair_id=0, upright=False,
                delta_s=float("inf"), model=MODEL_HOMOGRAPHY, alpha=0.0, border=False):
    """Sec. 2 end to end for one pair (Fig. 2): H from A to B and its inliers."""
    fa = features(imgA, Ls, upright=upright, alpha=alpha, border=border)
    fb = features(imgB, Ls, upright=upright, alpha=alpha, border=border)
    m, d1, d2, _, _ = match(fa["desc"], fa["valid"], fb["desc"], fb["valid"], ratio, delta_s)
    pts, rows = match_points(fa["idx"], fb["idx"], m, fa["gray"].shape[1], fb["gray"].shape[1])
    r = ransac(pts, T, thresh, seed, pair_id, model=model)
    r.update(fa=fa, fb=fb, match=m, d1=d1, d2=d2, pts=pts, rows=rows)
    return r


# ---------------------------------------------------------------------------
# Learned RANSAC proposal (not in the paper)
# ---------------------------------------------------------------------------
MLP_NPARAM = 4801


def mlp_split(params):
    """Views W1 (64x8), b1, W2 (64x64), b2, w3 (64), b3 of a flat parameter vector."""
    p = np.asarray(params)
    return (p[:512].reshape(64, 8), p[512:576], p[576:4672].reshape(64, 64), p[4672:4736], p[4736:4800],
            p[4800:4801])


def mlp_features(d1, d2, LA, Lmax, oriA, oriB, pts, WA, HA, WB, HB):
    d1 = _c(d1, np.float64)
    d2 = _c(d2, np.float64)
    LA = _c(LA, np.int32)
    oA = _c(oriA, np.uint8)
    oB = _c(oriB, np.uint8)
    p = _c(pts, np.float64).reshape(-1, 4)
    M = len(d1)
    f = np.empty((M, 8), np.float64)
    assert lib().or_mlp_features(M, _p(d1), _p(d2), _p(LA), int(Lmax), _p(oA), _p(oB), _p(p), WA, HA, WB, HB,
                                 _p(f)) == 0
    return f


def mlp_forward(params, x):
    P = _c(params, np.float64)
    x = _c(x, np.float64).reshape(-1, 8)
    z = np.empty(len(x), np.float64)
    pr = np.empty(len(x), np.float64)
    lib().or_mlp_forward(_p(P), _p(x), len(x), _p(z), _p(pr))
    return z, pr


def mlp_loss_grad(params, x, y):
    P = _c(params, np.float64)
    x = _c(x, np.float64).reshape(-1, 8)
    y = _c(y, np.uint8)
    g = np.empty(MLP_NPARAM, np.float64)
    L = C.c_double()
    assert lib().or_mlp_loss_grad(_p(P), _p(x), _p(y), len(x), C.byref(L), _p(g)) == 0
    return L.value, g


def mlp_adam(params, m, v, grad, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays params, m, v."""
    assert params.dtype == m.dtype == v.dtype == np.float64
    g = _c(grad, np.float64)
    assert lib().or_mlp_adam(_p(params), _p(m), _p(v), _p(g), len(params), int(t), lr, b1, b2, eps) == 0


def guided_weights(prob):
    pr = _c(prob, np.float32)
    out = np.empty(len(pr), np.uint64)
    lib().or_guided_weights(_p(pr), len(pr), _p(out))
    return out


def ransac_sample_guided(prefix, seed, pair_id, t, k=4):
    pf = _c(prefix, np.uint64)
    s = np.empty(k, np.int32)
    r = lib().or_ransac_sample_guided_k(len(pf), _p(pf), seed, pair_id, t, k, _p(s))
    return None if r else s


def ransac_prior(pts, prob, Tg=64, T=1000, thresh=3.0, seed=0, pair_id=0, want_counts=False,
                 model=MODEL_HOMOGRAPHY, min_support=8):
    """Guided phase of Tg hypotheses, then uniform fallback of T (see lp_oracle.h);
    the guided phase may end the search only with at least min_support inliers."""
    p = _c(pts, np.float64).reshape(-1, 4)
    pr = _c(prob, np.float32)
    M = len(p)
    H = np.empty(9, np.float64)
    inl = np.empty(max(M, 1), np.uint8)
    n_in = C.c_int32()
    bt = C.c_int32()
    it = C.c_int32()
    counts = np.empty(Tg + T, np.int32) if want_counts else None
    lib().or_ransac_prior_model(_p(p), M, int(model), _p(pr), int(Tg), int(T), float(thresh), seed, pair_id,
                                int(min_support), _p(H), _p(inl), C.byref(n_in), C.byref(bt), C.byref(it),
                                _p(counts))
    out = dict(H=H.reshape(3, 3), inliers=inl[:M], n_in=int(n_in.value), best_t=int(bt.value), iters=int(it.value))
    if want_counts:
        out["counts"] = counts
    return out


def guided_stop(s_in, total, Tg, k=4) -> bool:
    return bool(lib().or_guided_stop_k(int(s_in), int(total), int(Tg), int(k)))


def mosaic_plan(n_images, pairs, HM, valid, sizes):
    """Sec. 4 rounds.  pairs [(a, b)], HM [P, 3, 3] (x_b ~ H x_a), valid [P],
    sizes [(H, W)].  Returns dict(G [N, 3, 3] image -> canvas, round [N],
    ref [N], canvas (h, w))."""
    pr = _c(np.asarray(pairs, np.int32).reshape(-1, 2), np.int32)
    H = _c(np.asarray(HM, np.float64).reshape(-1, 9), np.float64)
    v = _c(np.asarray(valid, np.uint8), np.uint8)
    Hs = _c([s[0] for s in sizes], np.int32)
    Ws = _c([s[1] for s in sizes], np.int32)
    G = np.zeros((n_images, 9), np.float64)
    rnd = np.zeros(n_images, np.int32)
    ref = np.zeros(n_images, np.int32)
    cw, ch = C.c_int(), C.c_int()
    assert lib().or_mosaic_plan(n_images, _p(pr), len(pr), _p(H), _p(v), _p(Hs), _p(Ws), _p(G), _p(rnd), _p(ref),
                                C.byref(cw), C.byref(ch)) == 0
    return dict(G=G.reshape(-1, 3, 3), round=rnd, ref=ref, canvas=(ch.value, cw.value))


def mosaic_render(images, G, rounds, canvas_hw):
    """images: list of uint8 (H, W) or (H, W, 3); G [N, 3, 3]; -> (canvas, cover)."""
    C_ = 3 if images[0].ndim == 3 else 1
    ims = [np.ascontiguousarray(im, np.uint8) for im in images]
    ptrs = (C.c_void_p * len(ims))(*[im.ctypes.data for im in ims])
    Hs = _c([im.shape[0] for im in ims], np.int32)
    Ws = _c([im.shape[1] for im in ims], np.int32)
    pitch = _c([im.shape[1] * C_ for im in ims], np.int32)
    h, w = canvas_hw
    canvas = np.zeros((h, w, C_) if C_ == 3 else (h, w), np.uint8)
    cover = np.zeros((h, w), np.uint8)
    Gd = _c(np.asarray(G, np.float64).reshape(-1, 9), np.float64)
    r = _c(rounds, np.int32)
    assert lib().or_mosaic_render(len(ims), C.cast(ptrs, C.c_void_p), _p(Hs), _p(Ws), _p(pitch), C_, _p(Gd), _p(r),
                                  w, h, _p(canvas), _p(cover)) == 0
    return canvas, cover
