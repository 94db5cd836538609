"""ctypes binding of liblp (include/lp.h).  Argument marshalling only.

Every function has the C name and takes torch tensors where the C call takes
device pointers; the current torch CUDA stream is passed as ``stream``.  No
step of the method runs here: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

from . import build as _build

LP_OK = 0
ERR_NAMES = {0: "LP_OK", 1: "LP_ERR_ARG", 2: "LP_ERR_ALIGN", 3: "LP_ERR_CUDA", 4: "LP_ERR_TIMEOUT",
             5: "LP_ERR_NOMEM", 6: "LP_ERR_DEGENERATE", 7: "LP_ERR_UNSUPPORTED", 8: "LP_ERR_DEVICE"}
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2
MODEL_HOMOGRAPHY, MODEL_RIGID = 0, 1   # Sec. 2.5: Eq. 7 homography, Eq. 8 rigid
MAX_SCALES = 8


class LpError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class lp_host_pair(C.Structure):
    _fields_ = [("A", C.c_void_p), ("B", C.c_void_p), ("HA", C.c_int32), ("WA", C.c_int32), ("pitchA", C.c_int32),
                ("HB", C.c_int32), ("WB", C.c_int32), ("pitchB", C.c_int32)]


class lp_image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("H", C.c_int32), ("W", C.c_int32), ("pitch", C.c_int32),
                ("channels", C.c_int32)]


class lp_config(C.Structure):
    _fields_ = [("nL", C.c_int32), ("Ls", C.c_int32 * MAX_SCALES), ("beta0", C.c_double), ("ratio", C.c_float),
                ("delta_s", C.c_float), ("ransac_iters", C.c_int32), ("thresh_px", C.c_float),
                ("seed", C.c_uint64), ("min_inliers", C.c_int32), ("precision", C.c_int32),
                ("upright", C.c_int32), ("model", C.c_int32), ("alpha", C.c_double), ("border", C.c_int32),
                ("hard_bins", C.c_int32)]


_lib = None
SYMBOLS = ["lp_config_default", "lp_create", "lp_destroy", "lp_num_keypoints", "lp_detect", "lp_detect_batch",
           "lp_describe",
           "lp_match", "lp_compact", "lp_ransac", "lp_ransac_static", "lp_stitch_pair", "lp_stitch_pair_host", "lp_stitch_pairs_host", "lp_stitch_pairs", "lp_stitch_pairs_ids", "lp_sync_status",
           "lp_last_error", "lp_diag_last_rescans", "lp_diag_orient_bins", "lp_diag_orient_weights", "lp_diag_philox", "lp_diag_gray",
           "lp_mlp_create", "lp_mlp_destroy", "lp_mlp_set_params", "lp_mlp_get_params", "lp_mlp_get_state", "lp_mlp_save",
           "lp_mlp_load", "lp_mlp_features", "lp_mlp_forward", "lp_mlp_train_step", "lp_ransac_prior",
           "lp_diag_last_ransac_counts", "lp_set_proposal", "lp_set_profiling", "lp_diag_last_match_kernel_ms",
           "lp_set_autotune", "lp_autotune_table", "lp_diag_set_batch_hold",
           "lp_mosaic_plan", "lp_mosaic_render"]
MLP_PARAMS = 4801


def lib_path() -> str:
    return _build.OUT


def load(build_if_missing: bool = True):
    """Load liblp.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.OUT):
        raise RuntimeError(f"liblp.so not built at {_build.OUT}")
    L = C.CDLL(_build.OUT)
    P, i32, i64, u32 = C.c_void_p, C.c_int, C.c_int64, C.c_uint32
    sig = {
        "lp_config_default": (i32, [C.POINTER(lp_config)]),
        "lp_create": (i32, [C.POINTER(P), C.POINTER(lp_config)]),
        "lp_destroy": (i32, [P]),
        "lp_num_keypoints": (i64, [i32, i32, P, i32]),
        "lp_detect": (i32, [P, P, i32, i32, i32, i32, P, P, P]),
        "lp_detect_batch": (i32, [P, P, i32, P, P, P]),
        "lp_describe": (i32, [P, P, i32, i32, i32, P, i64, P, P, P, P, P]),
        "lp_match": (i32, [P, P, P, P, i64, P, P, P, i64, P, P, P, P]),
        "lp_compact": (i32, [P, P, i32, P, i32, P, i64, P, P, P, P]),
        "lp_ransac": (i32, [P, P, i64, P, u32, P, P, P, P, P]),
        "lp_ransac_static": (i32, [P, i64, P, i32, C.c_float, C.c_uint64, u32, P, P, P, P, P]),
        "lp_stitch_pair": (i32, [P, P, i32, i32, i32, P, i32, i32, i32, i32, u32, P, P, P, P]),
        "lp_stitch_pair_host": (i32, [P, P, i32, i32, i32, P, i32, i32, i32, i32, u32, P, P, P, P]),
        "lp_stitch_pairs_host": (i32, [P, P, i32, i32, u32, P, P, P, P]),
        "lp_stitch_pairs": (i32, [P, P, i32, P, i32, P, P, P, P, P]),
        "lp_stitch_pairs_ids": (i32, [P, P, i32, P, P, i32, P, P, P, P, P]),
        "lp_sync_status": (i32, [P]),
        "lp_last_error": (C.c_char_p, [P]),
        "lp_diag_last_rescans": (i32, [P, C.POINTER(C.c_int64)]),
        "lp_diag_orient_bins": (i32, [P, P]),
        "lp_diag_orient_weights": (i32, [P, P]),
        "lp_diag_philox": (i32, [P, i64, u32, u32, P, P]),
        "lp_diag_gray": (i32, [P, i64, P, P]),
        "lp_mlp_create": (i32, [C.POINTER(P), C.c_uint64]),
        "lp_mlp_destroy": (i32, [P]),
        "lp_mlp_set_params": (i32, [P, P]),
        "lp_mlp_get_params": (i32, [P, P]),
        "lp_mlp_get_state": (i32, [P, P, P]),
        "lp_mlp_save": (i32, [P, C.c_char_p]),
        "lp_mlp_load": (i32, [P, C.c_char_p]),
        "lp_mlp_features": (i32, [P, P, P, i32, i32, P, P, i32, i32, P, P, P, P, P, i64, P, P]),
        "lp_mlp_forward": (i32, [P, P, i64, P, P, P, P]),
        "lp_mlp_train_step": (i32, [P, P, P, i64, C.c_float, P, P]),
        "lp_ransac_prior": (i32, [P, P, i64, P, P, i32, u32, P, P, P, P, P, P]),
        "lp_diag_last_ransac_counts": (i32, [P, P, i32]),
        "lp_set_proposal": (i32, [P, P, i32]),
        "lp_set_profiling": (i32, [P, i32]),
        "lp_mosaic_plan": (i32, [i32, P, i32, P, P, P, P, P, P, P, P, P]),
        "lp_mosaic_render": (i32, [P, P, i32, P, P, P, i32, i32, i32, P, P]),
        "lp_diag_last_match_kernel_ms": (i32, [P, C.POINTER(C.c_float)]),
        "lp_set_autotune": (i32, [P, i32]),
        "lp_diag_set_batch_hold": (i32, [P, i32]),
        "lp_autotune_table": (i32, [P, P, i32, C.POINTER(C.c_int32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("liblp takes device tensors")
    return t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def config(Ls=(16, 32, 64, 128), beta0=0.0, ratio=0.8, delta_s=math.inf, ransac_iters=1000, thresh_px=3.0,
           seed=0, min_inliers=8, precision=PREC_FP32, upright=False, model=MODEL_HOMOGRAPHY, alpha=0.0,
           border=False, hard_bins=False) -> lp_config:
    c = lp_config()
    load().lp_config_default(C.byref(c))
    Ls = list(Ls)
    if not 1 <= len(Ls) <= MAX_SCALES:
        raise ValueError("1..8 window sizes")
    c.nL = len(Ls)
    for i, L in enumerate(Ls):
        c.Ls[i] = int(L)
    c.beta0, c.ratio, c.delta_s = float(beta0), float(ratio), float(delta_s)
    c.ransac_iters, c.thresh_px, c.seed = int(ransac_iters), float(thresh_px), int(seed)
    c.min_inliers, c.precision, c.upright = int(min_inliers), int(precision), int(bool(upright))
    c.model = int(model)
    c.alpha, c.border, c.hard_bins = float(alpha), int(bool(border)), int(bool(hard_bins))
    return c


class Context:
    """Owns an lp_ctx (config copy, status word, workspace)."""

    def __init__(self, cfg: lp_config | None = None, **kw):
        self.lib = load()
        self.cfg = cfg if cfg is not None else config(**kw)
        h = C.c_void_p()
        r = self.lib.lp_create(C.byref(h), C.byref(self.cfg))
        if r != LP_OK:
            raise LpError(r, "lp_create")
        self.h = h

    @property
    def Ls(self):
        return [self.cfg.Ls[i] for i in range(self.cfg.nL)]

    def close(self):
        if getattr(self, "h", None):
            self.lib.lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, r, what):
        if r != LP_OK:
            raise LpError(r, f"{what}: {self.lib.lp_last_error(self.h).decode(errors='replace')}")

    # ---- the C entry points, same names ----
    def lp_detect(self, img, H, W, pitch, channels, kp_idx, gray=None, stream=None):
        self._chk(self.lib.lp_detect(self.h, _ptr(img), H, W, pitch, channels, _ptr(kp_idx), _ptr(gray),
                                     _stream(stream)), "lp_detect")

    def lp_detect_batch(self, images, kps, grays=None, stream=None):
        """images: list of (device uint8 tensor, H, W, pitch, channels); kps: int32
        device tensors, one per image; grays: uint8 device tensors (RGB) or None."""
        n = len(images)
        arr = (lp_image * n)(*[lp_image(_ptr(t), H, W, p, ch) for (t, H, W, p, ch) in images])
        kp_arr = (C.c_void_p * n)(*[_ptr(k) for k in kps])
        g_arr = (C.c_void_p * n)(*[_ptr(g) if g is not None else None for g in (grays or [None] * n)])
        self._chk(self.lib.lp_detect_batch(self.h, arr, n, kp_arr, g_arr, _stream(stream)), "lp_detect_batch")

    def lp_describe(self, gray, H, W, gray_pitch, kp_idx, K, ori, desc, desc_bf16, valid, stream=None):
        self._chk(self.lib.lp_describe(self.h, _ptr(gray), H, W, gray_pitch, _ptr(kp_idx), K, _ptr(ori), _ptr(desc),
                                       _ptr(desc_bf16), _ptr(valid), _stream(stream)), "lp_describe")

    def lp_match(self, dA, dA16, vA, NA, dB, dB16, vB, NB, match, d1, d2, stream=None):
        self._chk(self.lib.lp_match(self.h, _ptr(dA), _ptr(dA16), _ptr(vA), NA, _ptr(dB), _ptr(dB16), _ptr(vB), NB,
                                    _ptr(match), _ptr(d1), _ptr(d2), _stream(stream)), "lp_match")

    def lp_compact(self, kpA, WA, kpB, WB, match, NA, pts, rows, d_M, stream=None):
        self._chk(self.lib.lp_compact(self.h, _ptr(kpA), WA, _ptr(kpB), WB, _ptr(match), NA, _ptr(pts), _ptr(rows),
                                      _ptr(d_M), _stream(stream)), "lp_compact")

    def lp_ransac(self, pts, M_cap, d_M, pair_id, H, inlier, n_inliers, best_t=None, stream=None):
        self._chk(self.lib.lp_ransac(self.h, _ptr(pts), M_cap, _ptr(d_M), pair_id, _ptr(H), _ptr(inlier),
                                     _ptr(n_inliers), _ptr(best_t), _stream(stream)), "lp_ransac")

    def lp_stitch_pair(self, imgA, HA, WA, pitchA, imgB, HB, WB, pitchB, channels, pair_id, H, n_in, M_out=None,
                       stream=None):
        self._chk(self.lib.lp_stitch_pair(self.h, _ptr(imgA), HA, WA, pitchA, _ptr(imgB), HB, WB, pitchB, channels,
                                          pair_id, _ptr(H), _ptr(n_in), _ptr(M_out), _stream(stream)),
                  "lp_stitch_pair")

    def lp_stitch_pair_host(self, imgA, HA, WA, pitchA, imgB, HB, WB, pitchB, channels, pair_id, stream=None):
        """imgA/imgB: host (ideally pinned) uint8 tensors.  Returns (H 3x3 float64, n_in, M)."""
        Hh = (C.c_double * 9)()
        n = C.c_int32()
        m = C.c_int32()
        self._chk(self.lib.lp_stitch_pair_host(self.h, imgA.data_ptr(), HA, WA, pitchA, imgB.data_ptr(), HB, WB,
                                               pitchB, channels, pair_id, Hh, C.byref(n), C.byref(m),
                                               _stream(stream)), "lp_stitch_pair_host")
        return [list(Hh[0:3]), list(Hh[3:6]), list(Hh[6:9])], n.value, m.value

    def lp_stitch_pairs_host(self, pairs, channels, pair_id0=0, stream=None):
        """pairs: list of (A, HA, WA, pitchA, B, HB, WB, pitchB) with host (ideally
        pinned) uint8 tensors.  Returns (H float64 array [P, 3, 3], n_in [P], M [P])."""
        import numpy as np
        P = len(pairs)
        arr = (lp_host_pair * max(P, 1))(*[lp_host_pair(A.data_ptr(), B.data_ptr(), HA, WA, pa, HB, WB, pb)
                                            for (A, HA, WA, pa, B, HB, WB, pb) in pairs])
        Hh = np.zeros((max(P, 1), 3, 3), np.float64)
        n = np.zeros(max(P, 1), np.int32)
        m = np.zeros(max(P, 1), np.int32)
        self._chk(self.lib.lp_stitch_pairs_host(self.h, arr, P, channels, pair_id0, Hh.ctypes.data, n.ctypes.data,
                                                m.ctypes.data, _stream(stream)), "lp_stitch_pairs_host")
        return Hh[:P], n[:P], m[:P]

    def lp_stitch_pairs(self, images, HM, n_in, valid, pairs=None, M_out=None, stream=None, pair_ids=None):
        """images: list of (device uint8 tensor, H, W, pitch, channels).  With
        pair_ids (one per pair) the call is lp_stitch_pairs_ids."""
        arr = (lp_image * len(images))(*[lp_image(_ptr(t), H, W, p, ch) for (t, H, W, p, ch) in images])
        if pairs is None:
            pp, P = None, 0
        else:
            flat = (C.c_int32 * (2 * len(pairs)))(*[int(v) for pr in pairs for v in pr])
            pp, P = C.cast(flat, C.c_void_p), len(pairs)
        if pair_ids is None:
            self._chk(self.lib.lp_stitch_pairs(self.h, C.cast(arr, C.c_void_p), len(images), pp, P, _ptr(HM),
                                               _ptr(n_in), _ptr(valid), _ptr(M_out), _stream(stream)),
                      "lp_stitch_pairs")
        else:
            ids = (C.c_uint32 * len(pair_ids))(*[int(v) for v in pair_ids])
            self._chk(self.lib.lp_stitch_pairs_ids(self.h, C.cast(arr, C.c_void_p), len(images), pp,
                                                   C.cast(ids, C.c_void_p), P, _ptr(HM), _ptr(n_in), _ptr(valid),
                                                   _ptr(M_out), _stream(stream)), "lp_stitch_pairs_ids")

    def lp_mlp_features(self, kpA, oriA, HA, WA, kpB, oriB, HB, WB, match, d1, d2, rows, d_M, M_cap, feat,
                        stream=None):
        self._chk(self.lib.lp_mlp_features(self.h, _ptr(kpA), _ptr(oriA), HA, WA, _ptr(kpB), _ptr(oriB), HB, WB,
                                           _ptr(match), _ptr(d1), _ptr(d2), _ptr(rows), _ptr(d_M), M_cap, _ptr(feat),
                                           _stream(stream)), "lp_mlp_features")

    def lp_ransac_prior(self, pts, M_cap, d_M, prior, guided_iters, pair_id, H, inlier, n_inliers, best_t=None,
                        iters_used=None, stream=None):
        self._chk(self.lib.lp_ransac_prior(self.h, _ptr(pts), M_cap, _ptr(d_M), _ptr(prior), int(guided_iters),
                                           pair_id, _ptr(H), _ptr(inlier), _ptr(n_inliers), _ptr(best_t),
                                           _ptr(iters_used), _stream(stream)), "lp_ransac_prior")

    def lp_diag_last_ransac_counts(self, n: int) -> list[int]:
        """n = T after lp_ransac, guided_iters + T after lp_ransac_prior."""
        arr = (C.c_int32 * n)()
        self._chk(self.lib.lp_diag_last_ransac_counts(self.h, C.cast(arr, C.c_void_p), n),
                  "lp_diag_last_ransac_counts")
        return list(arr)

    def lp_set_proposal(self, mlp, guided_iters: int = 64):
        """Guide the stitch calls' RANSAC with an Mlp (None detaches it)."""
        self._proposal = mlp                  # keep the network alive while attached
        self._chk(self.lib.lp_set_proposal(self.h, mlp.h if mlp is not None else None, int(guided_iters)),
                  "lp_set_proposal")

    def lp_set_profiling(self, on: bool = True):
        self._chk(self.lib.lp_set_profiling(self.h, int(bool(on))), "lp_set_profiling")

    def lp_diag_set_batch_hold(self, hold: int):
        self._chk(self.lib.lp_diag_set_batch_hold(self.h, int(hold)), "lp_diag_set_batch_hold")

    def lp_set_autotune(self, on: bool = True):
        self._chk(self.lib.lp_set_autotune(self.h, int(bool(on))), "lp_set_autotune")

    def lp_autotune_table(self) -> list[dict]:
        """Tuned classes: log2 buckets of NA and NB, S, pass-1 stride, tuned and built-in times (us)."""
        n = C.c_int32()
        self._chk(self.lib.lp_autotune_table(self.h, None, 0, C.byref(n)), "lp_autotune_table")
        rows = (C.c_int32 * (6 * max(n.value, 1)))()
        self._chk(self.lib.lp_autotune_table(self.h, rows, n.value, C.byref(n)), "lp_autotune_table")
        keys = ("log2_NA", "log2_NB", "splits", "pass1_stride", "tuned_us", "builtin_us")
        return [dict(zip(keys, rows[6 * k:6 * k + 6])) for k in range(n.value)]

    def lp_diag_last_match_kernel_ms(self) -> float:
        v = C.c_float()
        self._chk(self.lib.lp_diag_last_match_kernel_ms(self.h, C.byref(v)), "lp_diag_last_match_kernel_ms")
        return v.value

    def lp_mosaic_render(self, images, G, round_of, canvas, canvas_w, canvas_h, canvas_pitch, cover=None,
                         stream=None):
        """images: list of (device uint8 tensor, H, W, pitch, channels); G, round_of: lp_mosaic_plan's."""
        arr = (lp_image * len(images))(*[lp_image(_ptr(t), H, W, p, ch) for (t, H, W, p, ch) in images])
        Gh = np.ascontiguousarray(G, np.float64).reshape(-1)
        r = np.ascontiguousarray(round_of, np.int32)
        self._chk(self.lib.lp_mosaic_render(self.h, C.cast(arr, C.c_void_p), len(images),
                                            Gh.ctypes.data_as(C.c_void_p), r.ctypes.data_as(C.c_void_p), _ptr(canvas),
                                            int(canvas_w), int(canvas_h), int(canvas_pitch), _ptr(cover),
                                            _stream(stream)), "lp_mosaic_render")

    def lp_sync_status(self):
        return self.lib.lp_sync_status(self.h)

    def lp_diag_last_rescans(self) -> int:
        v = C.c_int64()
        self._chk(self.lib.lp_diag_last_rescans(self.h, C.byref(v)), "lp_diag_last_rescans")
        return v.value


class Mlp:
    """Owns an lp_mlp: the learned inlier-probability network (8-64-64-1)."""

    def __init__(self, seed: int = 0):
        self.lib = load()
        h = C.c_void_p()
        r = self.lib.lp_mlp_create(C.byref(h), int(seed))
        if r != LP_OK:
            raise LpError(r, "lp_mlp_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, r, what):
        if r != LP_OK:
            raise LpError(r, what)

    def lp_mlp_set_params(self, params):
        """params: host array-like of MLP_PARAMS floats (resets Adam)."""
        a = (C.c_float * MLP_PARAMS)(*[float(v) for v in params])
        self._chk(self.lib.lp_mlp_set_params(self.h, C.cast(a, C.c_void_p)), "lp_mlp_set_params")

    def lp_mlp_get_params(self) -> list[float]:
        a = (C.c_float * MLP_PARAMS)()
        self._chk(self.lib.lp_mlp_get_params(self.h, C.cast(a, C.c_void_p)), "lp_mlp_get_params")
        return list(a)

    def lp_mlp_get_state(self):
        """(master, m, v) as float32 numpy arrays, Adam step count."""
        a = np.zeros(3 * MLP_PARAMS, np.float32)
        st = C.c_int32()
        self._chk(self.lib.lp_mlp_get_state(self.h, a.ctypes.data_as(C.c_void_p), C.byref(st)), "lp_mlp_get_state")
        return a[:MLP_PARAMS], a[MLP_PARAMS:2 * MLP_PARAMS], a[2 * MLP_PARAMS:], st.value

    def lp_mlp_save(self, path: str):
        self._chk(self.lib.lp_mlp_save(self.h, os.fsencode(path)), "lp_mlp_save")

    def lp_mlp_load(self, path: str):
        self._chk(self.lib.lp_mlp_load(self.h, os.fsencode(path)), "lp_mlp_load")

    def lp_mlp_forward(self, feat, M_cap, d_M, prob, logit=None, stream=None):
        self._chk(self.lib.lp_mlp_forward(self.h, _ptr(feat), M_cap, _ptr(d_M), _ptr(prob), _ptr(logit),
                                          _stream(stream)), "lp_mlp_forward")

    def lp_mlp_train_step(self, feat, label, B, lr, loss=None, stream=None):
        self._chk(self.lib.lp_mlp_train_step(self.h, _ptr(feat), _ptr(label), B, float(lr), _ptr(loss),
                                             _stream(stream)), "lp_mlp_train_step")


def lp_mosaic_plan(n_images, pairs, HM, valid, sizes):
    """Sec. 4 rounds on the host.  pairs [(a, b)], HM [P, 9] or [P, 3, 3] (host
    arrays), valid [P], sizes [(H, W)].  Returns dict(G [N, 3, 3], round [N],
    ref [N], canvas (h, w))."""
    pr = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 2))
    Hm = np.ascontiguousarray(np.asarray(HM, np.float64).reshape(-1, 9))
    v = np.ascontiguousarray(np.asarray(valid, np.uint8))
    Hs = np.ascontiguousarray([s[0] for s in sizes], np.int32)
    Ws = np.ascontiguousarray([s[1] for s in sizes], np.int32)
    G = np.zeros((n_images, 9), np.float64)
    rnd = np.zeros(n_images, np.int32)
    ref = np.zeros(n_images, np.int32)
    cw, ch = C.c_int32(), C.c_int32()
    vp = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    r = load().lp_mosaic_plan(int(n_images), vp(pr), len(pr), vp(Hm), vp(v), vp(Hs), vp(Ws), vp(G), vp(rnd), vp(ref),
                              C.byref(cw), C.byref(ch))
    if r != LP_OK:
        raise LpError(r, "lp_mosaic_plan")
    return dict(G=G.reshape(-1, 3, 3), round=rnd, ref=ref, canvas=(ch.value, cw.value))


def lp_num_keypoints(H, W, Ls) -> int:
    arr = (C.c_int * len(Ls))(*[int(v) for v in Ls])
    return int(load().lp_num_keypoints(H, W, C.cast(arr, C.c_void_p), len(Ls)))


def lp_ransac_static(pts, M_cap, d_M, iters, thresh_px, seed, pair_id, H, inlier, n_inliers, best_t=None,
                     stream=None):
    """The allocation-free RANSAC entry point (no context; fixed scratch in
    the library).  Same results as Context.lp_ransac for the same settings."""
    r = load().lp_ransac_static(_ptr(pts), M_cap, _ptr(d_M), int(iters), float(thresh_px), int(seed), int(pair_id),
                                _ptr(H), _ptr(inlier), _ptr(n_inliers), _ptr(best_t), _stream(stream))
    if r != LP_OK:
        raise LpError(r, "lp_ransac_static")


def _diag(name, *args):
    r = getattr(load(), name)(*args)
    if r != LP_OK:
        raise LpError(r, name)


def lp_diag_orient_bins(out, stream=None):
    _diag("lp_diag_orient_bins", _ptr(out), _stream(stream))


def lp_diag_orient_weights(out, stream=None):
    _diag("lp_diag_orient_weights", _ptr(out), _stream(stream))


def lp_diag_philox(ctr, n, key0, key1, out, stream=None):
    _diag("lp_diag_philox", _ptr(ctr), n, key0, key1, _ptr(out), _stream(stream))


def lp_diag_gray(rgb, n, gray, stream=None):
    _diag("lp_diag_gray", _ptr(rgb), n, _ptr(gray), _stream(stream))


# ---------------------------------------------------------------------------
# Convenience layer: whole-image / whole-pair calls on torch tensors.
# ---------------------------------------------------------------------------
def pitched_device(img) -> tuple[torch.Tensor, int]:
    """(H, W) or (H, W, 3) uint8 array/tensor -> device buffer with a 16-byte row pitch."""
    t = torch.as_tensor(img)
    H = t.shape[0]
    row = t.shape[1] * (t.shape[2] if t.dim() == 3 else 1)
    pitch = (row + 15) // 16 * 16
    buf = torch.zeros((H, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :row] = t.reshape(H, row).to("cuda")
    return buf, pitch


class Features:
    def __init__(self, gray, H, W, gpitch, kp, ori, desc, desc16, valid):
        self.gray, self.H, self.W, self.gpitch = gray, H, W, gpitch
        self.kp, self.ori, self.desc, self.desc16, self.valid = kp, ori, desc, desc16, valid


def features(ctx: Context, img, stream=None) -> Features:
    """lp_detect + lp_describe for one image (numpy or tensor, gray or RGB)."""
    buf, pitch = pitched_device(img)
    H, W = int(buf.shape[0]), int(torch.as_tensor(img).shape[1])
    ch = 3 if torch.as_tensor(img).dim() == 3 else 1
    K = lp_num_keypoints(H, W, ctx.Ls)
    dev = "cuda"
    kp = torch.empty(max(K, 1), dtype=torch.int32, device=dev)
    gray = torch.empty(H * W + 16, dtype=torch.uint8, device=dev) if ch == 3 else None
    ctx.lp_detect(buf, H, W, pitch, ch, kp, gray, stream)
    g, gp = (gray, W) if ch == 3 else (buf, pitch)
    ori = torch.empty(max(K, 1), dtype=torch.uint8, device=dev)
    desc = torch.empty((max(K, 1), 128), dtype=torch.float32, device=dev)
    bf = ctx.cfg.precision == PREC_BF16
    desc16 = torch.empty((max(K, 1), 128), dtype=torch.bfloat16, device=dev) if bf else None
    valid = torch.empty(max(K, 1), dtype=torch.uint8, device=dev)
    ctx.lp_describe(g, H, W, gp, kp, K, ori, desc, desc16, valid, stream)
    return Features(g, H, W, gp, kp[:K], ori[:K], desc[:K], None if desc16 is None else desc16[:K], valid[:K])


def match(ctx: Context, fa: Features, fb: Features, stream=None):
    NA, NB = fa.desc.shape[0], fb.desc.shape[0]
    m = torch.empty(max(NA, 1), dtype=torch.int32, device="cuda")
    d1 = torch.empty(max(NA, 1), dtype=torch.float32, device="cuda")
    d2 = torch.empty(max(NA, 1), dtype=torch.float32, device="cuda")
    ctx.lp_match(fa.desc, fa.desc16, fa.valid, NA, fb.desc, fb.desc16, fb.valid, NB, m, d1, d2, stream)
    return m[:NA], d1[:NA], d2[:NA]


def ransac(ctx: Context, pts: torch.Tensor, pair_id: int = 0, d_M=None, stream=None):
    M = pts.shape[0]
    H = torch.empty(9, dtype=torch.float64, device="cuda")
    inl = torch.empty(max(M, 1), dtype=torch.uint8, device="cuda")
    n = torch.empty(1, dtype=torch.int32, device="cuda")
    bt = torch.empty(1, dtype=torch.int32, device="cuda")
    p = pts if M > 0 else torch.zeros((1, 4), dtype=torch.float32, device="cuda")
    ctx.lp_ransac(p, M, d_M, pair_id, H, inl, n, bt, stream)
    return H.view(3, 3), inl[:M], n, bt
