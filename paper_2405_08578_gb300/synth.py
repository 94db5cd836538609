"""Seeded synthetic inputs shaped like the paper's image-stitching workloads.

This module only *makes pictures and ground-truth homographies*; it holds none of
the LP-SIFT arithmetic (no detection, description, matching or fitting).  Both
the CUDA path and the CPU oracle consume its output, so it is the one piece of
code they share.

Recipe (a stand-in for the paper's Dataset-A/B photographs, Sec. 3.1, which are
not available):

* an FP64 "scene" canvas: base intensity 128, plus Gaussian blobs (centre
  uniform on the canvas, sigma ~ U[3, 40] px, amplitude ~ U[-80, 80]) at a
  density of 200 blobs per 640x480 pixels, plus band-limited noise (unit normal
  per pixel, Gaussian blur sigma = 1.5 px, rescaled to std 6);
* image A is an axis-aligned crop of the canvas; image B is the canvas seen
  through a known homography ``H`` (A pixel (x, y) -> B pixel H(x, y), the
  direction of Eq. 7), rendered by bilinear sampling of the FP64 canvas, so the
  part of B outside A still has scene content;
* ``clip(round-half-even(.), 0, 255)`` to uint8.  RGB views use per-channel
  gains (1.0, 0.9, 1.1) about 128 plus independent band-limited noise (std 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

try:  # scipy is present on both machines; keep a numpy fallback for the blur
    from scipy.ndimage import gaussian_filter as _gauss
except Exception:  # pragma: no cover
    _gauss = None

BLOB_DENSITY = 200.0 / (640.0 * 480.0)


def _blur(x: np.ndarray, sigma: float) -> np.ndarray:
    if _gauss is not None:
        return _gauss(x, sigma, mode="reflect")
    r = int(math.ceil(4 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    y = np.apply_along_axis(lambda v: np.convolve(np.pad(v, r, mode="reflect"), k, "valid"), 0, x)
    return np.apply_along_axis(lambda v: np.convolve(np.pad(v, r, mode="reflect"), k, "valid"), 1, y)


def band_noise(rng: np.random.Generator, h: int, w: int, std: float, sigma: float = 1.5) -> np.ndarray:
    n = _blur(rng.standard_normal((h, w)), sigma)
    return n * (std / max(n.std(), 1e-12))


def scene(h: int, w: int, seed: int, n_blobs: int | None = None) -> np.ndarray:
    """FP64 canvas of size h x w (rows x cols)."""
    rng = np.random.default_rng(seed)
    if n_blobs is None:
        n_blobs = max(1, int(round(BLOB_DENSITY * h * w)))
    c = np.full((h, w), 128.0)
    cy = rng.uniform(0, h, n_blobs)
    cx = rng.uniform(0, w, n_blobs)
    sg = rng.uniform(3.0, 40.0, n_blobs)
    amp = rng.uniform(-80.0, 80.0, n_blobs)
    for k in range(n_blobs):
        r = int(math.ceil(3.5 * sg[k]))
        y0, y1 = max(0, int(cy[k]) - r), min(h, int(cy[k]) + r + 1)
        x0, x1 = max(0, int(cx[k]) - r), min(w, int(cx[k]) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = (np.arange(y0, y1) - cy[k])[:, None]
        xx = (np.arange(x0, x1) - cx[k])[None, :]
        c[y0:y1, x0:x1] += amp[k] * np.exp(-(yy * yy + xx * xx) / (2.0 * sg[k] * sg[k]))
    c += band_noise(rng, h, w, 6.0)
    return c


def to_u8(x: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(x), 0, 255).astype(np.uint8)


def similarity(theta_deg: float, scale: float, tx: float, ty: float, cx: float, cy: float) -> np.ndarray:
    """H = T(tx, ty) . C . R(theta) . S(scale) . C^-1 (about the point (cx, cy))."""
    t = math.radians(theta_deg)
    c, s = math.cos(t) * scale, math.sin(t) * scale
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    C = np.array([[1.0, 0.0, cx], [0.0, 1.0, cy], [0.0, 0.0, 1.0]])
    Ci = np.array([[1.0, 0.0, -cx], [0.0, 1.0, -cy], [0.0, 0.0, 1.0]])
    T = np.array([[1.0, 0.0, tx], [0.0, 1.0, ty], [0.0, 0.0, 1.0]])
    return T @ C @ R @ Ci


def bilinear(canvas: np.ndarray, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    h, w = canvas.shape
    X = np.clip(X, 0.0, w - 1.000001)
    Y = np.clip(Y, 0.0, h - 1.000001)
    x0 = np.floor(X).astype(np.int64)
    y0 = np.floor(Y).astype(np.int64)
    fx = X - x0
    fy = Y - y0
    v00 = canvas[y0, x0]
    v01 = canvas[y0, x0 + 1]
    v10 = canvas[y0 + 1, x0]
    v11 = canvas[y0 + 1, x0 + 1]
    return (v00 * (1 - fx) + v01 * fx) * (1 - fy) + (v10 * (1 - fx) + v11 * fx) * fy


def _apply(H: np.ndarray, x: np.ndarray, y: np.ndarray):
    w = H[2, 0] * x + H[2, 1] * y + H[2, 2]
    return (H[0, 0] * x + H[0, 1] * y + H[0, 2]) / w, (H[1, 0] * x + H[1, 1] * y + H[1, 2]) / w


@dataclass
class Pair:
    A: np.ndarray          # uint8, (h, w) or (h, w, 3)
    B: np.ndarray          # uint8, same shape as A
    H: np.ndarray          # 3x3 float64, A pixel -> B pixel (x = column, y = row)


def make_pair(h: int, w: int, H: np.ndarray, seed: int, rgb: bool = False, margin: int = 8) -> Pair:
    """Render A (a crop of the scene) and B (the scene through H) of size h x w."""
    Hi = np.linalg.inv(H)
    # footprint of B in A's coordinates
    cx = np.array([0, w - 1, 0, w - 1], dtype=np.float64)
    cy = np.array([0, 0, h - 1, h - 1], dtype=np.float64)
    fx, fy = _apply(Hi, cx, cy)
    xmin = min(0.0, fx.min()) - margin
    ymin = min(0.0, fy.min()) - margin
    xmax = max(w - 1.0, fx.max()) + margin
    ymax = max(h - 1.0, fy.max()) + margin
    ox, oy = -int(math.floor(xmin)), -int(math.floor(ymin))
    ch, cw = int(math.ceil(ymax)) + oy + 2, int(math.ceil(xmax)) + ox + 2
    base = scene(ch, cw, seed)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    bx, by = _apply(Hi, xs, ys)
    if not rgb:
        A = to_u8(base[oy:oy + h, ox:ox + w])
        B = to_u8(bilinear(base, bx + ox, by + oy))
        return Pair(A, B, H)
    rng = np.random.default_rng(seed + 7919)
    gains = (1.0, 0.9, 1.1)
    A = np.empty((h, w, 3), np.uint8)
    B = np.empty((h, w, 3), np.uint8)
    for c, g in enumerate(gains):
        chan = 128.0 + g * (base - 128.0) + band_noise(rng, ch, cw, 2.0)
        A[:, :, c] = to_u8(chan[oy:oy + h, ox:ox + w])
        B[:, :, c] = to_u8(bilinear(chan, bx + ox, by + oy))
    return Pair(A, B, H)


# --------------------------------------------------------------------------
# Named workloads (sizes from the paper's Sec. 3-4 scale range)
# --------------------------------------------------------------------------
PAIR_640x480_LS = (8, 16, 32)
PAIR_2688x1600_LS = (16, 32, 64, 128)


def pair_640x480(seed: int = 0) -> Pair:
    """640x480 gray pair: B = A through T(220, 0) . R(5 deg) . S(1.05) about the centre."""
    h, w = 480, 640
    H = similarity(5.0, 1.05, 220.0, 0.0, w / 2.0, h / 2.0)
    return make_pair(h, w, H, seed)


def pair_640x480_random(seed: int) -> Pair:
    """640x480 gray pair with a seeded similarity: rotation U[-10, 10] deg,
    scale U[0.9, 1.1], x shift U[0.2, 0.5] w (either sign), y shift
    U[-0.1, 0.1] h.  Training and held-out pairs of the learned proposal."""
    h, w = 480, 640
    rng = np.random.default_rng(20_000 + seed)
    th = rng.uniform(-10.0, 10.0)
    sc = rng.uniform(0.9, 1.1)
    tx = rng.uniform(0.2, 0.5) * w * (1 if rng.uniform() < 0.5 else -1)
    ty = rng.uniform(-0.1, 0.1) * h
    return make_pair(h, w, similarity(th, sc, tx, ty, w / 2.0, h / 2.0), seed)


def pair_2688x1600(seed: int = 0, rgb: bool = True) -> Pair:
    """2688x1600 RGB pair: rotation U[-10, 10] deg, scale U[0.9, 1.1], ~40% overlap."""
    h, w = 1600, 2688
    rng = np.random.default_rng(10_000 + seed)
    th = rng.uniform(-10.0, 10.0)
    sc = rng.uniform(0.9, 1.1)
    tx = 0.6 * w * (1 if rng.uniform() < 0.5 else -1)
    ty = rng.uniform(-0.05, 0.05) * h
    H = similarity(th, sc, tx, ty, w / 2.0, h / 2.0)
    return make_pair(h, w, H, seed, rgb=rgb)


# Table 2's LP-SIFT rows: image size (width x height, as printed) and the
# window-size set [a, b], read as the two scales {a, b}.
TABLE2 = {
    "mountain": (602, 400, (32, 40)),
    "street_view": (653, 490, (32, 40)),
    "terrain": (1024, 768, (32, 64)),
    "building": (1080, 1920, (100, 128)),
    "campus_translation": (3072, 4096, (256, 512)),
    "campus_rotation": (3072, 4096, (256, 512)),
}


def table2_pair(name: str, seed: int = 0) -> tuple[Pair, tuple[int, ...]]:
    """Gray stand-in for a Table 2 pair: the printed size and L set, B = A
    through a seeded rigid motion about the centre (rotation U[-5, 5] deg, or
    U[8, 12] deg for the rotation pair; x shift 0.5 w; y shift U[-0.05, 0.05]
    h), about half the frame overlapping."""
    w, h, Ls = TABLE2[name]
    rng = np.random.default_rng(30_000 + seed + 97 * sorted(TABLE2).index(name))
    th = rng.uniform(8.0, 12.0) if name == "campus_rotation" else rng.uniform(-5.0, 5.0)
    H = similarity(th, 1.0, 0.5 * w, rng.uniform(-0.05, 0.05) * h, w / 2.0, h / 2.0)
    return make_pair(h, w, H, seed), Ls


def uneven_pairs(n: int = 64, seed: int = 2, long_lo: int = 480, long_hi: int = 4096, rgb: bool = False) -> list[Pair]:
    """Independent pairs of uneven sizes: long side U[long_lo, long_hi] (integer),
    aspect U[4/3, 16/9] (landscape), and B through a similarity drawn like the
    2688x1600 pair's (rotation U[-10, 10] deg, scale U[0.9, 1.1], x shift 0.6 w
    of either sign, y shift U[-0.05, 0.05] h: about 40% overlap)."""
    return [make_pair(*spec, rgb=rgb) for spec in uneven_pair_specs(n, seed, long_lo, long_hi)]


def uneven_pair_specs(n: int = 64, seed: int = 2, long_lo: int = 480, long_hi: int = 4096) -> list[tuple]:
    """The (h, w, H, canvas seed) of each pair of uneven_pairs, in order; each
    make_pair(*spec) can then be built independently."""
    rng = np.random.default_rng(40_000 + seed)
    out = []
    for q in range(n):
        w = int(rng.integers(long_lo, long_hi + 1))
        h = max(16, int(round(w / rng.uniform(4.0 / 3.0, 16.0 / 9.0))))
        th = rng.uniform(-10.0, 10.0)
        sc = rng.uniform(0.9, 1.1)
        tx = 0.6 * w * (1 if rng.uniform() < 0.5 else -1)
        ty = rng.uniform(-0.05, 0.05) * h
        out.append((h, w, similarity(th, sc, tx, ty, w / 2.0, h / 2.0), 1000 * seed + q))
    return out


def small_pair(h: int, w: int, seed: int, theta_deg: float = 4.0, scale: float = 1.03,
               shift: float = 0.3, rgb: bool = False) -> Pair:
    """Small pair for parity tests: similarity about the centre, x shift = shift * w."""
    H = similarity(theta_deg, scale, shift * w, 0.0, w / 2.0, h / 2.0)
    return make_pair(h, w, H, seed, rgb=rgb)


def random_u8(shape, seed: int, lo: int = 0, hi: int = 256) -> np.ndarray:
    return np.random.default_rng(seed).integers(lo, hi, size=shape, dtype=np.int64).astype(np.uint8)


def pitched(img: np.ndarray, pitch_multiple: int = 16) -> tuple[np.ndarray, int]:
    """Copy an image into a buffer whose row pitch (bytes) is a multiple of 16.

    Returns (buffer of shape (h, pitch) uint8, pitch).  The valid pixels are the
    first w*channels bytes of each row.
    """
    h = img.shape[0]
    row = img.shape[1] * (img.shape[2] if img.ndim == 3 else 1)
    pitch = (row + pitch_multiple - 1) // pitch_multiple * pitch_multiple
    buf = np.zeros((h, pitch), np.uint8)
    buf[:, :row] = img.reshape(h, row)
    return buf, pitch


@dataclass
class Batch:
    images: list           # uint8 tiles (h, w, 3), shuffled order
    H: dict                # (a, b) -> 3x3 homography from tile a to tile b (shuffled indices)
    order: np.ndarray      # order[k] = original grid position (row-major) of shuffled tile k


def batch_3x3(seed: int = 1, h: int = 1600, w: int = 2688, canvas_h: int = 4200, canvas_w: int = 7200,
              rgb: bool = True) -> Batch:
    """Nine h x w tiles of one scene on a 3 x 3 layout.

    Seam overlaps ~ U[0.20, 0.35] of the tile side; each tile sees the scene
    through its own perturbation (rotation U[-3, 3] deg, scale U[0.98, 1.02]
    about the tile centre); the tiles are then shuffled.  Tile k's pixel q maps
    to scene point C_k q; the homography from tile a to tile b is C_b^-1 C_a.
    """
    rng = np.random.default_rng(seed)
    ox = rng.uniform(0.20, 0.35, 2)
    oy = rng.uniform(0.20, 0.35, 2)
    xs = [0.0, w * (1 - ox[0]), w * (1 - ox[0]) + w * (1 - ox[1])]
    ys = [0.0, h * (1 - oy[0]), h * (1 - oy[0]) + h * (1 - oy[1])]
    span_x, span_y = xs[2] + w, ys[2] + h
    x0, y0 = (canvas_w - span_x) / 2.0, (canvas_h - span_y) / 2.0
    base = scene(canvas_h, canvas_w, seed)
    chans = None
    if rgb:
        nrng = np.random.default_rng(seed + 7919)
        chans = [128.0 + g * (base - 128.0) + band_noise(nrng, canvas_h, canvas_w, 2.0) for g in (1.0, 0.9, 1.1)]
    Cs, tiles = [], []
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    for r in range(3):
        for c in range(3):
            th = rng.uniform(-3.0, 3.0)
            sc = rng.uniform(0.98, 1.02)
            tx, ty = x0 + xs[c], y0 + ys[r]
            C = np.array([[1.0, 0, tx], [0, 1.0, ty], [0, 0, 1.0]]) @ similarity(th, sc, 0.0, 0.0, w / 2.0, h / 2.0)
            X, Y = _apply(C, xx, yy)
            if rgb:
                t = np.empty((h, w, 3), np.uint8)
                for k in range(3):
                    t[:, :, k] = to_u8(bilinear(chans[k], X, Y))
            else:
                t = to_u8(bilinear(base, X, Y))
            Cs.append(C)
            tiles.append(t)
    order = np.random.default_rng(seed).permutation(9)
    images = [tiles[k] for k in order]
    Hs = {}
    for a in range(9):
        for b in range(9):
            if a != b:
                Hab = np.linalg.inv(Cs[order[b]]) @ Cs[order[a]]
                Hs[(a, b)] = Hab / Hab[2, 2]
    return Batch(images, Hs, order)
