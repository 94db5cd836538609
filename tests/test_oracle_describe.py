"""Pins for the oracle's Sec. 2.3 functions: orientation and the 128-d descriptor."""
import math

import numpy as np
import pytest

import oracle


def test_orient_weight_exhaustive_integer_bracket():
    # m = round(65536 sqrt(s)) <=> (2m-1)^2 <= 4 * 2^32 * s < (2m+1)^2 (exact ints)
    s = np.arange(0, 2 * 255 * 255 + 1, dtype=np.int64)
    m = np.array([oracle.orient_weight(int(v)) for v in s], np.int64)
    N4 = s * (1 << 34)
    lo = (2 * m - 1) ** 2
    hi = (2 * m + 1) ** 2
    assert np.all((lo <= N4) | (m == 0)) and np.all(N4 < hi)


def _exact_bin(a, b):
    import mpmath
    mpmath.mp.dps = 40
    phi = mpmath.atan2(b, a)
    if phi < 0:
        phi += 2 * mpmath.pi
    return int(mpmath.floor(phi * 36 / (2 * mpmath.pi)))


def test_orient_bin_exhaustive():
    # every integer gradient (a, b) in [-255, 255]^2: the oracle's bin equals
    # the bin of the exact angle; pairs closest to a bin edge are re-derived
    # at 40 digits.
    a, b = np.meshgrid(np.arange(-255, 256), np.arange(-255, 256), indexing="ij")
    a = a.ravel()
    b = b.ravel()
    ob = np.array([oracle.orient_bin(int(x), int(y)) for x, y in zip(a, b)])
    phi = np.arctan2(b, a)
    phi = np.where(phi < 0, phi + 2 * np.pi, phi)
    q = phi * 36 / (2 * np.pi)
    axis = (a == 0) | (b == 0)
    frac = np.abs(q - np.rint(q))
    assert frac[~axis].min() > 6e-5                      # no pair sits on an edge
    nb = np.floor(q).astype(int) % 36
    nb[axis & (b == 0) & (a > 0)] = 0
    nb[axis & (b == 0) & (a < 0)] = 18
    nb[axis & (a == 0) & (b > 0)] = 9
    nb[axis & (a == 0) & (b < 0)] = 27
    nb[(a == 0) & (b == 0)] = 0
    assert np.array_equal(ob, nb)
    close = np.argsort(np.where(axis, 1.0, frac))[:40]
    pytest.importorskip("mpmath")
    for i in close:
        assert ob[i] == _exact_bin(int(a[i]), int(b[i]))


def _kp(H, W, y, x):
    return np.array([y * W + x], np.uint32)


@pytest.mark.parametrize("img,want", [("row", 0), ("col", 9), ("negcol", 27), ("diag", 4), ("negrow", 18)])
def test_orient_ramps(img, want):
    H = W = 64
    yy, xx = np.mgrid[0:H, 0:W]
    g = {"row": yy, "col": xx, "negcol": 255 - xx, "diag": (xx + yy) // 1, "negrow": 255 - 2 * yy}[img]
    g = np.clip(g, 0, 255).astype(np.uint8)
    ori = oracle.orient(g, _kp(H, W, 30, 31), np.array([4], np.int32))
    assert ori[0] == want


def _rot_setup(seed=5, H=72, W=96):
    rng = np.random.default_rng(seed)
    g = (rng.integers(0, 256, size=(H, W)) // 1).astype(np.uint8)
    B = np.ascontiguousarray(np.rot90(g))           # B[i, j] = g[j, W-1-i]
    ys = rng.integers(0, H, 40)
    xs = rng.integers(0, W, 40)
    idxA = (ys * W + xs).astype(np.uint32)
    # A (y, x) -> B (W-1-x, y); B has width H
    idxB = ((W - 1 - xs) * H + ys).astype(np.uint32)
    ws = rng.integers(1, 6, 40).astype(np.int32)
    return g, B, idxA, idxB, ws


def test_orient_rotation_90_histogram_roll():
    # Rotating the image by 90 degrees rotates every Eq. 5 gradient by 90
    # degrees, i.e. 9 bins, and the symmetric window onto itself.
    g, B, ia, ib, ws = _rot_setup()
    oa, ha = oracle.orient(g, ia, ws, want_hist=True)
    ob, hb = oracle.orient(B, ib, ws, want_hist=True)
    assert np.array_equal(hb, np.roll(ha, 9, axis=1))
    unique = np.array([(h == h.max()).sum() == 1 for h in ha])
    assert unique.sum() > 30
    assert np.array_equal(ob[unique], (oa[unique] + 9) % 36)


def test_describe_rotation_90_invariant():
    g, B, ia, ib, ws = _rot_setup(seed=8)
    oa = np.random.default_rng(3).integers(0, 36, len(ia)).astype(np.uint8)
    ob = ((oa.astype(int) + 9) % 36).astype(np.uint8)
    da, va = oracle.describe(g, ia, ws, oa)
    db, vb = oracle.describe(B, ib, ws, ob)
    assert np.array_equal(va, vb)
    assert np.abs(da - db).max() < 1e-9


def _ramp_desc_rotated(k):
    """Closed form for I(r, c) = r with the grid turned by (k+0.5)*10 deg."""
    th = math.radians((k + 0.5) * 10)
    a, b = 2 * math.cos(th), -2 * math.sin(th)
    o = 8 * math.atan2(b, a) / (2 * math.pi) % 8
    b0 = int(math.floor(o))
    t = o - b0
    v = np.zeros(8)
    v[b0] += 1 - t
    v[(b0 + 1) % 8] += t
    full = np.tile(v, 16)
    full /= np.linalg.norm(full)
    full = np.minimum(full, 0.2)
    return full / np.linalg.norm(full)


def test_describe_ramp_closed_forms():
    H = W = 96
    yy, xx = np.mgrid[0:H, 0:W]
    kp = _kp(H, W, 48, 47)
    ws = np.array([3], np.int32)
    # upright: one bin per cell, 16 cells -> every entry 1/4
    d, v = oracle.describe(yy.astype(np.uint8), kp, ws, None)
    want = np.zeros(128)
    want[0::8] = 0.25
    assert v[0] == 1 and np.abs(d[0] - want).max() < 1e-12
    d, v = oracle.describe(xx.astype(np.uint8), kp, ws, None)
    want = np.zeros(128)
    want[2::8] = 0.25                                  # gradient along +column = 90 deg = bin 2
    assert np.abs(d[0] - want).max() < 1e-12
    # rotated grid: bilinear sampling of a linear image is exact
    for k in (0, 7, 13, 22, 35):
        d, v = oracle.describe(yy.astype(np.uint8), kp, ws, np.array([k], np.uint8))
        assert np.abs(d[0] - _ramp_desc_rotated(k)).max() < 1e-12, k


def test_describe_unit_norm_and_invalid():
    rng = np.random.default_rng(4)
    g = rng.integers(0, 256, size=(60, 70)).astype(np.uint8)
    idx = rng.integers(0, 60 * 70, 50).astype(np.uint32)
    ws = rng.integers(1, 5, 50).astype(np.int32)
    ori = rng.integers(0, 36, 50).astype(np.uint8)
    d, v = oracle.describe(g, idx, ws, ori)
    assert v.all()
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    c = np.full((30, 30), 9, np.uint8)
    d, v = oracle.describe(c, np.array([0, 465], np.uint32), np.array([2, 3], np.int32), None)
    assert not v.any() and not d.any()


def test_describe_upright_equals_integer_eq5():
    # Upright samples sit on pixels, so the gradient is exactly Eq. 5; this
    # numpy restatement uses integer differences and no interpolation.
    rng = np.random.default_rng(9)
    H, W = 40, 44
    g = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    y, x, s = 20, 21, 3
    d, _ = oracle.describe(g, _kp(H, W, y, x), np.array([s], np.int32), None)
    G = g.astype(np.int64)
    h = np.zeros(128)
    R = 2 * s
    for u in range(-R, R):
        for v in range(-R, R):
            a = G[y + u + 1, x + v] - G[y + u - 1, x + v]
            b = G[y + u, x + v + 1] - G[y + u, x + v - 1]
            m = math.hypot(a, b)
            if m == 0:
                continue
            o = (8 * math.atan2(b, a) / (2 * math.pi)) % 8
            b0 = int(o)
            t = o - b0
            cell = ((u + R) // s) * 4 + (v + R) // s
            h[cell * 8 + b0] += m * (1 - t)
            h[cell * 8 + (b0 + 1) % 8] += m * t
    h /= np.linalg.norm(h)
    h = np.minimum(h, 0.2)
    h /= np.linalg.norm(h)
    assert np.abs(d[0] - h).max() < 1e-12


def test_describe_offset_and_gain_invariance():
    # Eq. 5 takes intensity differences only: a constant offset leaves every
    # gradient, the orientation histogram and the descriptor unchanged.  A gain
    # of 2 doubles every gradient (exactly, bilinear taps included), and the L2
    # normalisation removes it.
    rng = np.random.default_rng(12)
    g = rng.integers(0, 100, size=(70, 80)).astype(np.uint8)
    idx = (rng.integers(20, 50, 40) * 80 + rng.integers(20, 60, 40)).astype(np.uint32)
    ws = rng.integers(1, 5, 40).astype(np.int32)
    ori = oracle.orient(g, idx, ws)
    assert np.array_equal(oracle.orient(g + 37, idx, ws), ori)
    d, v = oracle.describe(g, idx, ws, ori)
    d1, v1 = oracle.describe(g + 37, idx, ws, ori)
    d2, v2 = oracle.describe(g * 2, idx, ws, ori)
    assert v.all() and np.array_equal(v, v1) and np.array_equal(v, v2)
    assert np.abs(d1 - d).max() < 1e-12 and np.abs(d2 - d).max() < 1e-12
    # the invariance is not vacuous: another orientation changes the descriptors
    d3, _ = oracle.describe(g, idx, ws, ((ori.astype(int) + 5) % 36).astype(np.uint8))
    assert np.abs(d3 - d).max(axis=1).min() > 1e-3


def test_orient_exact_tie_lowest_bin_wins():
    # I = 3 max(r - y0, c - x0): above the diagonal every gradient is (6, 0)
    # (bin 0), below it (0, 6) (bin 9), on it (3, 3) (bin 4).  The window is
    # symmetric about the diagonal, so bins 0 and 9 tie exactly and the lower
    # bin must win.
    H = W = 40
    yy, xx = np.mgrid[0:H, 0:W]
    g = (100 + 3 * np.maximum(yy - 20, xx - 20)).astype(np.uint8)
    ori, hist = oracle.orient(g, _kp(H, W, 20, 20), np.array([3], np.int32), want_hist=True)
    h = hist[0]
    assert h[0] == h[9] > h[4] > 0 and h.sum() == h[0] + h[9] + h[4]
    assert ori[0] == 0
