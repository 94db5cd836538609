"""Pins for the paper-literal hard 8-direction histogram of Sec. 2.3 in the
oracle: the sector rule (or_octant), the fixed-point turn table (or_turn_fx)
and the descriptor built with them (or_describe_ex, hard = 1)."""
import math

import numpy as np
import pytest

import oracle
import test_oracle_describe as DS


def _atan2_sector(a, b):
    q = (8 * math.atan2(b, a) / (2 * math.pi)) % 8
    return int(math.floor(q)) % 8, abs(q - round(q))


def test_octant_edges_and_interiors():
    # a direction on an edge belongs to the sector it starts: 0, 45, ... 315 deg
    edges = [(1, 0, 0), (1, 1, 1), (0, 1, 2), (-1, 1, 3), (-1, 0, 4), (-1, -1, 5), (0, -1, 6), (1, -1, 7)]
    for a, b, k in edges:
        for sc in (1e-300, 1e-3, 1.0, 255.0, 1e300):
            assert oracle.octant(a * sc, b * sc) == k, (a, b, sc)
    # (k + 1/2) * 45 deg and directions just either side of every edge
    for k in range(8):
        th = math.radians(45 * k + 22.5)
        assert oracle.octant(math.cos(th), math.sin(th)) == k
        for d, want in ((1e-9, k), (-1e-9, (k - 1) % 8)):
            th = math.radians(45 * k) + d
            assert oracle.octant(math.cos(th), math.sin(th)) == want, (k, d)
    # -0 is a zero: (a, -0) with a > 0 points along 0 deg, (-0, b) with b > 0 along 90
    assert oracle.octant(1.0, -0.0) == 0 and oracle.octant(-0.0, 1.0) == 2


def test_octant_matches_atan2_sector_away_from_edges():
    rng = np.random.default_rng(3)
    ab = rng.standard_normal((20000, 2)) * rng.choice([1e-3, 1.0, 300.0], (20000, 1))
    n = 0
    for a, b in ab:
        k, gap = _atan2_sector(a, b)
        if gap > 1e-9:
            assert oracle.octant(a, b) == k, (a, b)
            n += 1
    assert n > 19900
    # every integer gradient of 8-bit differences: edges are exact integer
    # conditions, the rest lie far from any edge
    for a in range(-255, 256):
        for b in range(-255, 256):
            if a == 0 and b == 0:
                continue
            if b == 0 or a == 0 or a == b or a == -b:
                want = {(1, 0): 0, (1, 1): 1, (0, 1): 2, (-1, 1): 3, (-1, 0): 4, (-1, -1): 5, (0, -1): 6,
                        (1, -1): 7}[(int(np.sign(a)), int(np.sign(b)))]
            else:
                want, gap = _atan2_sector(a, b)
                assert gap > 1e-6
            assert oracle.octant(a, b) == want, (a, b)


def _single_bin(k):
    want = np.zeros(128)
    want[k::8] = 0.25
    return want


def test_describe_hard_ramp_closed_forms():
    # a linear image gives every sample the same gradient: one bin per cell,
    # equal in all 16 cells, so every entry of that bin is 1/4
    H = W = 64
    yy, xx = np.mgrid[0:H, 0:W]
    kp = DS._kp(H, W, 32, 31)
    ws = np.array([3], np.int32)
    for img, k in ((yy, 0), (xx, 2), (yy + 2 * xx, 1), (63 - yy, 4), (126 - 2 * yy + xx, 3)):
        d, v = oracle.describe(img.astype(np.uint8), kp, ws, None, hard=True)
        assert v[0] == 1 and np.abs(d[0] - _single_bin(k)).max() < 1e-12, k
    # the soft split differs on a direction inside a sector (63.4 deg)
    ds, _ = oracle.describe((yy + 2 * xx).astype(np.uint8), kp, ws, None)
    assert np.abs(ds[0] - _single_bin(1)).max() > 0.05
    # turned fixed-point grid (e_u = (cq, sq) / 2048, e_v = (-sq, cq) / 2048 in
    # (row, col)) on I = r and on I = r + 2c: bilinear sampling of a linear
    # image is exact, so every sample has the frame gradient
    # 2 (grad I . e_u, grad I . e_v)
    for k in (0, 7, 11, 20, 35):
        th = math.radians((k + 0.5) * 10)
        cq, sq = round(2048 * math.cos(th)), round(2048 * math.sin(th))
        for img, gr, gc in ((yy, 1, 0), (yy + 2 * xx, 1, 2)):
            sec, gap = _atan2_sector(gr * cq + gc * sq, -gr * sq + gc * cq)
            assert gap > 0.05
            d, _ = oracle.describe(img.astype(np.uint8), kp, ws, np.array([k], np.uint8), hard=True)
            assert np.abs(d[0] - _single_bin(sec)).max() < 1e-12, (k, gc)


def _hard_eq5(g, y, x, s):
    """Upright samples sit on pixels: integer Eq. 5 gradients, sectors from
    atan2 with the edges decided on the integers."""
    G = g.astype(np.int64)
    h = np.zeros(128)
    R = 2 * s
    for u in range(-R, R):
        for v in range(-R, R):
            a = G[y + u + 1, x + v] - G[y + u - 1, x + v]
            b = G[y + u, x + v + 1] - G[y + u, x + v - 1]
            if a == 0 and b == 0:
                continue
            if b == 0 or a == 0 or a == b or a == -b:
                k = {(1, 0): 0, (1, 1): 1, (0, 1): 2, (-1, 1): 3, (-1, 0): 4, (-1, -1): 5, (0, -1): 6,
                     (1, -1): 7}[(int(np.sign(a)), int(np.sign(b)))]
            else:
                k, _ = _atan2_sector(a, b)
            h[(((u + R) // s) * 4 + (v + R) // s) * 8 + k] += math.hypot(a, b)
    c = np.minimum(h / np.linalg.norm(h), 0.2)
    return c / np.linalg.norm(c)


def test_describe_hard_upright_equals_integer_eq5():
    rng = np.random.default_rng(19)
    H, W = 44, 48
    for levels, (y, x, s) in ((256, (21, 22, 3)), (9, (22, 23, 4)), (256, (20, 25, 2))):
        g = rng.integers(0, levels, size=(H, W)).astype(np.uint8)
        d, v = oracle.describe(g, DS._kp(H, W, y, x), np.array([s], np.int32), None, hard=True)
        assert v[0] == 1 and np.abs(d[0] - _hard_eq5(g, y, x, s)).max() < 1e-12, levels


def test_turn_table_is_rounded_2048_cos_sin():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for k in range(36):
        th = (k + mpmath.mpf(1) / 2) * 10 * mpmath.pi / 180
        cq, sq = oracle.turn_fx(k)
        for got, exact in ((cq, 2048 * mpmath.cos(th)), (sq, 2048 * mpmath.sin(th))):
            assert got == int(mpmath.nint(exact))
            assert abs(abs(exact - int(mpmath.floor(exact))) - 0.5) > 1e-6    # no rounding tie
        assert abs(math.hypot(cq, sq) / 2048 - 1) < 5e-4
    # bin k + 9 is bin k turned by 90 degrees, exactly
    for k in range(27):
        cq, sq = oracle.turn_fx(k)
        assert oracle.turn_fx(k + 9) == (-sq, cq)


def test_describe_hard_rotation_90_invariant():
    # Bin k + 9's fixed-point turn is bin k's turned by 90 degrees exactly, so
    # A and A rotated by 90 degrees read the same intensities at every sample
    # (clamped borders included) and give identical integer gradients.
    g, B, ia, ib, ws = DS._rot_setup(seed=8)
    oa = np.random.default_rng(3).integers(0, 27, len(ia)).astype(np.uint8)
    ob = (oa.astype(int) + 9).astype(np.uint8)
    da, va = oracle.describe(g, ia, ws, oa, hard=True)
    db, vb = oracle.describe(B, ib, ws, ob, hard=True)
    assert np.array_equal(va, vb)
    assert np.abs(da - db).max() < 1e-12
    # the hard rule is not the soft one on these points
    ds, _ = oracle.describe(g, ia, ws, oa)
    assert np.abs(ds - da).max() > 0.05


def test_soft_path_unchanged_through_describe_ex():
    rng = np.random.default_rng(23)
    g = rng.integers(0, 256, size=(70, 80)).astype(np.uint8)
    idx = (rng.integers(15, 55, 30) * 80 + rng.integers(15, 65, 30)).astype(np.uint32)
    ws = rng.integers(1, 4, 30).astype(np.int32)
    ori = oracle.orient(g, idx, ws)
    d0, v0 = oracle.describe(g, idx, ws, ori)
    d1, v1 = oracle.describe(g, idx, ws, ori, hard=False)
    dh, vh = oracle.describe(g, idx, ws, ori, hard=True)
    assert np.array_equal(d0, d1) and np.array_equal(v0, v1) and np.array_equal(v0, vh)
    assert np.allclose(np.linalg.norm(dh, axis=1), 1.0, atol=1e-12)
    # the two readings give different, but related, descriptors
    cos = (d0 * dh).sum(axis=1)
    assert cos.max() < 0.999 and cos.mean() > 0.7
