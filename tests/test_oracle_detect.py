"""Pins for the oracle's Sec. 2.1-2.2 functions (intensity, Eq. 1-2 peaks, Eq. 3-4 sizes).

Each check is independent of the oracle's own formulation: exact rational
arithmetic, a brute force written another way, closed forms, or invariants.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from conftest import golden_rows


def test_gray_exact_rational():
    rng = np.random.default_rng(1)
    rgb = rng.integers(0, 256, size=(64, 80, 3)).astype(np.uint8)
    g = oracle.gray(rgb)
    for y in range(0, 64, 3):
        for x in range(0, 80, 5):
            r, gg, b = (int(v) for v in rgb[y, x])
            v = Fraction(299, 1000) * r + Fraction(587, 1000) * gg + Fraction(114, 1000) * b
            # round half up of the exact weighted sum
            want = int(v + Fraction(1, 2))
            assert g[y, x] == want


def test_gray_axis_and_extremes():
    v = np.arange(256, dtype=np.uint8)
    rgb = np.stack([v, v, v], axis=-1).reshape(16, 16, 3)
    assert np.array_equal(oracle.gray(rgb).reshape(-1), v)          # weights sum to 1
    pure = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255]]], np.uint8)
    assert oracle.gray(pure).tolist() == [[76, 150, 29]]             # 76.245, 149.685, 29.07


def brute_peaks(g, Ls):
    """Brute force with a different formulation: a 64-bit key g*2^32 + raster."""
    H, W = g.shape
    key = g.astype(np.int64) * (1 << 32) + np.arange(H * W, dtype=np.int64).reshape(H, W)
    out = []
    for L in sorted(Ls):
        for wy in range(H // L):
            for wx in range(W // L):
                blk = key[wy * L:(wy + 1) * L, wx * L:(wx + 1) * L]
                out.append(int(blk.max() & 0xFFFFFFFF))
                out.append(int(blk.min() & 0xFFFFFFFF))
    return np.array(out, np.uint32)


@pytest.mark.parametrize("shape,Ls,levels", [((16, 16), (2, 4, 8, 16), 256), ((13, 17), (3, 4), 4),
                                              ((40, 24), (8, 5, 12), 3), ((1, 9), (1 + 1,), 2)])
def test_detect_bruteforce(shape, Ls, levels):
    rng = np.random.default_rng(sum(shape) + len(Ls))
    for trial in range(5):
        g = rng.integers(0, levels, size=shape).astype(np.uint8)
        assert np.array_equal(oracle.detect(g, Ls), brute_peaks(g, Ls))


def test_detect_constant_image_ramp_tiebreak():
    # Eq. 1's ramp makes the last pixel of each window the max, the first the min.
    H, W, L = 48, 64, 16
    g = np.full((H, W), 77, np.uint8)
    idx = oracle.detect(g, (L,))
    k = 0
    for wy in range(H // L):
        for wx in range(W // L):
            assert idx[k] == (wy * L + L - 1) * W + wx * L + L - 1
            assert idx[k + 1] == (wy * L) * W + wx * L
            k += 2


def test_detect_literal_alpha_equals_limit():
    # For alpha*H*W < 1 the FP64 ramp only breaks ties, as the limit rule does.
    rng = np.random.default_rng(7)
    g = rng.integers(0, 8, size=(48, 56)).astype(np.uint8)
    Ls = (4, 8, 16)
    assert np.array_equal(oracle.detect(g, Ls, alpha=1e-9), oracle.detect(g, Ls))


def test_detect_scale_consistency_2x():
    # A 2x pixel-replicated image with window 2L has its peaks at 2p+(1,1) (max)
    # and 2p (min) of the original peaks p found with window L.
    rng = np.random.default_rng(11)
    g = rng.integers(0, 5, size=(24, 40)).astype(np.uint8)
    g2 = np.kron(g, np.ones((2, 2), np.uint8))
    for L in (2, 4, 8):
        a = oracle.detect(g, (L,)).astype(np.int64)
        b = oracle.detect(g2, (2 * L,)).astype(np.int64)
        W, W2 = g.shape[1], g2.shape[1]
        ya, xa = a // W, a % W
        yb, xb = b // W2, b % W2
        assert np.array_equal(yb[0::2], 2 * ya[0::2] + 1) and np.array_equal(xb[0::2], 2 * xa[0::2] + 1)
        assert np.array_equal(yb[1::2], 2 * ya[1::2]) and np.array_equal(xb[1::2], 2 * xa[1::2])


def test_num_keypoints_closed_form():
    assert oracle.num_keypoints(480, 640, (8, 16, 32)) == 12600
    assert oracle.num_keypoints(1600, 2688, (16, 32, 64, 128)) == 44604
    assert oracle.num_keypoints(7, 7, (8,)) == 0


def test_table2_counts_under_full_window_bound():
    # Table 2's LP-SIFT point counts never exceed the Eq. 2 full-window count.
    for name, nr, nc, l1, l2, c1, c2 in golden_rows("table2_counts.txt"):
        bound = oracle.num_keypoints(int(nr), int(nc), (int(l1), int(l2)))
        assert int(c1) <= bound and int(c2) <= bound, name


def test_region_ws_closed_form():
    for Ls, ws in golden_rows("region_ws.txt"):
        Ls = [int(v) for v in Ls.split(",")]
        ws = [int(v) for v in ws.split(",")]
        assert oracle.region_ws(Ls).tolist() == ws
        # Eq. 4's purpose: the described region w = d*w_s never exceeds L by
        # more than the rounding of w_s
        for L, w in zip(Ls, ws):
            assert 4 * w <= L + 2


def test_detect_invariant_under_strictly_increasing_intensity_maps():
    # Eq. 1-2 peaks (alpha -> 0+) depend on the order of the intensities and on
    # raster position only, so a strictly increasing map keeps every peak; a map
    # that merges two levels creates new ties and moves some peaks
    rng = np.random.default_rng(13)
    g = rng.integers(0, 128, size=(45, 70)).astype(np.uint8)
    lut = np.concatenate([[0], np.cumsum(rng.integers(1, 3, 127))]).astype(np.uint8)
    assert (np.diff(lut.astype(int)) > 0).all()
    for Ls in ((4, 8), (5, 7, 12), (3,)):
        assert np.array_equal(oracle.detect(lut[g], Ls), oracle.detect(g, Ls))
    merged = (g // 2).astype(np.uint8)
    assert not np.array_equal(oracle.detect(merged, (4, 8)), oracle.detect(g, (4, 8)))
