"""Host checks of the exactness claims the kernels' integer and rounding
shortcuts rest on.  Each test restates a claim from a kernel comment in exact
integer or rational arithmetic and checks it over the whole range the kernel
uses; none of them runs GPU code.
"""
import zlib
from fractions import Fraction

import numpy as np
import pytest

# 299 R + 587 G + 114 B + 500 over all 8-bit triples spans [500, 255,500]
S_MAX = 299 * 255 + 587 * 255 + 114 * 255 + 500


def _all_weighted_sums():
    r = np.arange(256, dtype=np.int64)
    s = (299 * r[:, None, None] + 587 * r[None, :, None] + 114 * r[None, None, :] + 500).ravel()
    return np.unique(s)


def test_intensity_division_by_1000_on_the_fp32_pipe():
    # fma_rz(s, 0.001f, 2^23) = 2^23 + floor(s * 0.001f) in [2^23, 2^24), where
    # the float spacing is 1; the claim is floor(s * 0.001f) = floor(s / 1000)
    c = Fraction(float(np.float32(0.001)))
    num, den = c.numerator, c.denominator
    assert 0 < c - Fraction(1, 1000) < Fraction(48, 10 ** 12)
    s = np.arange(0, S_MAX + 1, dtype=object)
    got = (s * num) // den
    assert (got == s // 1000).all()
    # and the sum 2^23 + s * 0.001f stays below 2^24, so the spacing is 1
    assert (1 << 23) + S_MAX // 1000 + 1 < (1 << 24)
    # 2^23 + s is exact as a float for every weighted sum
    sums = _all_weighted_sums()
    assert sums.min() == 500 and sums.max() == S_MAX
    assert np.array_equal(np.float32(np.float32(1 << 23) + sums.astype(np.float32)).astype(np.int64) - (1 << 23), sums)


def test_intensity_division_by_1000_by_high_multiply():
    # the other detect kernels: the high word of s * ceil(2^32 / 1000)
    C = -(-(1 << 32) // 1000)
    assert C == 4294968
    s = np.arange(0, S_MAX + 1, dtype=np.uint64)
    assert np.array_equal((s * np.uint64(C)) >> np.uint64(32), s // np.uint64(1000))


def test_lane_walk_start_from_a_float_quotient():
    # Walk2D: r = (int)((lane + 1/2) * rcp(n)), dr = (int)(32.5 * rcp(n)) for
    # n <= 127.  The exact quotient lies at least 1/(2n) from an integer; the
    # approximate reciprocal (2 ulp) and the rounded product move it by less
    # than 4 * 2^-24 of its value, far less.
    for n in range(1, 128):
        for x2 in list(range(1, 64, 2)) + [65]:   # 2 * (lane + 1/2) for lane 0..31, and 2 * 32.5
            q = Fraction(x2, 2 * n)
            gap = min(q - int(q), int(q) + 1 - q)
            assert gap >= Fraction(1, 2 * n)
            assert q * Fraction(4, 1 << 24) < gap
            assert int(q) == (x2 // 2) // n


def _argmax_lowest(v):
    best = 0
    for b in range(1, 36):
        if v[b] > v[best]:
            best = b
    return best


def _argmax_by_key(v):
    # the orientation argmax of the describe kernels: key = (v << 6) | (63 - bin),
    # lane l holds bins l and l + 32 (l < 4); maximum of the high words, then of
    # the low words among the lanes holding the top high word
    keys = [(int(v[b]) << 6) | (63 - b) for b in range(36)]
    lane_key = [max(keys[l], keys[l + 32]) if l < 4 else keys[l] for l in range(32)]
    hi = [k >> 32 for k in lane_key]
    lo = [k & 0xFFFFFFFF for k in lane_key]
    top = max(hi)
    low = max(lo[l] if hi[l] == top else 0 for l in range(32))
    assert low != 0
    return 63 - (low & 63)


@pytest.mark.parametrize("case", ["random", "ties", "high_word_ties", "zeros", "maximal"])
def test_orientation_argmax_by_two_word_reduction(case):
    rng = np.random.default_rng(zlib.crc32(case.encode()))
    vmax = 3721 * ((1 << 25) - 1)      # 61^2 samples of weight < 2^25: v < 2^37
    assert vmax < (1 << 37)
    for _ in range(400):
        if case == "random":
            v = rng.integers(0, vmax, 36)
        elif case == "ties":
            v = rng.integers(0, 4, 36) * rng.integers(1, 1 << 30)
        elif case == "high_word_ties":
            # equal high words (bits 26.. of v), different low parts
            v = (rng.integers(0, 3, 36) << 26) + rng.integers(0, 1 << 26, 36)
        elif case == "zeros":
            v = np.zeros(36, np.int64)
            v[rng.integers(0, 36, rng.integers(0, 3))] = rng.integers(0, 2)
        else:
            v = np.full(36, vmax, np.int64)
            v[rng.integers(0, 36, 5)] = vmax - rng.integers(0, 2, 5)
        assert _argmax_by_key(v) == _argmax_lowest(v)


def test_pixel_row_and_column_from_a_float_quotient():
    # y = (int)(id / W) from an approximate float quotient, corrected by
    # integer steps: the estimate is within a few units, and the correction
    # makes it exact.  Checked with the quotient perturbed by 2 ulp either way.
    rng = np.random.default_rng(7)
    for W in (1, 2, 3, 7, 480, 640, 1600, 2688, 4096, 65535, 1 << 20, (1 << 24) - 1):
        H = max(1, (1 << 24) // W)
        ids = np.unique(np.concatenate([rng.integers(0, H * W, 2000), [0, H * W - 1, W - 1, W]]))
        ids = ids[ids < H * W]
        for pert in (-2, 0, 2):
            q = (ids.astype(np.float32) / np.float32(W)).astype(np.float32)
            for _ in range(abs(pert)):
                q = np.nextafter(q, np.float32(np.inf if pert > 0 else -np.inf))
            y = q.astype(np.int64)
            x = ids - y * W
            for _ in range(8):
                low, high = x < 0, x >= W
                y = np.where(low, y - 1, np.where(high, y + 1, y))
                x = np.where(low, x + W, np.where(high, x - W, x))
            assert np.array_equal(y, ids // W) and np.array_equal(x, ids % W), W
