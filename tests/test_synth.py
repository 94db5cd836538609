"""Properties of the seeded input generators: the uneven-size pairs have the
stated size and aspect ranges, are reproducible, and B is the scene seen
through H (A pixel -> B pixel)."""
import numpy as np

from paper_2405_08578_gb300 import synth


def _bilinear(img, x, y):
    x0, y0 = np.floor(x).astype(int), np.floor(y).astype(int)
    fx, fy = x - x0, y - y0
    a = img[y0, x0] * (1 - fx) + img[y0, x0 + 1] * fx
    b = img[y0 + 1, x0] * (1 - fx) + img[y0 + 1, x0 + 1] * fx
    return a * (1 - fy) + b * fy


def test_uneven_pairs_sizes_and_reproducibility():
    ps = synth.uneven_pairs(6, seed=5, long_lo=200, long_hi=420)
    for p in ps:
        h, w = p.A.shape
        assert p.B.shape == p.A.shape and p.A.dtype == np.uint8
        assert 200 <= w <= 420
        assert 4.0 / 3.0 - 0.02 <= w / h <= 16.0 / 9.0 + 0.02
    again = synth.uneven_pairs(6, seed=5, long_lo=200, long_hi=420)
    assert all(np.array_equal(a.A, b.A) and np.array_equal(a.B, b.B) and np.array_equal(a.H, b.H)
               for a, b in zip(ps, again))
    assert len({p.A.shape for p in ps}) > 1


def test_uneven_pairs_b_is_a_through_h():
    for p in synth.uneven_pairs(3, seed=7, long_lo=300, long_hi=400):
        h, w = p.A.shape
        A = p.A.astype(np.float64)
        ys, xs = np.mgrid[4:h - 4:7, 4:w - 4:7]
        xb, yb = xs.ravel().astype(np.float64), ys.ravel().astype(np.float64)
        v = np.linalg.inv(p.H) @ np.vstack([xb, yb, np.ones_like(xb)])
        xa, ya = v[0] / v[2], v[1] / v[2]
        ok = (xa >= 1) & (xa < w - 2) & (ya >= 1) & (ya < h - 2)
        assert ok.sum() > 200
        # B rounds the scene sampled at H^-1 x; A rounds the scene on the grid:
        # they agree to within the two roundings and the scene's curvature
        err = np.abs(p.B[yb[ok].astype(int), xb[ok].astype(int)] - _bilinear(A, xa[ok], ya[ok]))
        assert np.median(err) <= 0.5 and err.max() <= 2.0
