"""Pins for the oracle's Sec. 2.4 matching and Sec. 2.5 RANSAC / Eq. 7 homography."""
import numpy as np
import pytest

import oracle
from conftest import golden_rows


def _unit(rng, n):
    d = np.abs(rng.standard_normal((n, 128)))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_match_vs_numpy_bruteforce():
    rng = np.random.default_rng(0)
    A = _unit(rng, 150)
    B = _unit(rng, 170)
    B[:60] = A[:60] + 0.02 * rng.standard_normal((60, 128))   # some true matches
    vA = np.ones(150, np.uint8)
    vB = np.ones(170, np.uint8)
    vA[5] = 0
    vB[7] = 0
    m, d1, d2, j1, j2 = oracle.match(A, vA, B, vB, 0.8)
    D = ((A[:, None, :] - B[None, :, :]) ** 2).sum(-1)
    D[:, vB == 0] = np.inf
    order = np.argsort(D, axis=1, kind="stable")
    for i in range(150):
        if not vA[i]:
            assert m[i] == -1
            continue
        a, b = order[i, 0], order[i, 1]
        assert j1[i] == a and j2[i] == b
        assert abs(d1[i] - np.sqrt(D[i, a])) < 1e-12 and abs(d2[i] - np.sqrt(D[i, b])) < 1e-12
        assert m[i] == (a if D[i, a] < 0.64 * D[i, b] else -1)
    assert (m[:60] == np.arange(60)).sum() >= 55


def test_match_permutation_and_rows_subset():
    rng = np.random.default_rng(1)
    A = _unit(rng, 80)
    B = _unit(rng, 90)
    B[:30] = A[:30] + 0.01 * rng.standard_normal((30, 128))
    v = np.ones(90, np.uint8)
    m, *_ = oracle.match(A, np.ones(80, np.uint8), B, v)
    perm = rng.permutation(90)
    mp, *_ = oracle.match(A, np.ones(80, np.uint8), B[perm], v)
    inv = np.argsort(perm)
    assert np.array_equal(np.where(mp >= 0, perm[np.maximum(mp, 0)], -1), m)
    rows = np.array([3, 70, 0, 29])
    ms, *_ = oracle.match(A, np.ones(80, np.uint8), B, v, rows=rows)
    assert np.array_equal(ms, m[rows])
    del inv


def test_match_exact_tie_takes_the_lowest_index():
    # duplicated candidates are equally near: the lowest index is the nearest
    # neighbour (ratio test off), and the ratio test rejects the tie
    rng = np.random.default_rng(6)
    A = _unit(rng, 12)
    B = _unit(rng, 30)
    B[7] = A[4] + 0.02 * rng.standard_normal(128)
    B[19] = B[7]
    v = np.ones(30, np.uint8)
    m, d1, d2, j1, j2 = oracle.match(A, np.ones(12, np.uint8), B, v, ratio=0.0)
    assert m[4] == 7 and j1[4] == 7 and j2[4] == 19 and d1[4] == d2[4]
    m, *_ = oracle.match(A, np.ones(12, np.uint8), B, v, ratio=0.8)
    assert m[4] == -1


def test_match_delta_s_and_too_few_valid():
    rng = np.random.default_rng(2)
    A = _unit(rng, 10)
    B = A + 0.05 * rng.standard_normal((10, 128))
    ones = np.ones(10, np.uint8)
    m0, d1, *_ = oracle.match(A, ones, B, ones, 0.99)
    cut = float(np.median(d1))
    m, *_ = oracle.match(A, ones, B, ones, 0.99, delta_s=cut)
    assert np.all(m[d1 >= cut] == -1) and np.array_equal(m[d1 < cut], m0[d1 < cut])
    vb = np.zeros(10, np.uint8)
    vb[3] = 1
    m, *_ = oracle.match(A, ones, B, vb)
    assert np.all(m == -1)


def test_philox_known_answers():
    for row in golden_rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        assert oracle.philox4x32_10(v[0:4], v[4:6]).tolist() == v[6:10]


def test_ransac_sample_distinct_uniform():
    M = 37
    counts = np.zeros(M)
    for t in range(3000):
        s = oracle.ransac_sample(M, 1234, 5, t)
        assert s is not None and len(set(s.tolist())) == 4 and s.min() >= 0 and s.max() < M
        counts[s] += 1
    exp = counts.sum() / M
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 80          # 36 dof: mean 36, p(chi2 > 80) ~ 3e-5
    assert oracle.ransac_sample(3, 0, 0, 0) is None        # only 3 distinct values exist


def _proj(H, p):
    q = np.c_[p, np.ones(len(p))] @ H.T
    return q[:, :2] / q[:, 2:]


def _rand_H(rng):
    H = np.eye(3)
    H[:2, :2] += 0.1 * rng.standard_normal((2, 2))
    H[:2, 2] = rng.uniform(-200, 200, 2)
    H[2, :2] = rng.uniform(-2e-4, 2e-4, 2)
    return H


def test_dlt4_exact_and_square_to_quad():
    rng = np.random.default_rng(3)
    for _ in range(20):
        H = _rand_H(rng)
        src = rng.uniform(0, 1000, (4, 2))
        Hd = oracle.dlt4(src, _proj(H, src))
        assert np.abs(Hd / Hd[2, 2] - H / H[2, 2]).max() < 1e-9 * np.abs(H).max()
    # closed-form projective map of the unit square onto a quadrilateral
    # (Heckbert 1989): x = (a x + b y + c)/(g x + h y + 1), ...
    q = np.array([[10.0, 20.0], [210.0, 35.0], [190.0, 260.0], [5.0, 230.0]])
    (x0, y0), (x1, y1), (x2, y2), (x3, y3) = q
    sx, sy = x0 - x1 + x2 - x3, y0 - y1 + y2 - y3
    dx1, dx2, dy1, dy2 = x1 - x2, x3 - x2, y1 - y2, y3 - y2
    den = dx1 * dy2 - dx2 * dy1
    g = (sx * dy2 - dx2 * sy) / den
    h = (dx1 * sy - sx * dy1) / den
    Hc = np.array([[x1 - x0 + g * x1, x3 - x0 + h * x3, x0],
                   [y1 - y0 + g * y1, y3 - y0 + h * y3, y0],
                   [g, h, 1.0]])
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    Hd = oracle.dlt4(sq, q)
    assert np.abs(Hd - Hc).max() < 1e-9 * np.abs(Hc).max()
    # collinear target -> singular
    assert oracle.dlt4(sq, np.array([[0.0, 0], [1, 1], [2, 2], [3, 3]])) is None


def _hartley_np(p):
    c = p.mean(0)
    s = np.sqrt(2) / np.linalg.norm(p - c, axis=1).mean()
    return np.array([[s, 0, -s * c[0]], [0, s, -s * c[1]], [0, 0, 1]])


def test_refit_equals_numpy_svd():
    rng = np.random.default_rng(4)
    H = _rand_H(rng)
    pa = rng.uniform(0, 800, (60, 2))
    pb = _proj(H, pa) + 0.5 * rng.standard_normal((60, 2))
    pts = np.c_[pa, pb]
    mask = (rng.uniform(size=60) < 0.8).astype(np.uint8)
    Ho = oracle.refit(pts, mask)
    a, b = pa[mask == 1], pb[mask == 1]
    Ta, Tb = _hartley_np(a), _hartley_np(b)
    an = (np.c_[a, np.ones(len(a))] @ Ta.T)[:, :2]
    bn = (np.c_[b, np.ones(len(b))] @ Tb.T)[:, :2]
    rows = []
    for (x, y), (u, v) in zip(an, bn):
        rows.append([-x, -y, -1, 0, 0, 0, x * u, y * u, u])
        rows.append([0, 0, 0, -x, -y, -1, x * v, y * v, v])
    _, _, Vt = np.linalg.svd(np.array(rows))
    Hn = Vt[-1].reshape(3, 3)
    Hs = np.linalg.inv(Tb) @ Hn @ Ta
    Hs /= Hs[2, 2]
    assert np.abs(Ho - Hs).max() < 1e-8 * np.abs(Hs).max()


def test_eig_sym_vs_numpy():
    rng = np.random.default_rng(5)
    for n in (3, 9):
        X = rng.standard_normal((n + 4, n))
        A = X.T @ X
        ev, V = oracle.eig_sym(A)
        evn = np.linalg.eigvalsh(A)
        assert np.allclose(ev, evn, rtol=1e-10, atol=1e-12)
        assert np.allclose(A @ V, V * ev, atol=1e-9)


def test_score_counts_and_w_nonpositive():
    H = np.array([[1.0, 0, 5], [0, 1, 0], [0.01, 0, 1]])
    pts = np.array([[0.0, 0, 5, 0], [0, 0, 9, 0], [-150, 0, 0, 0], [10, 0, 15 / 1.1, 0]])
    n, m = oracle.score(H, pts, 3.0)
    assert m.tolist() == [1, 0, 0, 1] and n == 2       # x = -150 gives w = -0.5 -> outlier
    # an error of exactly the threshold is not an inlier (e < thresh)
    n, m = oracle.score(H, np.array([[0.0, 0, 8, 0], [0, 0, 7.999, 0]]), 3.0)
    assert m.tolist() == [0, 1] and n == 1
    # x = -200 gives w = -1 and projects exactly onto (195, 0): still not an inlier
    n, m = oracle.score(H, np.array([[-200.0, 0, 195, 0]]), 3.0)
    assert m.tolist() == [0] and n == 0


def test_ransac_recovers_known_h_with_outliers():
    rng = np.random.default_rng(6)
    H = _rand_H(rng)
    n_in, n_out = 200, 200
    pa = rng.uniform(0, 1000, (n_in + n_out, 2))
    pb = _proj(H, pa)
    pb[:n_in] += 0.3 * rng.standard_normal((n_in, 2))
    pb[n_in:] = rng.uniform(0, 1000, (n_out, 2))
    perm = rng.permutation(n_in + n_out)
    pts = np.c_[pa, pb][perm]
    r = oracle.ransac(pts, T=1000, thresh=3.0, seed=7, pair_id=1)
    corners = np.array([[0.0, 0], [1000, 0], [1000, 1000], [0, 1000]])
    assert np.abs(_proj(r["H"], corners) - _proj(H, corners)).max() < 0.5
    truth = perm < n_in
    assert (r["inliers"].astype(bool) & truth).sum() >= n_in - 3
    assert (r["inliers"].astype(bool) & ~truth).sum() <= 3
    # noise-free: the refit is exact
    pb0 = _proj(H, pa)
    pts0 = np.c_[pa, np.where((np.arange(len(pa)) < n_in)[:, None], pb0, pb)][perm]
    r0 = oracle.ransac(pts0, T=300, seed=1)
    assert np.abs(r0["H"] - H / H[2, 2]).max() < 1e-9 * np.abs(H).max()


def test_ransac_degenerate_inputs():
    r = oracle.ransac(np.zeros((3, 4)), T=10)
    assert r["n_in"] == 0 and r["best_t"] == -1 and not r["H"].any()
    line = np.array([[i, 2.0 * i, i + 1.0, 2.0 * i] for i in range(10)])
    r = oracle.ransac(line, T=50)
    assert r["n_in"] == 0 and r["best_t"] == -1


def test_ransac_best_is_earliest_max():
    rng = np.random.default_rng(8)
    H = _rand_H(rng)
    pa = rng.uniform(0, 500, (40, 2))
    pts = np.c_[pa, _proj(H, pa)]
    pts[30:, 2:] = rng.uniform(0, 500, (10, 2))
    r = oracle.ransac(pts, T=200, seed=3, want_all=True)
    c = r["counts"]
    assert r["best_t"] == int(np.argmax(c)) and c[r["best_t"]] == c.max()
