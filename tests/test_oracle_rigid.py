"""Pins of the oracle's rigid model (Eq. 8: rotation theta and translation
t_x, t_y) against closed forms, an independent least-squares solver and
brute-force recounts."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle

RIGID = oracle.MODEL_RIGID


def _rigid(theta, tx, ty):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s, tx], [s, c, ty], [0.0, 0.0, 1.0]])


def _apply(H, p):
    q = np.c_[p, np.ones(len(p))] @ H.T
    return q[:, :2] / q[:, 2:]


def _case(rng, M, frac_in, theta, t, noise=0.3, size=1500.0):
    Ht = _rigid(theta, *t)
    pa = np.round(rng.uniform(0, size, (M, 2)))
    pb = _apply(Ht, pa) + noise * rng.standard_normal((M, 2))
    out = rng.uniform(size=M) > frac_in
    pb[out] = rng.uniform(0, size, (out.sum(), 2))
    return np.c_[pa, pb], Ht, ~out


@pytest.mark.parametrize("theta", [0.0, 0.3, -1.2, 2.9, -3.1, math.pi / 2])
def test_rigid_fit_recovers_exact_transform(theta):
    rng = np.random.default_rng(5)
    Ht = _rigid(theta, 312.5, -47.25)
    pa = rng.uniform(0, 2000, (50, 2))
    pts = np.c_[pa, _apply(Ht, pa)]
    H = oracle.rigid_fit(pts)
    assert np.abs(H[:2, :2] - Ht[:2, :2]).max() < 1e-12
    assert np.abs(H[:2, 2] - Ht[:2, 2]).max() < 1e-9
    assert np.array_equal(H[2], [0.0, 0.0, 1.0])


@pytest.mark.parametrize("theta", [0.05, -2.0, 3.05])
def test_rigid_fit_is_the_least_squares_minimiser(theta):
    # an independent numerical minimiser of sum |R p_A + t - p_B|^2
    opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(11)
    pa = rng.uniform(0, 1000, (80, 2))
    pb = _apply(_rigid(theta, 40.0, 90.0), pa) + 2.0 * rng.standard_normal((80, 2))
    H = oracle.rigid_fit(np.c_[pa, pb])

    def res(x):
        return (_apply(_rigid(*x), pa) - pb).ravel()

    th0 = math.atan2(H[1, 0], H[0, 0])
    x0 = np.array([th0 + 0.2, 0.0, 0.0])
    sol = opt.least_squares(res, x0, xtol=1e-15, ftol=1e-15, gtol=1e-15)
    d = (sol.x[0] - th0 + math.pi) % (2 * math.pi) - math.pi
    assert abs(d) < 1e-9
    assert np.abs(sol.x[1:] - H[:2, 2]).max() < 1e-6
    f = lambda x: float((res(x) ** 2).sum())  # noqa: E731
    best = f(np.r_[th0, H[:2, 2]])
    for dx in ([1e-4, 0, 0], [-1e-4, 0, 0], [0, 1e-3, 0], [0, 0, -1e-3]):
        assert f(np.r_[th0, H[:2, 2]] + np.array(dx)) > best


def test_rigid_fit_of_the_swapped_pairs_is_the_inverse():
    rng = np.random.default_rng(3)
    pa = rng.uniform(0, 800, (40, 2))
    pb = _apply(_rigid(0.7, -20.0, 15.0), pa) + rng.standard_normal((40, 2))
    H = oracle.rigid_fit(np.c_[pa, pb])
    Hi = oracle.rigid_fit(np.c_[pb, pa])
    assert np.abs(Hi @ H - np.eye(3)).max() < 1e-10


def test_two_point_fit_is_the_angle_between_the_difference_vectors():
    p = np.array([[100.0, 200.0], [400.0, 250.0]])
    q = np.array([[50.0, 60.0], [260.0, 330.0]])   # different length: no exact fit
    H = oracle.rigid_fit(np.c_[p, q])
    d, e = p[1] - p[0], q[1] - q[0]
    want = math.atan2(e[1], e[0]) - math.atan2(d[1], d[0])
    assert abs(math.atan2(H[1, 0], H[0, 0]) - want) < 1e-14
    # the midpoint of A maps onto the midpoint of B
    assert np.abs(_apply(H, p.mean(0)[None]) - q.mean(0)).max() < 1e-11
    # equal lengths: both points map exactly
    q2 = _apply(_rigid(-0.4, 7.0, 3.0), p)
    H2 = oracle.rigid_fit(np.c_[p, q2])
    assert np.abs(_apply(H2, p) - q2).max() < 1e-11


def test_rigid_fit_degenerate_sets():
    assert oracle.rigid_fit(np.array([[1.0, 2.0, 3.0, 4.0]])) is None
    assert oracle.rigid_fit(np.array([[5.0, 5.0, 1.0, 2.0], [5.0, 5.0, 8.0, 9.0]])) is None
    pts = np.array([[0.0, 0.0, 1.0, 1.0], [10.0, 0.0, 11.0, 1.0], [0.0, 10.0, 1.0, 11.0]])
    assert oracle.rigid_fit(pts, np.array([1, 0, 0], np.uint8)) is None
    assert oracle.rigid_fit(pts, np.array([1, 0, 1], np.uint8)) is not None


def test_two_index_draw_is_the_prefix_of_the_four_index_draw():
    for M in (2, 3, 7, 1000, 2**20):
        for t in range(200):
            s2 = oracle.ransac_sample(M, 99, 4, t, k=2)
            s4 = oracle.ransac_sample(M, 99, 4, t, k=4)
            assert s2 is not None and len(set(s2.tolist())) == 2
            if s4 is not None:
                assert np.array_equal(s2, s4[:2])


def test_rigid_ransac_hypotheses_counts_and_winner():
    rng = np.random.default_rng(21)
    pts, Ht, inl = _case(rng, 400, 0.45, 0.35, (120.0, -80.0))
    T = 300
    o = oracle.ransac(pts, T=T, seed=6, pair_id=2, want_all=True, model=RIGID)
    for t in range(T):
        s = oracle.ransac_sample(len(pts), 6, 2, t, k=2)
        p, q = pts[s, :2], pts[s, 2:]
        d, e = p[1] - p[0], q[1] - q[0]
        th = math.atan2(e[1], e[0]) - math.atan2(d[1], d[0])
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        tt = q.mean(0) - R @ p.mean(0)
        Hs = o["Hs"][t].reshape(3, 3)
        assert np.abs(Hs[:2, :2] - R).max() < 1e-12 and np.abs(Hs[:2, 2] - tt).max() < 1e-9
        e2 = ((_apply(Hs, pts[:, :2]) - pts[:, 2:]) ** 2).sum(1)
        assert o["counts"][t] == int((e2 < 9.0).sum())
    assert o["best_t"] == int(np.argmax(o["counts"]))
    assert np.abs(_apply(o["H"], pts[inl, :2]) - _apply(Ht, pts[inl, :2])).max() < 0.2
    assert o["inliers"][inl].mean() > 0.98 and o["inliers"][~inl].sum() <= 2


def test_rigid_data_gives_the_homography_models_inliers():
    # Eq. 8 is a special case of Eq. 7: on exact rigid data both models find
    # the same transform and inlier set
    rng = np.random.default_rng(2)
    pts, Ht, inl = _case(rng, 300, 0.5, -0.6, (300.0, 20.0), noise=0.0)
    r = oracle.ransac(pts, T=500, seed=1, model=RIGID)
    h = oracle.ransac(pts, T=500, seed=1)
    assert np.array_equal(r["inliers"].astype(bool), inl)
    assert np.array_equal(h["inliers"], r["inliers"])
    assert np.abs(r["H"] - Ht).max() < 1e-9
    assert np.abs(_apply(h["H"], pts[inl, :2]) - _apply(Ht, pts[inl, :2])).max() < 1e-6


def test_rigid_ransac_small_and_degenerate_inputs():
    assert oracle.ransac(np.zeros((1, 4)), T=10, model=RIGID)["best_t"] == -1
    # two matches: one sample, exact fit
    pts = np.array([[0.0, 0.0, 10.0, 5.0], [100.0, 0.0, 110.0, 5.0]])
    o = oracle.ransac(pts, T=5, model=RIGID)
    assert o["best_t"] == 0 and o["n_in"] == 2 and np.abs(o["H"] - _rigid(0, 10, 5)).max() < 1e-12
    # all A points on one spot: every sample is degenerate
    o = oracle.ransac(np.array([[3.0, 3.0, i, 2 * i] for i in range(6)]), T=20, model=RIGID)
    assert o["best_t"] == -1 and o["n_in"] == 0


def test_guided_stop_with_two_point_samples_is_the_standard_bound():
    for w_num, w_den in [(1, 2), (3, 10), (9, 10), (1, 7)]:
        w = w_num / w_den
        need = math.ceil(math.log(0.01) / math.log1p(-w ** 2))
        assert oracle.guided_stop(w_num, w_den, need, k=2) and not oracle.guided_stop(w_num, w_den, need - 1, k=2)
    assert oracle.guided_stop(4, 4, 1, k=2) and not oracle.guided_stop(0, 4, 10**6, k=2)


def test_rigid_prior_falls_back_to_uniform():
    rng = np.random.default_rng(8)
    pts, _, inl = _case(rng, 300, 0.5, 0.2, (10.0, 10.0))
    prior = np.where(inl, 0.0, 1.0).astype(np.float32)   # points only at outliers
    g = oracle.ransac_prior(pts, prior, Tg=6, T=200, seed=4, want_counts=True, model=RIGID)
    u = oracle.ransac(pts, T=200, seed=4, want_all=True, model=RIGID)
    assert g["iters"] == 206 and g["best_t"] == 6 + u["best_t"]
    assert np.array_equal(g["inliers"], u["inliers"]) and np.array_equal(g["H"], u["H"])
    assert np.array_equal(g["counts"][6:], u["counts"])


def test_rigid_prior_stops_on_a_good_prior():
    rng = np.random.default_rng(9)
    pts, Ht, inl = _case(rng, 300, 0.7, -0.9, (5.0, 60.0))
    prior = np.where(inl, 0.99, 0.001).astype(np.float32)
    g = oracle.ransac_prior(pts, prior, Tg=16, T=500, seed=3, model=RIGID)
    assert g["iters"] == 16 and 0 <= g["best_t"] < 16
    u = oracle.ransac(pts, T=500, seed=3, model=RIGID)
    assert np.array_equal(g["inliers"], u["inliers"])
