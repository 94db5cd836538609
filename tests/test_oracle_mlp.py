"""Pins for the oracle's learned-proposal functions (not in the paper):
features, the 8-64-64-1 network, its loss gradient, Adam, and guided sampling."""
import math

import numpy as np

import oracle


def test_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    P = rng.standard_normal(oracle.MLP_NPARAM) * 0.3
    x = rng.standard_normal((40, 8))
    y = (rng.uniform(size=40) < 0.4).astype(np.uint8)
    L, g = oracle.mlp_loss_grad(P, x, y)
    h = 1e-6
    fd = np.empty_like(g)
    for i in range(oracle.MLP_NPARAM):
        e = np.zeros_like(P)
        e[i] = h
        fd[i] = (oracle.mlp_loss_grad(P + e, x, y)[0] - oracle.mlp_loss_grad(P - e, x, y)[0]) / (2 * h)
    scale = np.abs(g).max()
    assert np.abs(fd - g).max() < 1e-6 * max(scale, 1e-3) + 1e-9


def test_closed_form_networks():
    # only b3 set: z = b3 everywhere, every other gradient vanishes
    P = np.zeros(oracle.MLP_NPARAM)
    P[4800] = 0.7
    x = np.random.default_rng(1).standard_normal((9, 8))
    y = np.array([1, 0, 1, 1, 0, 0, 1, 0, 1], np.uint8)
    z, p = oracle.mlp_forward(P, x)
    assert np.allclose(z, 0.7) and np.allclose(p, 1 / (1 + math.exp(-0.7)))
    L, g = oracle.mlp_loss_grad(P, x, y)
    want = np.mean([math.log1p(math.exp(-0.7)) if t else 0.7 + math.log1p(math.exp(-0.7)) for t in y])
    assert abs(L - want) < 1e-12
    assert abs(g[4800] - np.mean(1 / (1 + math.exp(-0.7)) - y)) < 1e-12
    assert np.abs(g[:4800]).max() == 0
    # one path: z = relu(relu(x0)) = max(x0, 0)
    P = np.zeros(oracle.MLP_NPARAM)
    W1, b1, W2, b2, w3, b3 = oracle.mlp_split(P)
    P[0] = 1.0            # W1[0][0]
    P[576] = 1.0          # W2[0][0]
    P[4736] = 1.0         # w3[0]
    x = np.linspace(-2, 2, 17)[:, None] * np.eye(8)[0][None, :]
    z, _ = oracle.mlp_forward(P, x)
    assert np.allclose(z, np.maximum(x[:, 0], 0))


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    oracle.mlp_adam(p, m, v, g, 1, lr=0.01)
    want = -0.01 * g / (np.abs(g) + 1e-8)          # m-hat = g, v-hat = g^2
    assert np.allclose(p, want, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_features_by_hand():
    pts = np.array([[10.0, 20, 300, 40], [639, 479, 0, 0]])
    f = oracle.mlp_features([0.2, 0.3], [0.5, 0.6], [16, 128], 128, [3, 35], [5, 0], pts, 640, 480, 640, 480)
    assert np.allclose(f[0], [0.4, 0.2, 4 / 7, 20 / 180, 10 / 640, 20 / 480, 300 / 640, 40 / 480])
    # 0 - 35 bins = -350 deg -> wraps to +10 deg
    assert np.allclose(f[1], [0.5, 0.3, 1.0, 10 / 180, 639 / 640, 479 / 480, 0, 0])
    # a half turn lands on the closed end of [-180, 180): -180 deg
    f = oracle.mlp_features([0.2], [0.5], [32], 128, [0], [18], pts[:1], 640, 480, 640, 480)
    assert np.allclose(f[0, :4], [0.4, 0.2, 5 / 7, -1.0])


def test_guided_weights_are_exact_integers():
    pr = np.array([0.0, 1.0, 0.5, 1e-3, 2e-3, np.float32("nan")], np.float32)
    pf = oracle.guided_weights(pr)
    q = np.diff(np.r_[0, pf.astype(np.int64)])
    assert q.tolist() == [66, 65536, 32768, 66, 131, 66]


def test_guided_draws_follow_weights():
    pr = np.array([0.9, 0.05, 0.5, 0.2, 0.7, 0.01, 0.3, 0.6], np.float32)
    pf = oracle.guided_weights(pr)
    q = np.diff(np.r_[0, pf.astype(np.int64)]).astype(np.float64)
    first = np.zeros(8)
    for t in range(6000):
        s = oracle.ransac_sample_guided(pf, 99, 4, t)
        assert s is not None and len(set(s.tolist())) == 4
        first[s[0]] += 1
    exp = 6000 * q / q.sum()
    chi2 = ((first - exp) ** 2 / exp).sum()
    assert chi2 < 30          # 7 dof


def _prior_case(frac_out, M=400, seed=5):
    rng = np.random.default_rng(seed)
    H = np.array([[1.02, 0.05, 30.0], [-0.04, 0.99, -12.0], [1e-5, -2e-5, 1.0]])
    pa = np.round(rng.uniform(0, 900, (M, 2)))
    q = np.c_[pa, np.ones(M)] @ H.T
    pb = q[:, :2] / q[:, 2:]
    out = rng.uniform(size=M) < frac_out
    pb[out] = rng.uniform(0, 900, (out.sum(), 2))
    return np.c_[pa, pb], out


def test_ransac_prior_finds_the_model_early():
    # 70% inliers: after 24 guided draws (1 - 0.7^4)^24 < 0.01 holds for the
    # plain fraction as well as for the prior-weighted one
    pts, out = _prior_case(0.3)
    prior = np.where(out, 0.0, 1.0).astype(np.float32)
    g = oracle.ransac_prior(pts, prior, Tg=24, T=200, seed=3, want_counts=True)
    u = oracle.ransac(pts, T=200, seed=3, want_all=True)
    assert g["n_in"] == u["n_in"] == (~out).sum()
    assert np.array_equal(g["inliers"], u["inliers"])
    assert g["iters"] == 24 and g["best_t"] <= u["best_t"]
    assert (g["counts"][24:] == -1).all()


def test_guided_stop_is_the_standard_bound():
    # T(w) = ceil(log(0.01) / log(1 - w^4)); w = 1/2 -> 71.36 -> 72
    assert oracle.guided_stop(1, 2, 72) and not oracle.guided_stop(1, 2, 71)
    for w_num, w_den in [(3, 10), (9, 10), (1, 7), (999, 1000)]:
        w = w_num / w_den
        need = math.ceil(math.log(0.01) / math.log1p(-w ** 4))
        assert oracle.guided_stop(w_num, w_den, need) and not oracle.guided_stop(w_num, w_den, need - 1)
    assert oracle.guided_stop(5, 5, 1)          # every draw an inlier
    assert not oracle.guided_stop(0, 5, 10**6)  # no inlier weight
    assert not oracle.guided_stop(0, 0, 10)


def test_ransac_prior_support_floor():
    # the prior puts nearly all its mass on a model's exact inliers, so the
    # prior-weighted bound holds; the search still ends on the guided winner
    # only when it has min_support inliers and its plain inlier fraction
    # (inliers / M) passes the same bound
    rng = np.random.default_rng(11)
    H = np.array([[0.97, 0.08, 40.0], [-0.06, 1.03, -25.0], [2e-5, 1e-5, 1.0]])

    def case(n_in, M):
        pa = np.round(rng.uniform(0, 900, (M, 2)))
        q = np.c_[pa, np.ones(M)] @ H.T
        pb = rng.uniform(0, 900, (M, 2))
        pb[:n_in] = q[:n_in, :2] / q[:n_in, 2:]
        prior = np.full(M, 1e-3, np.float32)
        prior[:n_in] = 0.99
        return np.c_[pa, pb], prior

    pts, prior = case(10, 12)                      # plain fraction 10/12
    u = oracle.ransac(pts, T=300, seed=6)
    g = oracle.ransac_prior(pts, prior, Tg=32, T=300, seed=6, min_support=12)
    assert g["iters"] == 332 and g["best_t"] == 32 + u["best_t"]          # 10 < 12: uniform RANSAC's result
    assert g["n_in"] == u["n_in"] and np.array_equal(g["inliers"], u["inliers"])
    g = oracle.ransac_prior(pts, prior, Tg=32, T=300, seed=6, min_support=8)
    assert g["iters"] == 32 and g["n_in"] == 10 and g["inliers"][:10].all()   # enough support: stopped
    pts, prior = case(5, 45)                       # plain fraction 5/45
    u = oracle.ransac(pts, T=300, seed=6)
    g = oracle.ransac_prior(pts, prior, Tg=32, T=300, seed=6, min_support=4)
    assert g["iters"] == 332 and g["n_in"] == u["n_in"] and np.array_equal(g["inliers"], u["inliers"])


def test_ransac_prior_falls_back_to_uniform():
    # a prior that points only at outliers never passes the stop test: the
    # result is uniform RANSAC's, iteration numbers offset by Tg
    pts, out = _prior_case(0.5, seed=8)
    prior = np.where(out, 1.0, 0.0).astype(np.float32)
    g = oracle.ransac_prior(pts, prior, Tg=8, T=300, seed=4, want_counts=True)
    u = oracle.ransac(pts, T=300, seed=4, want_all=True)
    assert g["iters"] == 308 and g["best_t"] == 8 + u["best_t"]
    assert g["n_in"] == u["n_in"] and np.array_equal(g["inliers"], u["inliers"])
    assert np.array_equal(g["H"], u["H"])
    assert np.array_equal(g["counts"][8:], u["counts"])
    # too few matches: no model, no stop
    g = oracle.ransac_prior(pts[:3], prior[:3], Tg=8, T=30)
    assert g["best_t"] == -1 and g["n_in"] == 0 and g["iters"] == 38
