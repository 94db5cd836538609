"""Eq. 8 rigid model (rotation + translation) on the GPU against the oracle:
RANSAC stage parity, per-hypothesis counts, the guided proposal and a whole
pair through the C ABI."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2405_08578_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2405_08578_gb300 import lp  # noqa: E402
import gpu_util as G  # noqa: E402

RIGID = lp.MODEL_RIGID


def _rigid_pts(rng, M, frac_in, noise=0.4, size=1500.0):
    th = rng.uniform(-math.pi, math.pi)
    Ht = np.array([[math.cos(th), -math.sin(th), rng.uniform(-300, 300)],
                   [math.sin(th), math.cos(th), rng.uniform(-300, 300)], [0.0, 0.0, 1.0]])
    pa = np.round(rng.uniform(0, size, (M, 2)))
    pb = G.proj(Ht, pa) + noise * rng.standard_normal((M, 2))
    out = rng.uniform(size=M) > frac_in
    pb[out] = rng.uniform(0, size, (out.sum(), 2))
    return np.c_[pa, np.round(pb)].astype(np.float32), Ht, out


def _check(g, o, pts, thresh=3.0):
    assert g["best_t"] == o["best_t"]
    if o["best_t"] < 0:
        assert g["n_in"] == 0 and not g["H"].any()
        return
    p64 = pts.astype(np.float64)
    e = np.sqrt(((G.proj(o["H"], p64[:, :2]) - p64[:, 2:]) ** 2).sum(1))
    border = np.abs(e - thresh) <= 1e-4
    assert np.array_equal(g["inliers"][~border], o["inliers"][~border])
    assert abs(g["n_in"] - o["n_in"]) <= border.sum()
    # rigid form: a rotation block, no projective row
    assert np.array_equal(g["H"][2], [0.0, 0.0, 1.0])
    assert np.abs(g["H"][:2, :2] - o["H"][:2, :2]).max() < 1e-9
    assert np.abs(g["H"][:2, 2] - o["H"][:2, 2]).max() < 1e-6


@pytest.mark.parametrize("M,frac", [(2, 1.0), (3, 0.7), (60, 0.5), (700, 0.3), (5000, 0.6), (20000, 0.15)])
def test_rigid_ransac_matches_oracle(M, frac):
    rng = np.random.default_rng(100 + M)
    pts, _, _ = _rigid_pts(rng, M, frac)
    T = 500
    ctx = lp.Context(Ls=(16,), ransac_iters=T, seed=13, model=RIGID)
    g = G.ransac(ctx, pts, pair_id=5)
    counts = np.array(ctx.lp_diag_last_ransac_counts(T))
    o = oracle.ransac(pts.astype(np.float64), T=T, seed=13, pair_id=5, want_all=True, model=oracle.MODEL_RIGID)
    _check(g, o, pts)
    # the same samples are degenerate, and no certain count exceeds the exact one
    assert np.array_equal(counts < 0, o["counts"] < 0)
    ok = o["counts"] >= 0
    assert (counts[ok] <= o["counts"][ok]).all()
    if o["best_t"] >= 0:
        assert counts[o["best_t"]] == o["counts"][o["best_t"]]


def test_rigid_ransac_recovers_the_transform():
    rng = np.random.default_rng(7)
    pts, Ht, out = _rigid_pts(rng, 3000, 0.25, noise=0.3)
    ctx = lp.Context(Ls=(16,), ransac_iters=1000, seed=2, model=RIGID)
    g = G.ransac(ctx, pts)
    q = pts[~out, :2].astype(np.float64)
    assert np.abs(G.proj(g["H"], q) - G.proj(Ht, q)).max() < 0.3
    assert g["inliers"][~out].mean() > 0.97


def test_rigid_ransac_degenerate():
    ctx = lp.Context(Ls=(16,), ransac_iters=50, model=RIGID)
    assert G.ransac(ctx, np.zeros((1, 4), np.float32))["best_t"] == -1
    assert G.ransac(ctx, np.zeros((0, 4), np.float32))["best_t"] == -1
    same = np.array([[3.0, 3.0, i, 2.0 * i] for i in range(8)], np.float32)   # all A points on one spot
    r = G.ransac(ctx, same)
    assert r["best_t"] == -1 and r["n_in"] == 0 and not r["H"].any()


def test_unknown_model_is_rejected():
    with pytest.raises(lp.LpError):
        lp.Context(Ls=(16,), model=2)


def _gpu_prior(ctx, pts, prior, Tg, pair_id):
    M = len(pts)
    p = G.dev(pts)
    pr = G.dev(prior.astype(np.float32))
    dM = G.dev(np.array([M], np.int32))
    H = torch.zeros(9, dtype=torch.float64, device="cuda")
    inl = torch.zeros(M, dtype=torch.uint8, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    bt = torch.zeros(1, dtype=torch.int32, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.lp_ransac_prior(p, M, dM, pr, Tg, pair_id, H, inl, n, bt, it)
    return dict(H=G.host(H).reshape(3, 3), inliers=G.host(inl)[:M], n_in=int(G.host(n)[0]),
                best_t=int(G.host(bt)[0]), iters=int(G.host(it)[0]))


@pytest.mark.parametrize("kind,Tg", [("labels", 8), ("inverted", 8), ("noisy", 32)])
def test_rigid_prior_matches_oracle(kind, Tg):
    rng = np.random.default_rng(55 + Tg)
    pts, _, out = _rigid_pts(rng, 1200, 0.35)
    if kind == "labels":
        prior = np.where(out, 0.0, 1.0)
    elif kind == "inverted":
        prior = np.where(out, 1.0, 0.0)
    else:
        prior = np.clip(np.where(out, 0.3, 0.7) + 0.25 * rng.standard_normal(len(pts)), 0, 1)
    prior = prior.astype(np.float32)
    T = 300
    ctx = lp.Context(Ls=(16,), ransac_iters=T, seed=8, model=RIGID)
    g = _gpu_prior(ctx, pts, prior, Tg, pair_id=1)
    o = oracle.ransac_prior(pts.astype(np.float64), prior, Tg=Tg, T=T, seed=8, pair_id=1, model=oracle.MODEL_RIGID)
    assert g["iters"] == o["iters"]
    _check(g, o, pts)


def test_rigid_pair_640x480_vs_oracle_and_truth():
    h, w = 480, 640
    Ht = synth.similarity(6.0, 1.0, 200.0, 15.0, w / 2.0, h / 2.0)
    p = synth.make_pair(h, w, Ht, seed=4)
    Ls = synth.PAIR_640x480_LS
    ctx = lp.Context(Ls=Ls, model=RIGID)
    Hg, n_in, M = G.stitch(ctx, p.A, p.B)
    o = oracle.stitch_pair(p.A, p.B, Ls, model=oracle.MODEL_RIGID)
    ys, xs = np.mgrid[0:h:40, 0:w:40]
    q = np.c_[xs.ravel(), ys.ravel()].astype(np.float64)
    pb = G.proj(Ht, q)
    q = q[(pb[:, 0] >= 0) & (pb[:, 0] < w) & (pb[:, 1] >= 0) & (pb[:, 1] < h)]
    assert n_in >= 50 and len(q) > 50
    assert np.abs(G.proj(Hg, q) - G.proj(Ht, q)).max() < 1.0
    assert np.abs(G.proj(Hg, q) - G.proj(o["H"], q)).max() < 0.5
    assert abs(n_in - o["n_in"]) <= max(2, 0.01 * o["n_in"])
    assert np.array_equal(Hg[2], [0.0, 0.0, 1.0])
    th = math.degrees(math.atan2(Hg[1, 0], Hg[0, 0]))
    assert abs(th - 6.0) < 0.1
