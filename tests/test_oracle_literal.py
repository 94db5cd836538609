"""Pins of the oracle's paper-literal variants: the finite-alpha ramp of Eq. 1,
border rejection, and the match rule of Sec. 2.4 without a ratio test."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2405_08578_gb300 import synth


def _ramp_brute(g, Ls, alpha):
    # Eq. 1 evaluated with NumPy: M_n = M + alpha * (raster index + 1); argmax
    # and argmin take the first (lowest raster index) of equal values
    H, W = g.shape
    r = np.arange(H * W, dtype=np.float64).reshape(H, W)
    v = g.astype(np.float64) + alpha * (r + 1.0)
    out = []
    for L in sorted(Ls):
        for wy in range(H // L):
            for wx in range(W // L):
                blk = v[wy * L:(wy + 1) * L, wx * L:(wx + 1) * L].ravel()
                ids = r[wy * L:(wy + 1) * L, wx * L:(wx + 1) * L].ravel().astype(np.int64)
                out += [ids[np.argmax(blk)], ids[np.argmin(blk)]]
    return np.array(out, np.uint32)


@pytest.mark.parametrize("alpha", [1e-6, 1e-3, 0.02, 0.5, 3.0])
def test_finite_alpha_ramp_is_eq1(alpha):
    rng = np.random.default_rng(int(alpha * 1e6) % 1000)
    for levels in (256, 4):
        g = rng.integers(0, levels, size=(37, 53)).astype(np.uint8)
        for Ls in ((4, 8), (5, 7, 12)):
            assert np.array_equal(oracle.detect(g, Ls, alpha), _ramp_brute(g, Ls, alpha))


def test_large_alpha_follows_the_ramp():
    # alpha * H * W far above the intensity range: the ramp decides, so every
    # window's maximum is its last pixel and its minimum its first
    g = np.random.default_rng(1).integers(0, 256, size=(32, 48)).astype(np.uint8)
    idx = oracle.detect(g, (8,), 1000.0)
    W = 48
    for w, (mx, mn) in enumerate(idx.reshape(-1, 2)):
        wy, wx = divmod(w, W // 8)
        assert mx == (wy * 8 + 7) * W + wx * 8 + 7 and mn == (wy * 8) * W + wx * 8


@pytest.mark.parametrize("upright", [False, True])
def test_border_rejection_keeps_exactly_clamp_free_points(upright):
    # a kept point reads no pixel outside the image: embedding the image in
    # random padding leaves its orientation and descriptor bit-identical
    p = synth.small_pair(150, 190, seed=3)
    g = p.A
    H, W = g.shape
    Ls = (8, 16, 32)
    idx = oracle.detect(g, Ls)
    _, ws = oracle.keypoint_scales(H, W, Ls)
    ori = None if upright else oracle.orient(g, idx, ws)
    desc, valid = oracle.describe(g, idx, ws, ori, border=True)
    _, valid_all = oracle.describe(g, idx, ws, ori)
    pad = 60
    big = np.random.default_rng(4).integers(0, 256, size=(H + 2 * pad, W + 2 * pad)).astype(np.uint8)
    big[pad:pad + H, pad:pad + W] = g
    y, x = idx // W, idx % W
    idx2 = ((y + pad) * (W + 2 * pad) + x + pad).astype(np.uint32)
    ori2 = None if upright else oracle.orient(big, idx2, ws)
    desc2, _ = oracle.describe(big, idx2, ws, ori2)
    keep = valid.astype(bool)
    assert keep.sum() > 50 and (~keep & valid_all.astype(bool)).sum() > 50
    assert not (valid.astype(bool) & ~valid_all.astype(bool)).any()
    if not upright:
        assert np.array_equal(ori[keep], ori2[keep])
    # upright samples sit on integer offsets: bit-identical; turned samples are
    # rounded at absolute coordinates, which the padding shifts (~1e-14)
    tol = 0.0 if upright else 1e-12
    assert np.abs(desc[keep] - desc2[keep]).max() <= tol
    # the rule is not vacuous: padding changes some rejected point's description
    rej = ~keep & valid_all.astype(bool)
    assert (np.abs(desc[rej] - desc2[rej]).max(axis=1) > 0).any()
    # the radius of each kept point fits, the closed form per scale
    P = np.ceil(2.0 * np.sqrt(2.0) * ws + 1.5).astype(int) + 1
    inside = (x >= P) & (y >= P) & (x + P <= W - 1) & (y + P <= H - 1)
    assert np.array_equal(keep, inside & valid_all.astype(bool))


def _brute_nn(dA, vA, dB, vB):
    d2 = ((dA[:, None, :] - dB[None, :, :]) ** 2).sum(-1)
    d2[:, ~vB.astype(bool)] = np.inf
    j = np.argmin(d2, axis=1)
    return j, np.sqrt(d2[np.arange(len(dA)), j])


def test_match_without_ratio_test_is_the_nearest_neighbour():
    rng = np.random.default_rng(9)
    dA = np.abs(rng.standard_normal((60, 128)))
    dB = np.abs(rng.standard_normal((80, 128)))
    dA /= np.linalg.norm(dA, axis=1, keepdims=True)
    dB /= np.linalg.norm(dB, axis=1, keepdims=True)
    vA = (rng.uniform(size=60) > 0.1).astype(np.uint8)
    vB = (rng.uniform(size=80) > 0.1).astype(np.uint8)
    j, d1 = _brute_nn(dA, vA, dB, vB)
    m, od1, _, _, _ = oracle.match(dA, vA, dB, vB, ratio=0.0)
    assert np.array_equal(m, np.where(vA.astype(bool), j, -1))
    assert np.allclose(od1[vA.astype(bool)], d1[vA.astype(bool)], rtol=0, atol=1e-12)
    ds = float(np.median(d1))
    m2, _, _, _, _ = oracle.match(dA, vA, dB, vB, ratio=0.0, delta_s=ds)
    assert np.array_equal(m2, np.where(vA.astype(bool) & (d1 < ds), j, -1))
    # one valid candidate: no second neighbour, still a match without the ratio test
    vB1 = np.zeros(80, np.uint8)
    vB1[17] = 1
    m3, _, _, _, _ = oracle.match(dA, vA, dB, vB1, ratio=0.0)
    assert np.array_equal(m3, np.where(vA.astype(bool), 17, -1))
    m4, _, _, _, _ = oracle.match(dA, vA, dB, vB1, ratio=0.8)
    assert (m4 == -1).all()
