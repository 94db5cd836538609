"""GPU parity of each stage against the FP64 oracle, through the C ABI.

Integer work (intensity, peaks, orientation bins, Philox, compaction) must be
bit-exact.  Descriptors: |gpu - oracle| <= 1e-4 per component.  Matching is
stage-isolated (both sides get the same FP32 descriptors): identical match[]
except stated near-ties, distances within 1e-5.  RANSAC is stage-isolated
(same matches, same Philox stream): identical winning iteration and inlier set
except points within 1e-4 px of the threshold; H agrees to well under 0.5 px.
"""
import numpy as np
import pytest

import oracle
from paper_2405_08578_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_08578_gb300 import lp  # noqa: E402
import gpu_util as G  # noqa: E402

DESC_TOL = 1e-4
NEAR_TIE = 1e-5


def ctx_for(Ls, **kw):
    return lp.Context(Ls=Ls, **kw)


# ------------------------------------------------------------------ diagnostics
def test_gray_exhaustive_rgb():
    v = np.arange(1 << 24, dtype=np.uint32)
    rgb = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8)
    out = torch.zeros(1 << 24, dtype=torch.uint8, device="cuda")
    lp.lp_diag_gray(G.dev(rgb), 1 << 24, out)
    want = oracle.gray(rgb.reshape(4096, 4096, 3)).reshape(-1)
    assert np.array_equal(G.host(out), want)


def test_orient_bins_and_weights_exhaustive():
    bins = torch.zeros(511 * 511, dtype=torch.int32, device="cuda")
    lp.lp_diag_orient_bins(bins)
    a, b = np.meshgrid(np.arange(-255, 256), np.arange(-255, 256), indexing="ij")
    want = np.array([oracle.orient_bin(int(x), int(y)) for x, y in zip(a.ravel(), b.ravel())], np.int32)
    assert np.array_equal(G.host(bins), want)
    w = torch.zeros(130051, dtype=torch.int32, device="cuda")
    lp.lp_diag_orient_weights(w)
    want = np.array([oracle.orient_weight(s) for s in range(130051)], np.uint32)
    assert np.array_equal(G.host(w).view(np.uint32), want)
    # the describe kernels add the zero gradient's entry without testing for it
    assert G.host(bins)[255 * 511 + 255] == 0 and G.host(w)[0] == 0


def test_philox_matches_oracle_stream():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    out = torch.zeros((4096, 4), dtype=torch.int32, device="cuda")
    for key in ((0, 0), (0xA4093822, 0x299F31D0), (12345, 678)):
        lp.lp_diag_philox(G.dev(ctr.view(np.int32)), 4096, key[0], key[1], out)
        got = G.host(out).view(np.uint32)
        for i in range(0, 4096, 97):
            assert got[i].tolist() == oracle.philox4x32_10(ctr[i], key).tolist()


# ------------------------------------------------------------------ detection
DETECT_CASES = [
    ((40, 56), (8, 16), 1), ((37, 61), (4, 8, 16), 1), ((100, 130), (16, 32), 3), ((96, 112), (5, 7), 1),
    ((33, 45), (2, 4, 8), 3), ((240, 320), (16, 32, 64, 128), 1), ((150, 300), (128, 256), 1),
    ((480, 640), (8, 16, 32), 1), ((12, 12), (16,), 1), ((31, 17), (16,), 3),
    ((200, 330), (32, 64), 3), ((130, 270), (48, 96), 1), ((97, 161), (16, 48), 3),
]


@pytest.mark.parametrize("shape,Ls,ch", DETECT_CASES)
def test_detect_bitexact(shape, Ls, ch):
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    for levels in (256, 3):
        img = rng.integers(0, levels, size=shape + ((3,) if ch == 3 else ())).astype(np.uint8)
        ctx = ctx_for(Ls)
        kp, g = G.detect(ctx, img)
        og = oracle.gray(img)
        assert np.array_equal(kp, oracle.detect(og, Ls))
        if ch == 3:
            assert np.array_equal(g, og)


def test_detect_2688x1600_rgb_full():
    pair = synth.pair_2688x1600(0)
    ctx = ctx_for(synth.PAIR_2688x1600_LS)
    for img in (pair.A, pair.B):
        kp, g = G.detect(ctx, img)
        og = oracle.gray(img)
        assert np.array_equal(g, og)
        assert len(kp) == 44604
        assert np.array_equal(kp, oracle.detect(og, synth.PAIR_2688x1600_LS))


def test_detect_rejects_bad_args():
    ctx = ctx_for((16,))
    buf = torch.zeros((32, 48), dtype=torch.uint8, device="cuda")
    kp = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(lp.LpError) as e:
        ctx.lp_detect(buf, 32, 40, 40, 1, kp)            # pitch not a multiple of 16
    assert e.value.code == 2
    with pytest.raises(lp.LpError) as e:
        ctx.lp_detect(buf, 32, 48, 48, 2, kp)            # channels
    assert e.value.code == 1
    with pytest.raises(lp.LpError) as e:
        ctx.lp_detect(buf, 32, 16, 48, 3, kp)            # RGB without gray output
    assert e.value.code == 1


# ------------------------------------------------------------------ description
def _describe_parity(gray, Ls, sample=None, upright=False):
    ctx = ctx_for(Ls, upright=upright)
    H, W = gray.shape
    kp = oracle.detect(gray, Ls)
    ori, desc, valid, d16 = G.describe(ctx, gray, kp, bf16=True)
    _, ws = oracle.keypoint_scales(H, W, Ls)
    sel = np.arange(len(kp)) if sample is None else sample
    o_ori = oracle.orient(gray, kp[sel], ws[sel])
    o_desc, o_valid = oracle.describe(gray, kp[sel], ws[sel], None if upright else o_ori)
    if upright:
        assert not ori[sel].any()
    else:
        assert np.array_equal(ori[sel], o_ori)
    assert np.array_equal(valid[sel], o_valid)
    err = np.abs(desc[sel] - o_desc).max() if len(sel) else 0.0
    assert err <= DESC_TOL, err
    # the bf16 copy is the FP32 descriptor rounded to nearest
    assert np.array_equal(d16, torch.tensor(desc).to(torch.bfloat16).float().numpy())
    return err


@pytest.mark.parametrize("shape,Ls", [((64, 80), (8, 16)), ((75, 93), (8, 16, 32)), ((120, 200), (16, 32, 64)),
                                      ((128, 160), (32, 40)), ((200, 300), (100, 128)),
                                      ((500, 700), (64, 160)), ((700, 900), (256, 512))])
def test_describe_small(shape, Ls):
    p = synth.small_pair(shape[0], shape[1], seed=shape[0] + shape[1])
    _describe_parity(p.A, Ls)
    _describe_parity(p.A, Ls, upright=True)


def test_describe_huge_scale_global_path():
    # w_s = 256 (L = 1024): each cell's grid exceeds the shared-memory budget of
    # the split path, so these points take the global-memory kernel
    p = synth.small_pair(2048, 2048, seed=9)
    _describe_parity(p.A, (1024,))
    _describe_parity(p.A, (1024,), upright=True)


def test_describe_640x480():
    p = synth.pair_640x480(0)
    _describe_parity(p.A, synth.PAIR_640x480_LS)


def test_describe_2688x1600_sampled():
    p = synth.pair_2688x1600(0)
    g = oracle.gray(p.A)
    Ls = synth.PAIR_2688x1600_LS
    K = oracle.num_keypoints(1600, 2688, Ls)
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([rng.choice(K, 1500, replace=False), np.arange(K - 300, K), np.arange(200)]))
    _describe_parity(g, Ls, sample=sample)


@pytest.mark.parametrize("shape,Ls", [((48, 64), (8, 16)), ((260, 300), (100, 128))])
def test_describe_flat_image_invalid(shape, Ls):
    ctx = ctx_for(Ls)
    g = np.full(shape, 100, np.uint8)
    kp = oracle.detect(g, Ls)
    ori, desc, valid = G.describe(ctx, g, kp)
    assert len(kp) and not valid.any() and not desc.any() and not ori.any()


# ------------------------------------------------------------------ matching
def _match_parity(ctx, dA, vA, dB, vB, rows=None):
    m, d1, d2 = G.match(ctx, dA, vA, dB, vB)
    r = np.arange(len(dA)) if rows is None else rows
    om, od1, od2, oj1, oj2 = oracle.match(dA.astype(np.float64), vA, dB.astype(np.float64), vB,
                                          ratio=float(np.float32(ctx.cfg.ratio)), rows=r)
    fin = np.isfinite(od2)
    near = fin & ((np.abs(od1 - 0.8 * od2) <= NEAR_TIE) | (od2 - od1 <= NEAR_TIE))
    ok = ~near
    assert np.array_equal(m[r][ok], om[ok])
    both = ok & np.isfinite(od1)
    assert np.abs(d1[r][both] - od1[both]).max(initial=0) < 1e-5
    both = ok & fin
    assert np.abs(d2[r][both] - od2[both]).max(initial=0) < 1e-5
    return near.sum(), (om >= 0).sum()


def _unit(rng, n):
    d = np.abs(rng.standard_normal((n, 128))).astype(np.float32)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("precision", [lp.PREC_FP32, lp.PREC_BF16, lp.PREC_FP8])
@pytest.mark.parametrize("NA,NB", [(1, 2), (130, 1), (300, 517), (1000, 777), (2049, 4099), (257, 129)])
def test_match_synthetic(NA, NB, precision):
    rng = np.random.default_rng(NA + NB)
    A = _unit(rng, NA)
    B = _unit(rng, NB)
    k = min(NA, NB) // 2
    B[:k] = A[:k] + 0.03 * rng.standard_normal((k, 128)).astype(np.float32)
    B[:k] /= np.linalg.norm(B[:k], axis=1, keepdims=True)
    vA = (rng.uniform(size=NA) > 0.05).astype(np.uint8)
    vB = (rng.uniform(size=NB) > 0.05).astype(np.uint8)
    ctx = ctx_for((16,), precision=precision)
    _match_parity(ctx, A, vA, B, vB)


@pytest.mark.parametrize("precision", [lp.PREC_FP32, lp.PREC_BF16])
def test_match_640x480_stage_isolated(precision):
    p = synth.pair_640x480(0)
    Ls = synth.PAIR_640x480_LS
    fa = oracle.features(p.A, Ls)
    fb = oracle.features(p.B, Ls)
    dA = fa["desc"].astype(np.float32)
    dB = fb["desc"].astype(np.float32)
    rows = np.random.default_rng(1).choice(len(dA), 800, replace=False)
    ctx = ctx_for(Ls, precision=precision)
    near, acc = _match_parity(ctx, dA, fa["valid"], dB, fb["valid"], rows=rows)
    assert acc > 50 and near <= 2


def _same(a, b):
    return np.array_equal(a, b, equal_nan=True)


@pytest.mark.parametrize("low", [lp.PREC_BF16, lp.PREC_FP8])
@pytest.mark.parametrize("NA,NB", [(5, 7), (700, 1300), (5000, 4500)])
def test_match_bf16_bitidentical_to_fp32(NA, NB, low):
    # the BF16 and E4M3 forms re-rank exactly with the FP32 form's arithmetic:
    # identical outputs, bit for bit, on every row
    rng = np.random.default_rng(NA * 3 + NB)
    A = _unit(rng, NA)
    B = _unit(rng, NB)
    k = min(NA, NB) // 3
    B[:k] = A[:k] + 0.05 * rng.standard_normal((k, 128)).astype(np.float32)
    B[:k] = np.abs(B[:k]) / np.linalg.norm(B[:k], axis=1, keepdims=True)
    vA = (rng.uniform(size=NA) > 0.03).astype(np.uint8)
    vB = (rng.uniform(size=NB) > 0.03).astype(np.uint8)
    r32 = G.match(ctx_for((16,), precision=lp.PREC_FP32), A, vA, B, vB)
    r16 = G.match(ctx_for((16,), precision=low), A, vA, B, vB)
    for x, y in zip(r32, r16):
        assert _same(x, y)


def test_match_fp8_tensor_values_certify_exact_inputs():
    """E4M3 operands whose values are exact (four entries of 1/2 per unit
    descriptor: x 2^8 = 128, an E4M3 number): the tensor-core values equal the
    exact ones, the certified filter keeps a few columns per row, so nearly
    every row is decided by the E4M3 passes and the FP32 re-rank of their
    candidates, not by the FP32 re-scan -- and the outputs equal the FP32
    form's bit for bit (ties included)."""
    rng = np.random.default_rng(17)
    N = 6000

    def sparse(n):
        d = np.zeros((n, 128), np.float32)
        for i in range(n):
            d[i, rng.choice(128, 4, replace=False)] = 0.5
        return d
    A = sparse(N)
    B = sparse(N)
    B[: N // 2] = A[: N // 2]                   # exact duplicates for half the rows
    vA = np.ones(N, np.uint8)
    vB = np.ones(N, np.uint8)
    r32 = G.match(ctx_for((16,), precision=lp.PREC_FP32), A, vA, B, vB)
    c8 = ctx_for((16,), precision=lp.PREC_FP8)
    r8 = G.match(c8, A, vA, B, vB)
    for x, y in zip(r32, r8):
        assert _same(x, y)
    assert c8.lp_diag_last_rescans() < N // 20
    assert (r8[0] >= 0).sum() > N // 4


def test_match_bf16_bitidentical_2688x1600():
    """BF16 and E4M3 forms on the 2688x1600 pair: every output equals the FP32
    form's bit for bit.  The E4M3 filter's error bound (u = 2^-4) is 16 times
    the BF16 one, so many more of its rows fall back to the FP32 re-scan."""
    p = synth.pair_2688x1600(0)
    out, rescans = {}, {}
    for prec in (lp.PREC_FP32, lp.PREC_BF16, lp.PREC_FP8):
        ctx = ctx_for(synth.PAIR_2688x1600_LS, precision=prec)
        fa = lp.features(ctx, p.A)
        fb = lp.features(ctx, p.B)
        out[prec] = [G.host(t) for t in lp.match(ctx, fa, fb)]
        rescans[prec] = ctx.lp_diag_last_rescans()
    for low in (lp.PREC_BF16, lp.PREC_FP8):
        for x, y in zip(out[lp.PREC_FP32], out[low]):
            assert _same(x, y), low
    assert (out[lp.PREC_BF16][0] >= 0).sum() > 500
    assert rescans[lp.PREC_FP8] > rescans[lp.PREC_BF16]


def test_match_edge_cases():
    ctx = ctx_for((16,))
    rng = np.random.default_rng(3)
    A = _unit(rng, 10)
    m, d1, d2 = G.match(ctx, A, np.ones(10, np.uint8), A[:1], np.ones(1, np.uint8))
    assert (m == -1).all() and np.isinf(d2).all()                     # a single candidate: no ratio test
    m, d1, d2 = G.match(ctx, A, np.ones(10, np.uint8), A, np.zeros(10, np.uint8))
    assert (m == -1).all() and np.isinf(d1).all()                     # no valid candidate
    m, d1, d2 = G.match(ctx, A, np.zeros(10, np.uint8), A, np.ones(10, np.uint8))
    assert (m == -1).all()                                            # invalid queries
    m, d1, d2 = G.match(ctx, A, np.ones(10, np.uint8), A, np.ones(10, np.uint8))
    assert np.array_equal(m, np.arange(10)) and (d1 < 1e-3).all()     # identity


# ------------------------------------------------------------------ compaction + RANSAC
def test_compact_bitexact():
    rng = np.random.default_rng(4)
    NA, NB, WA, WB = 5000, 4000, 333, 250
    kpA = rng.integers(0, WA * 200, NA).astype(np.uint32)
    kpB = rng.integers(0, WB * 190, NB).astype(np.uint32)
    m = np.where(rng.uniform(size=NA) < 0.3, rng.integers(0, NB, NA), -1).astype(np.int32)
    pts, rows = G.compact(lp.Context(Ls=(16,)), kpA, WA, kpB, WB, m)
    want, wrows = oracle.match_points(kpA, kpB, m, WA, WB)
    assert np.array_equal(rows, wrows) and np.array_equal(pts, want.astype(np.float32))


def _synthetic_pts(rng, M, frac_in, noise=0.4, size=1500.0):
    Ht = np.eye(3)
    Ht[:2, :2] += 0.08 * rng.standard_normal((2, 2))
    Ht[:2, 2] = rng.uniform(-300, 300, 2)
    Ht[2, :2] = rng.uniform(-1e-4, 1e-4, 2)
    pa = np.round(rng.uniform(0, size, (M, 2)))
    pb = G.proj(Ht, pa) + noise * rng.standard_normal((M, 2))
    out = rng.uniform(size=M) > frac_in
    pb[out] = rng.uniform(0, size, (out.sum(), 2))
    return np.c_[pa, np.round(pb)].astype(np.float32), Ht


def _ransac_parity(ctx, pts, pair_id=0):
    r = G.ransac(ctx, pts, pair_id)
    o = oracle.ransac(pts.astype(np.float64), T=ctx.cfg.ransac_iters, thresh=float(ctx.cfg.thresh_px),
                      seed=int(ctx.cfg.seed), pair_id=pair_id)
    assert r["best_t"] == o["best_t"]
    if o["best_t"] < 0:
        assert r["n_in"] == 0 and not r["H"].any()
        return r, o
    e = np.sqrt(((G.proj(o["H"], pts[:, :2].astype(np.float64)) - pts[:, 2:]) ** 2).sum(1))
    border = np.abs(e - float(ctx.cfg.thresh_px)) <= 1e-4
    assert np.array_equal(r["inliers"][~border], o["inliers"][~border])
    sel = o["inliers"].astype(bool)
    q = pts[sel, :2].astype(np.float64)
    assert np.abs(G.proj(r["H"], q) - G.proj(o["H"], q)).max() < 1e-3
    return r, o


@pytest.mark.parametrize("M,frac", [(4, 1.0), (5, 0.8), (60, 0.5), (700, 0.35), (3000, 0.6), (9000, 0.2)])
def test_ransac_stage_isolated(M, frac):
    rng = np.random.default_rng(M)
    pts, Ht = _synthetic_pts(rng, M, frac)
    ctx = ctx_for((16,), seed=17)
    _ransac_parity(ctx, pts, pair_id=3)


def test_ransac_degenerate():
    ctx = ctx_for((16,))
    r = G.ransac(ctx, np.zeros((3, 4), np.float32))
    assert r["best_t"] == -1 and r["n_in"] == 0
    line = np.array([[i, 2 * i, i + 1, 2 * i] for i in range(12)], np.float32)
    r = G.ransac(ctx, line)
    assert r["best_t"] == -1 and r["n_in"] == 0 and not r["H"].any()
    r = G.ransac(ctx, np.zeros((0, 4), np.float32))
    assert r["best_t"] == -1


# ------------------------------------------------------------------ whole pair
# End-to-end match sets: GPU matches from GPU descriptors against oracle
# matches from oracle descriptors.  Descriptors agree within 1e-4 per
# component, so distances within 1e-4 * sqrt(128) * 2 plus margin: a row is an
# end-to-end near-tie when its ratio test or its runner-up is within 5e-3.
E2E_NEAR = 5e-3


def _e2e_near(om, od1, od2):
    """Rows whose ratio test is within E2E_NEAR of its boundary, and accepted
    rows whose runner-up is within E2E_NEAR of the nearest neighbour (a
    rejected row stays rejected whichever of the two is nearer)."""
    fin = np.isfinite(od2)
    return fin & ((np.abs(od1 - 0.8 * od2) <= E2E_NEAR) | ((om >= 0) & (od2 - od1 <= E2E_NEAR)))


def _match_set_parity(m_gpu, om, od1, od2, label):
    near = _e2e_near(om, od1, od2)
    ok = ~near
    diff = np.nonzero(m_gpu[ok] != om[ok])[0]
    print(f"{label}: {len(om)} rows, {int((om >= 0).sum())} oracle matches, {int(near.sum())} near-ties excluded, "
          f"{len(diff)} differing rows")
    assert len(diff) == 0, f"match[] differs from the oracle on {len(diff)} non-near-tie rows"
    assert near.sum() <= max(3, 0.03 * len(om))
    return int(near.sum())


def _overlap_points(Ht, h, w):
    ys, xs = np.mgrid[0:h:50, 0:w:50]
    q = np.c_[xs.ravel(), ys.ravel()].astype(np.float64)
    pb = G.proj(Ht, q)
    inside = (pb[:, 0] >= 0) & (pb[:, 0] < w) & (pb[:, 1] >= 0) & (pb[:, 1] < h)
    return q[inside]


@pytest.mark.parametrize("precision", [lp.PREC_FP32, lp.PREC_BF16])
def test_stitch_640x480_vs_oracle(precision):
    p = synth.pair_640x480(0)
    Ls = synth.PAIR_640x480_LS
    ctx = ctx_for(Ls, precision=precision)
    fa = lp.features(ctx, p.A)
    fb = lp.features(ctx, p.B)
    m = G.host(lp.match(ctx, fa, fb)[0])
    Hg, n_in, M = G.stitch(ctx, p.A, p.B)
    o = oracle.stitch_pair(p.A, p.B, Ls)
    # the whole match set, row by row (the stitch call's count is the same set's)
    _match_set_parity(m, o["match"], o["d1"], o["d2"], "640x480 end to end")
    assert M == int((m >= 0).sum())
    q = _overlap_points(p.H, 480, 640)
    assert np.abs(G.proj(Hg, q) - G.proj(o["H"], q)).max() < 0.5
    assert np.abs(G.proj(Hg, q) - G.proj(p.H, q)).max() < 2.0
    # RANSAC of the oracle on the GPU's own matches: same winner, same inliers
    # away from the 3 px boundary, H within 1e-3 px
    pts, _ = G.compact(ctx, G.host(fa.kp).astype(np.uint32), 640, G.host(fb.kp).astype(np.uint32), 640, m)
    r, orr = _ransac_parity(ctx, pts)
    assert r["n_in"] == n_in


def test_stitch_2688x1600_vs_oracle_sampled():
    """Paper-scale pair: 2,000 sampled query rows of the GPU match set against
    the oracle's (oracle descriptors of the sampled A points, all of B), and
    the GPU homography against the oracle's RANSAC on the GPU's own matches
    within 0.5 px over the overlap."""
    p = synth.pair_2688x1600(0)
    Ls = synth.PAIR_2688x1600_LS
    ctx = ctx_for(Ls, precision=lp.PREC_BF16)
    fa = lp.features(ctx, p.A)
    fb = lp.features(ctx, p.B)
    m = G.host(lp.match(ctx, fa, fb)[0])
    Hg, n_in, M = G.stitch(ctx, p.A, p.B)
    H_img, W_img = 1600, 2688
    kpA = G.host(fa.kp).astype(np.uint32)
    kpB = G.host(fb.kp).astype(np.uint32)
    gA = oracle.gray(p.A)
    gB = oracle.gray(p.B)
    assert np.array_equal(kpA, oracle.detect(gA, Ls)) and np.array_equal(kpB, oracle.detect(gB, Ls))
    _, ws = oracle.keypoint_scales(H_img, W_img, Ls)
    rows = np.sort(np.random.default_rng(7).choice(len(kpA), 2000, replace=False))
    oriA = oracle.orient(gA, kpA[rows], ws[rows])
    dA, vA = oracle.describe(gA, kpA[rows], ws[rows], oriA)
    oriB = oracle.orient(gB, kpB, ws)
    dB, vB = oracle.describe(gB, kpB, ws, oriB)
    om, od1, od2, _, _ = oracle.match(dA, vA, dB, vB, ratio=0.8)
    _match_set_parity(m[rows], om, od1, od2, "2688x1600 end to end, 2,000 sampled rows")
    assert M == int((m >= 0).sum()) and M > 500
    pts, _ = G.compact(ctx, kpA, W_img, kpB, W_img, m)
    orr = oracle.ransac(pts.astype(np.float64), T=ctx.cfg.ransac_iters, thresh=float(ctx.cfg.thresh_px),
                        seed=int(ctx.cfg.seed), pair_id=0)
    q = _overlap_points(p.H, H_img, W_img)
    inl = pts[orr["inliers"].astype(bool), :2].astype(np.float64)
    assert len(q) > 100 and orr["n_in"] >= 50
    dev = max(np.abs(G.proj(Hg, q) - G.proj(orr["H"], q)).max(), np.abs(G.proj(Hg, inl) - G.proj(orr["H"], inl)).max())
    print(f"2688x1600: H within {dev:.2e} px of the oracle's RANSAC on the GPU matches; n_in {n_in} / {orr['n_in']}")
    assert dev < 0.5
    assert abs(n_in - orr["n_in"]) <= max(2, 0.002 * orr["n_in"])
    assert np.abs(G.proj(Hg, q) - G.proj(p.H, q)).max() < 2.0
