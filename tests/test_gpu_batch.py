"""H_M of Sec. 4 through lp_stitch_pairs: every entry equals the single-pair
path with the same pair index, the captured graph replays identically, and on
the 3 x 3 tile batch the neighbouring tiles are registered to their true
homographies."""
import numpy as np
import pytest

from paper_2405_08578_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_08578_gb300 import lp  # noqa: E402
import gpu_util as G  # noqa: E402


def _outputs(P):
    return (torch.zeros((P, 9), dtype=torch.float64, device="cuda"), torch.zeros(P, dtype=torch.int32, device="cuda"),
            torch.zeros(P, dtype=torch.uint8, device="cuda"), torch.zeros(P, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("precision", [lp.PREC_FP32, lp.PREC_BF16, lp.PREC_FP8])
def test_stitch_pairs_equals_single_pair_path(precision):
    h, w = 240, 320
    base = synth.small_pair(h, w, seed=21, theta_deg=3.0, scale=1.02, shift=0.25)
    other = synth.small_pair(h, w, seed=22, theta_deg=-2.0, scale=0.99, shift=0.2)
    imgs = [base.A, base.B, other.A, other.B]
    bufs = [lp.pitched_device(im) for im in imgs]
    ctx = lp.Context(Ls=(8, 16, 32), precision=precision, seed=5)
    images = [(b, h, w, p, 1) for (b, p) in bufs]
    P = 6
    HM, n_in, valid, M = _outputs(P)
    ctx.lp_stitch_pairs(images, HM, n_in, valid, M_out=M)
    torch.cuda.synchronize()
    first = [t.clone() for t in (HM, n_in, valid, M)]
    q = 0
    for i in range(4):
        for j in range(i + 1, 4):
            H1 = torch.zeros(9, dtype=torch.float64, device="cuda")
            n1 = torch.zeros(1, dtype=torch.int32, device="cuda")
            M1 = torch.zeros(1, dtype=torch.int32, device="cuda")
            ctx.lp_stitch_pair(bufs[i][0], h, w, bufs[i][1], bufs[j][0], h, w, bufs[j][1], 1, q, H1, n1, M1)
            torch.cuda.synchronize()
            assert torch.equal(HM[q], H1) and int(n_in[q]) == int(n1) and int(M[q]) == int(M1)
            assert int(valid[q]) == int(int(n1) >= 8)
            q += 1
    assert int(valid[0]) == 1 and int(valid[5]) == 1          # (A, B) pairs of each scene
    # graph replay: same outputs
    for t in (HM, n_in, valid, M):
        t.zero_()
    ctx.lp_stitch_pairs(images, HM, n_in, valid, M_out=M)
    torch.cuda.synchronize()
    for a, b in zip(first, (HM, n_in, valid, M)):
        assert torch.equal(a, b)


def test_stitch_pairs_explicit_pair_list_and_errors():
    h, w = 160, 224
    p = synth.small_pair(h, w, seed=3)
    bufs = [lp.pitched_device(im) for im in (p.A, p.B)]
    ctx = lp.Context(Ls=(8, 16))
    images = [(b, h, w, q, 1) for (b, q) in bufs]
    HM, n_in, valid, M = _outputs(2)
    ctx.lp_stitch_pairs(images, HM, n_in, valid, pairs=[(0, 1), (1, 0)], M_out=M)
    torch.cuda.synchronize()
    H01 = HM[0].cpu().numpy().reshape(3, 3)
    H10 = HM[1].cpu().numpy().reshape(3, 3)
    q = np.array([[60.0, 50], [150, 50], [150, 120], [60, 120]])
    assert np.abs(G.proj(H10, G.proj(H01, q)) - q).max() < 1.0   # the two directions invert each other
    with pytest.raises(lp.LpError):
        ctx.lp_stitch_pairs(images, HM, n_in, valid, pairs=[(0, 2)])
    with pytest.raises(lp.LpError):
        ctx.lp_stitch_pairs(images[:1], HM, n_in, valid)


def test_stitch_pairs_3x3_tiles():
    b = synth.batch_3x3(seed=1)
    ctx = lp.Context(Ls=synth.PAIR_2688x1600_LS, precision=lp.PREC_BF16)
    bufs = [lp.pitched_device(im) for im in b.images]
    images = [(t, 1600, 2688, p, 3) for (t, p) in bufs]
    HM, n_in, valid, M = _outputs(36)
    ctx.lp_stitch_pairs(images, HM, n_in, valid, M_out=M)
    torch.cuda.synchronize()
    HMh, v = HM.cpu().numpy().reshape(36, 3, 3), valid.cpu().numpy()
    q = 0
    found = 0
    for i in range(9):
        for j in range(i + 1, 9):
            gi, gj = divmod(int(b.order[i]), 3), divmod(int(b.order[j]), 3)
            neighbour = abs(gi[0] - gj[0]) + abs(gi[1] - gj[1]) == 1
            if neighbour:
                assert v[q] == 1, (i, j)
                Ht = b.H[(i, j)]
                ys, xs = np.mgrid[0:1600:40, 0:2688:40]
                pts = np.c_[xs.ravel(), ys.ravel()].astype(np.float64)
                pb = G.proj(Ht, pts)
                ov = (pb[:, 0] >= 0) & (pb[:, 0] < 2688) & (pb[:, 1] >= 0) & (pb[:, 1] < 1600)
                assert np.abs(G.proj(HMh[q], pts[ov]) - pb[ov]).max() < 2.0, (i, j)
                found += 1
            q += 1
    assert found == 12


def test_pair_ids_let_a_shard_reproduce_the_full_list():
    """The pair subset a rank would run (shard.shard) with lp_stitch_pairs_ids
    gives exactly the full list's entries for those pairs."""
    from paper_2405_08578_gb300 import shard
    h, w = 240, 320
    s1 = synth.small_pair(h, w, seed=31, theta_deg=2.0, shift=0.25)
    s2 = synth.small_pair(h, w, seed=32, theta_deg=-3.0, shift=0.3)
    imgs = [s1.A, s1.B, s2.A, s2.B, s1.B]
    bufs = [lp.pitched_device(im) for im in imgs]
    images = [(b, h, w, p, 1) for (b, p) in bufs]
    ctx = lp.Context(Ls=(8, 16, 32), precision=lp.PREC_BF16, seed=9)
    pl = shard.all_pairs(len(imgs))
    P = len(pl)
    HM, n_in, valid, M = _outputs(P)
    ctx.lp_stitch_pairs(images, HM, n_in, valid, M_out=M)
    torch.cuda.synchronize()
    for world in (2, 3):
        for rank in range(world):
            mine = shard.shard(P, world, rank)
            h2, n2, v2, m2 = _outputs(len(mine))
            ctx.lp_stitch_pairs(images, h2, n2, v2, pairs=[pl[q] for q in mine], M_out=m2, pair_ids=mine)
            torch.cuda.synchronize()
            idx = torch.tensor(mine, device="cuda")
            assert torch.equal(h2, HM[idx]) and torch.equal(n2, n_in[idx]) and torch.equal(m2, M[idx])


@pytest.mark.parametrize("rgb", [False, True])
def test_host_buffer_pair_equals_device_pair(rgb):
    """lp_stitch_pair_host (host images, uploads on two streams) returns the
    device call's H, inlier count and match count exactly, on repeated calls
    that alternate between two pairs (its upload buffers are reused)."""
    pairs = [synth.small_pair(240, 320, s, theta_deg=3.0 * s, shift=0.3, rgb=rgb) for s in (1, 2)]
    ctx = lp.Context(Ls=(8, 16, 32), precision=lp.PREC_BF16)
    ch = 3 if rgb else 1
    want = []
    for k, p in enumerate(pairs):
        H, n, M = G.stitch(ctx, p.A, p.B, pair_id=k)
        want.append((H, n, M))
    hosts = []
    for p in pairs:
        a, pa = lp.pitched_device(p.A)
        b, pb = lp.pitched_device(p.B)
        hosts.append((a.cpu().pin_memory(), pa, b.cpu().pin_memory(), pb))
    for rep in range(3):
        for k, (a, pa, b, pb) in enumerate(hosts):
            H, n, M = ctx.lp_stitch_pair_host(a, 240, 320, pa, b, 240, 320, pb, ch, k)
            assert np.array_equal(np.array(H), want[k][0]) and n == want[k][1] and M == want[k][2], (rep, k)


@pytest.mark.parametrize("rgb", [False, True])
def test_host_stream_equals_host_pair_calls(rgb):
    """lp_stitch_pairs_host (uploads of the next pair on a copy stream while
    the current pair is computed, two alternating upload slots) gives every
    pair exactly what lp_stitch_pair_host gives it, for pairs of different
    sizes (slots reused, buffers grown), pageable or pinned host images, and
    on a second call; P = 0 is a no-op and bad arguments are refused."""
    ch = 3 if rgb else 1
    ps = [synth.small_pair(240, 320, 1, theta_deg=3.0, shift=0.3, rgb=rgb),
          synth.small_pair(300, 416, 2, theta_deg=-4.0, shift=0.25, rgb=rgb),
          synth.small_pair(200, 272, 3, theta_deg=6.0, shift=0.3, rgb=rgb),
          synth.small_pair(240, 320, 4, theta_deg=1.0, shift=0.35, rgb=rgb),
          synth.small_pair(320, 480, 5, theta_deg=-2.0, shift=0.3, rgb=rgb)]
    ctx = lp.Context(Ls=(8, 16, 32), precision=lp.PREC_BF16)
    entries = []
    for q, p in enumerate(ps):
        a, pa = lp.pitched_device(p.A)
        b, pb = lp.pitched_device(p.B)
        h, w = p.A.shape[:2]
        A, B = a.cpu(), b.cpu()
        if q % 2:
            A, B = A.pin_memory(), B.pin_memory()
        entries.append((A, h, w, pa, B, h, w, pb))
    want = [ctx.lp_stitch_pair_host(A, h, w, pa, B, h2, w2, pb, ch, 7 + q)
            for q, (A, h, w, pa, B, h2, w2, pb) in enumerate(entries)]
    for rep in range(2):
        H, n, M = ctx.lp_stitch_pairs_host(entries, ch, pair_id0=7)
        for q in range(len(ps)):
            assert np.array_equal(H[q], np.array(want[q][0])) and n[q] == want[q][1] and M[q] == want[q][2], (rep, q)
    assert int(n.min()) >= 8
    H0, n0, M0 = ctx.lp_stitch_pairs_host([], ch)
    assert len(n0) == 0
    A, h, w, pa, B, h2, w2, pb = entries[0]
    with pytest.raises(lp.LpError):
        ctx.lp_stitch_pairs_host([(A, h, w, pa + 1, B, h2, w2, pb)], ch)


@pytest.mark.parametrize("rgb", [False, True])
def test_stitch_pairs_uneven_sizes_equal_single_pairs(rgb):
    """Images of different sizes in one batch (unequal point counts per pair):
    every H_M entry, inlier and match count equals the single-pair call's."""
    s1 = synth.small_pair(240, 320, seed=31, theta_deg=2.0, shift=0.25, rgb=rgb)
    s2 = synth.small_pair(300, 420, seed=32, theta_deg=-3.0, shift=0.3, rgb=rgb)
    imgs = [s1.A, s2.A, s1.B, s2.B]
    ch = 3 if rgb else 1
    bufs = [lp.pitched_device(im) for im in imgs]
    ctx = lp.Context(Ls=(8, 16, 32), precision=lp.PREC_BF16, seed=3)
    images = [(b, im.shape[0], im.shape[1], p, ch) for (b, p), im in zip(bufs, imgs)]
    P = 6
    HM, n_in, valid, M = _outputs(P)
    for rep in range(2):                       # eager, then graph replay
        for t in (HM, n_in, valid, M):
            t.zero_()
        ctx.lp_stitch_pairs(images, HM, n_in, valid, M_out=M)
        torch.cuda.synchronize()
        q = 0
        for i in range(4):
            for j in range(i + 1, 4):
                (bi, pi), (bj, pj) = bufs[i], bufs[j]
                H1 = torch.zeros(9, dtype=torch.float64, device="cuda")
                n1 = torch.zeros(1, dtype=torch.int32, device="cuda")
                M1 = torch.zeros(1, dtype=torch.int32, device="cuda")
                ctx.lp_stitch_pair(bi, imgs[i].shape[0], imgs[i].shape[1], pi, bj, imgs[j].shape[0],
                                   imgs[j].shape[1], pj, ch, q, H1, n1, M1)
                torch.cuda.synchronize()
                assert torch.equal(HM[q], H1) and int(n_in[q]) == int(n1) and int(M[q]) == int(M1), (rep, i, j)
                q += 1
        assert int(valid[1]) == 1 and int(valid[4]) == 1   # (s1.A, s1.B) and (s2.A, s2.B)


def test_uneven_pairs_batch_equals_single_pairs_and_truth():
    """Independent pairs of uneven sizes and aspect ratios in one explicit pair
    list (the 64-pair uneven workload's shape, here at long sides 480..1024):
    every entry equals lp_stitch_pair with the same pair id, every pair is
    registered within 1 px of its true homography, and two of them agree with
    the oracle's H within 0.5 px."""
    import oracle
    ps = synth.uneven_pairs(12, seed=2, long_hi=1024)
    Ls = synth.PAIR_2688x1600_LS
    imgs = [im for p in ps for im in (p.A, p.B)]
    bufs = [lp.pitched_device(im) for im in imgs]
    images = [(b, im.shape[0], im.shape[1], pt, 1) for (b, pt), im in zip(bufs, imgs)]
    ctx = lp.Context(Ls=Ls, precision=lp.PREC_BF16, seed=0)
    P = len(ps)
    HM, n_in, valid, M = _outputs(P)
    ctx.lp_stitch_pairs(images, HM, n_in, valid, pairs=[(2 * q, 2 * q + 1) for q in range(P)], M_out=M,
                        pair_ids=list(range(P)))
    torch.cuda.synchronize()
    assert int(valid.sum()) == P
    HMh = HM.cpu().numpy().reshape(P, 3, 3)
    for q, p in enumerate(ps):
        h, w = p.A.shape
        (ba, pa), (bb, pb_) = bufs[2 * q], bufs[2 * q + 1]
        H1 = torch.zeros(9, dtype=torch.float64, device="cuda")
        n1 = torch.zeros(1, dtype=torch.int32, device="cuda")
        M1 = torch.zeros(1, dtype=torch.int32, device="cuda")
        ctx.lp_stitch_pair(ba, h, w, pa, bb, h, w, pb_, 1, q, H1, n1, M1)
        torch.cuda.synchronize()
        assert torch.equal(HM[q], H1) and int(n_in[q]) == int(n1) and int(M[q]) == int(M1), q
        ys, xs = np.mgrid[0:h:max(1, h // 12), 0:w:max(1, w // 12)]
        pts = np.c_[xs.ravel(), ys.ravel()].astype(np.float64)
        tb = G.proj(p.H, pts)
        ov = (tb[:, 0] >= 0) & (tb[:, 0] < w) & (tb[:, 1] >= 0) & (tb[:, 1] < h)
        assert np.abs(G.proj(HMh[q], pts[ov]) - tb[ov]).max() < 1.0, q
        if q in (2, 10):
            o = oracle.stitch_pair(p.A, p.B, Ls)
            assert abs(int(n_in[q]) - o["n_in"]) <= 3, q
            assert np.abs(G.proj(HMh[q], pts[ov]) - G.proj(o["H"], pts[ov])).max() < 0.5, q


def test_degenerate_pairs_report_no_model():
    """Edge cases of the whole path: an image smaller than every window (no
    feature points), a flat image (no valid descriptor), and both in a batch:
    the calls succeed, report no model (H = 0, n_in = 0) and leave the context
    usable."""
    ctx = lp.Context(Ls=(16, 32), precision=lp.PREC_BF16)
    tiny = np.full((12, 12), 90, np.uint8)
    flat = np.full((64, 96), 90, np.uint8)
    real = synth.small_pair(128, 160, seed=41, shift=0.2)
    for A, B in ((tiny, real.A), (real.A, tiny), (tiny, tiny), (flat, real.B), (real.A, flat)):
        H, n, M = G.stitch(ctx, A, B)
        assert n == 0 and M == 0 and not H.any(), (A.shape, B.shape)
        assert ctx.lp_sync_status() == 0
    H, n, M = G.stitch(ctx, real.A, real.B, pair_id=4)   # the batch's pair (1, 3) has pair id 4
    assert n >= 8
    imgs = [tiny, real.A, flat, real.B]
    bufs = [lp.pitched_device(im) for im in imgs]
    images = [(b, im.shape[0], im.shape[1], p, 1) for (b, p), im in zip(bufs, imgs)]
    HM, n_in, valid, Mo = _outputs(6)
    ctx.lp_stitch_pairs(images, HM, n_in, valid, M_out=Mo)
    torch.cuda.synchronize()
    assert ctx.lp_sync_status() == 0
    # only (real.A, real.B) = pair (1, 3), index 4, has a model
    v = valid.cpu().numpy()
    assert v[4] == 1 and v.sum() == 1 and int(n_in[4]) == n
    assert not HM[[0, 1, 2, 3, 5]].any()


@pytest.mark.parametrize("case", ["gray14", "rgb5", "nonnested", "alpha", "tma_rgb_ragged", "tma_gray_ragged",
                                  "tiles3x3"])
def test_detect_batch_equals_single_images(case):
    """lp_detect_batch (images sharing launches) gives every image exactly the
    peaks and intensity of lp_detect: more images than one launch takes, mixed
    sizes, RGB widths that are not multiples of 16, the configurations that
    detect image by image, the tile-streaming path on ragged sizes (partial
    128-pixel tiles at the right and bottom) and the nine 2688x1600 RGB tiles
    of the shuffled 3x3 batch."""
    rng = np.random.default_rng(len(case))
    Ls, alpha, ch, n = (16, 32, 64), 0.0, 1, 5
    lo, hi = (70, 400), (70, 500)
    if case == "gray14":
        n = 14
    elif case == "rgb5":
        ch = 3
    elif case == "nonnested":
        Ls = (12, 20)
    elif case == "alpha":
        alpha = 1e-4
    elif case.startswith("tma"):
        Ls, ch, n, lo, hi = (16, 32, 64, 128), 3 if "rgb" in case else 1, 13, (128, 700), (130, 900)
    if case == "tiles3x3":
        Ls, ch = (16, 32, 64, 128), 3
        imgs = synth.batch_3x3(seed=1).images
    else:
        shapes = [(int(rng.integers(*lo)), int(rng.integers(*hi))) for _ in range(n)]
        imgs = [rng.integers(0, 256, size=s + ((3,) if ch == 3 else ())).astype(np.uint8) for s in shapes]
    ctx = lp.Context(Ls=Ls, alpha=alpha)
    bufs = [lp.pitched_device(im) for im in imgs]
    images = [(b, im.shape[0], im.shape[1], p, ch) for (b, p), im in zip(bufs, imgs)]
    Ks = [lp.lp_num_keypoints(im.shape[0], im.shape[1], Ls) for im in imgs]
    kps = [torch.full((max(K, 1),), -1, dtype=torch.int32, device="cuda") for K in Ks]
    grays = [torch.zeros(im.shape[0] * im.shape[1] + 16, dtype=torch.uint8, device="cuda") for im in imgs] \
        if ch == 3 else None
    ctx.lp_detect_batch(images, kps, grays)
    torch.cuda.synchronize()
    assert ctx.lp_sync_status() == 0
    for i, im in enumerate(imgs):
        kp1, g1 = G.detect(ctx, im)
        assert np.array_equal(G.host(kps[i])[:Ks[i]].astype(np.uint32), kp1), (case, i, im.shape)
        if ch == 3:
            assert np.array_equal(G.host(grays[i])[:im.shape[0] * im.shape[1]].reshape(im.shape[:2]), g1)


def test_autotuned_matcher_equals_builtin_and_caches():
    """lp_set_autotune: the tuned (splits, pass-1 stride) give the built-in
    choice's outputs bit for bit, one table row per size class, reused on the
    class's later calls."""
    Ls = (16, 32, 64, 128)
    base = lp.Context(Ls=Ls, precision=lp.PREC_BF16)
    tun = lp.Context(Ls=Ls, precision=lp.PREC_BF16)
    tun.lp_set_autotune(True)
    pairs = synth.uneven_pairs(3, seed=5, long_lo=480, long_hi=900)
    for rep in range(2):
        for p in pairs:
            fa, fb = lp.features(base, p.A), lp.features(base, p.B)
            want = [G.host(t) for t in lp.match(base, fa, fb)]
            got = [G.host(t) for t in lp.match(tun, fa, fb)]
            for x, y in zip(want, got):
                assert np.array_equal(x, y, equal_nan=True)
        table = tun.lp_autotune_table()
        if rep == 0:
            first = table
        assert table == first and 1 <= len(table) <= 3
    for row in table:
        assert 1 <= row["splits"] <= 16 and row["pass1_stride"] in (2, 3, 4)
        assert 0 < row["tuned_us"] <= row["builtin_us"]
    assert tun.lp_sync_status() == 0


def test_autotuned_batch_equals_builtin_and_fills_the_table():
    """lp_stitch_pairs with the tuner on: the first call runs the built-in
    choice and tunes every size class it met, later calls run the tuned
    choice (a new graph); every call's outputs equal the built-in context's
    bit for bit."""
    Ls = (16, 32, 64, 128)
    ps = synth.uneven_pairs(4, seed=7, long_lo=480, long_hi=1400)
    imgs = [im for p in ps for im in (p.A, p.B)]
    bufs = [lp.pitched_device(im) for im in imgs]
    images = [(b, im.shape[0], im.shape[1], pt, 1) for (b, pt), im in zip(bufs, imgs)]
    plist = [(2 * q, 2 * q + 1) for q in range(len(ps))]
    base = lp.Context(Ls=Ls, precision=lp.PREC_BF16)
    tun = lp.Context(Ls=Ls, precision=lp.PREC_BF16)
    tun.lp_set_autotune(True)
    want = _outputs(len(ps))
    base.lp_stitch_pairs(images, *want[:3], pairs=plist, M_out=want[3])
    torch.cuda.synchronize()
    buckets = {int(np.ceil(np.log2(lp.lp_num_keypoints(p.A.shape[0], p.A.shape[1], Ls)))) for p in ps}
    for call in range(3):
        got = _outputs(len(ps))
        tun.lp_stitch_pairs(images, *got[:3], pairs=plist, M_out=got[3])
        torch.cuda.synchronize()
        for x, y in zip(want, got):
            assert torch.equal(x, y), call
        table = tun.lp_autotune_table()
        assert {(r["log2_NA"], r["log2_NB"]) for r in table} == {(b, b) for b in buckets}
        if call == 0:
            first = table
        assert table == first
    for row in table:
        assert 1 <= row["splits"] <= 16 and row["pass1_stride"] in (2, 3, 4)
    assert tun.lp_sync_status() == 0 and base.lp_sync_status() == 0


def test_batch_wait_gives_up_and_context_recovers():
    """The batched distance passes run in one persistent launch in which a
    pass-2 unit waits (at most 2 s) for its rows' pass-1 values.  A hold makes
    every such wait expect a count the launch never reaches: the waits give up,
    the status word reports LP_ERR_TIMEOUT, the call returns, and once the hold
    is removed the same context gives the results of a fresh one."""
    import time
    Ls = (16, 32, 64, 128)
    imgs = [synth.small_pair(300, 400, seed=s).A for s in (11, 12, 13)]
    bufs = [lp.pitched_device(im) for im in imgs]
    images = [(b, im.shape[0], im.shape[1], p, 1) for (b, p), im in zip(bufs, imgs)]
    ctx = lp.Context(Ls=Ls, precision=lp.PREC_BF16)
    HM, n_in, valid, _ = _outputs(3)
    ctx.lp_diag_set_batch_hold(1)
    t0 = time.time()
    ctx.lp_stitch_pairs(images, HM, n_in, valid)
    st = ctx.lp_sync_status()
    assert st == 4, lp.ERR_NAMES.get(st, st)          # LP_ERR_TIMEOUT
    assert time.time() - t0 < 60
    ctx.lp_diag_set_batch_hold(0)
    ctx.lp_stitch_pairs(images, HM, n_in, valid)
    assert ctx.lp_sync_status() == 0
    fresh = lp.Context(Ls=Ls, precision=lp.PREC_BF16)
    HM2, n2, v2, _ = _outputs(3)
    fresh.lp_stitch_pairs(images, HM2, n2, v2)
    assert fresh.lp_sync_status() == 0
    assert torch.equal(HM, HM2) and torch.equal(n_in, n2) and torch.equal(valid, v2)
