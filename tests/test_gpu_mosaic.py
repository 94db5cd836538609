"""Sec. 4 mosaic on the GPU: H_M of a shuffled 3 x 3 tile batch through
lp_stitch_pairs, the rounds (lp_mosaic_plan), and the canvas render against
the oracle's render of the same placements."""
import numpy as np
import pytest
import torch

import oracle
from paper_2405_08578_gb300 import lp, shard, synth

import gpu_util as G

pytestmark = pytest.mark.gpu


def _proj(Hm, pts):
    q = np.c_[pts, np.ones(len(pts))] @ np.asarray(Hm).T
    return q[:, :2] / q[:, 2:]


def _link_error(plan, Htrue, h, w):
    gy, gx = np.mgrid[0:h:16, 0:w:16]
    grid = np.c_[gx.ravel(), gy.ravel()].astype(np.float64)
    worst = 0.0
    for j, r in enumerate(plan["ref"]):
        if r < 0 or r == j:
            continue
        q = _proj(Htrue[(j, r)], grid)
        inside = (q[:, 0] >= 0) & (q[:, 0] <= w - 1) & (q[:, 1] >= 0) & (q[:, 1] <= h - 1)
        if inside.any():
            d = _proj(plan["G"][j], grid[inside]) - _proj(plan["G"][r], q[inside])
            worst = max(worst, float(np.abs(d).max()))
    return worst


@pytest.mark.parametrize("rgb", [True, False])
def test_mosaic_of_a_shuffled_tile_batch(rgb):
    h, w = 240, 320
    bt = synth.batch_3x3(seed=3, h=h, w=w, canvas_h=900, canvas_w=1300, rgb=rgb)
    ch = 3 if rgb else 1
    # 240 x 320 tiles: non-overlapping pairs can reach 8-10 chance inliers, so
    # an H_M entry needs 20 here (true neighbours have 24 or more)
    ctx = lp.Context(Ls=(8, 16, 32), precision=lp.PREC_BF16, min_inliers=20)
    bufs = [lp.pitched_device(im) for im in bt.images]
    images = [(b, h, w, p, ch) for (b, p) in bufs]
    P = 36
    HM = torch.zeros((P, 9), dtype=torch.float64, device="cuda")
    nin = torch.zeros(P, dtype=torch.int32, device="cuda")
    val = torch.zeros(P, dtype=torch.uint8, device="cuda")
    ctx.lp_stitch_pairs(images, HM, nin, val)
    pairs = shard.all_pairs(9)
    plan = lp.lp_mosaic_plan(9, pairs, G.host(HM), G.host(val), [(h, w)] * 9)
    assert (plan["round"] >= 0).all(), plan["round"]
    # each image agrees with the reference it was placed through, on the part
    # of the image that truly overlaps that reference
    err = _link_error(plan, bt.H, h, w)
    assert err < 3.0, err
    ch_, cw_ = plan["canvas"]
    pitch = (cw_ * ch + 15) // 16 * 16
    canvas = torch.zeros((ch_, pitch), dtype=torch.uint8, device="cuda")
    cover = torch.zeros((ch_, cw_), dtype=torch.uint8, device="cuda")
    ctx.lp_mosaic_render(images, plan["G"], plan["round"], canvas, cw_, ch_, pitch, cover)
    assert ctx.lp_sync_status() == 0
    got = G.host(canvas)[:, : cw_ * ch].reshape(ch_, cw_, ch) if rgb else G.host(canvas)[:, :cw_]
    gcov = G.host(cover)
    want, wcov = oracle.mosaic_render(bt.images, plan["G"], plan["round"], (ch_, cw_))
    same = gcov == wcov
    assert same.mean() > 0.999
    diff = np.abs(got.astype(np.int32) - want.astype(np.int32))
    d = diff[same] if not rgb else diff[same].reshape(-1)
    assert d.max() <= 1 and (d == 0).mean() > 0.99
    assert (gcov > 0).mean() > 0.5


def test_render_rejects_bad_input():
    ctx = lp.Context(Ls=(8,))
    img, pitch = lp.pitched_device(np.zeros((16, 16), np.uint8))
    canvas = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(lp.LpError):   # canvas pitch smaller than the width
        ctx.lp_mosaic_render([(img, 16, 16, pitch, 1)], np.eye(3)[None], [0], canvas, 16, 16, 8)
    with pytest.raises(lp.LpError):   # singular placement
        ctx.lp_mosaic_render([(img, 16, 16, pitch, 1)], np.zeros((1, 3, 3)), [0], canvas, 16, 16, 16)
