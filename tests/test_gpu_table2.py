"""Table 2's LP-SIFT workloads (image sizes and window-size sets, including the
non-nested [32, 40] and [100, 128] and the large [256, 512]) through the C ABI
against the oracle: bit-exact peaks, and the whole pair's homography."""
from __future__ import annotations

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


@pytest.mark.parametrize("name", sorted(synth.TABLE2))
def test_table2_pair_vs_oracle(name):
    p, Ls = synth.table2_pair(name)
    h, w = p.A.shape
    ctx = lp.Context(Ls=Ls, precision=lp.PREC_BF16)
    o = oracle.stitch_pair(p.A, p.B, Ls)
    for img, f in ((p.A, o["fa"]), (p.B, o["fb"])):
        kp, _ = G.detect(ctx, img)
        assert len(kp) == lp.lp_num_keypoints(h, w, Ls)
        assert np.array_equal(kp, f["idx"])
    Hg, n_in, M = G.stitch(ctx, p.A, p.B)
    assert abs(M - (o["match"] >= 0).sum()) <= max(2, 0.01 * M)
    assert abs(n_in - o["n_in"]) <= max(2, 0.02 * o["n_in"])
    ys, xs = np.mgrid[0:h:32, 0:w:32]
    q = np.c_[xs.ravel(), ys.ravel()].astype(np.float64)
    pb = G.proj(p.H, q)
    q = q[(pb[:, 0] >= 0) & (pb[:, 0] < w) & (pb[:, 1] >= 0) & (pb[:, 1] < h)]
    assert n_in >= 20 and len(q) > 20
    assert np.abs(G.proj(Hg, q) - G.proj(o["H"], q)).max() < 0.5
    assert np.abs(G.proj(Hg, q) - G.proj(p.H, q)).max() < 3.0
