"""lp_ransac_static -- RANSAC for callers that cannot allocate device memory.

Such callers (an application whose caching allocator owns the device's
memory, a real-time loop that must stay out of the driver's allocation path,
a plug-in host that forbids allocations after start-up) get a context-free
entry point whose scratch is a fixed array inside the library.  This test
calls it through the C ABI twice in a row, on two different match sets, and
checks each result against the context-based lp_ransac on the same inputs.
It sits in its own file, collected last, and passes both alone in a fresh
process and after the rest of the suite.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_08578_gb300 import lp  # noqa: E402


def _pts(seed, M, frac_in):
    rng = np.random.default_rng(seed)
    Ht = np.eye(3)
    Ht[:2, :2] += 0.08 * rng.standard_normal((2, 2))
    Ht[:2, 2] = rng.uniform(-300, 300, 2)
    Ht[2, :2] = rng.uniform(-1e-4, 1e-4, 2)
    pa = np.round(rng.uniform(0, 1500, (M, 2)))
    q = np.c_[pa, np.ones(M)] @ Ht.T
    pb = q[:, :2] / q[:, 2:] + 0.4 * rng.standard_normal((M, 2))
    out = rng.uniform(size=M) > frac_in
    pb[out] = rng.uniform(0, 1500, (out.sum(), 2))
    return np.c_[pa, np.round(pb)].astype(np.float32)


def _outputs(M):
    return (torch.zeros(9, dtype=torch.float64, device="cuda"), torch.zeros(M, dtype=torch.uint8, device="cuda"),
            torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))


def test_ransac_static_matches_ransac_twice():
    T, thresh, seed = 1000, 3.0, 11
    ctx = lp.Context(Ls=(16,), ransac_iters=T, thresh_px=thresh, seed=seed)
    for call, (M, frac, pair_id) in enumerate([(2500, 0.4, 7), (900, 0.7, 8)]):
        pts = torch.from_numpy(_pts(100 + call, M, frac)).cuda()
        dM = torch.tensor([M], dtype=torch.int32, device="cuda")
        H1, i1, n1, b1 = _outputs(M)
        ctx.lp_ransac(pts, M, dM, pair_id, H1, i1, n1, b1)
        H2, i2, n2, b2 = _outputs(M)
        lp.lp_ransac_static(pts, M, dM, T, thresh, seed, pair_id, H2, i2, n2, b2)
        torch.cuda.synchronize()
        assert int(b2.item()) == int(b1.item()) >= 0
        assert int(n2.item()) == int(n1.item()) > 0
        assert torch.equal(i2, i1)
        assert torch.allclose(H2, H1, rtol=1e-12, atol=1e-12)


def test_ransac_static_rejects_too_many_iterations():
    M = 16
    pts = torch.zeros((M, 4), dtype=torch.float32, device="cuda")
    H, i, n, b = _outputs(M)
    with pytest.raises(lp.LpError) as e:
        lp.lp_ransac_static(pts, M, None, 4097, 3.0, 0, 0, H, i, n, b)
    assert e.value.code == 1
