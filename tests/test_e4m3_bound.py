"""The E4M3 filter's error bound, checked on the host.

The E4M3 form of the tensor-core matcher rounds every entry of a unit
descriptor times 2^8 to E4M3 (3 mantissa bits: u = 2^-4, subnormals below
2^-6) and sums the exact products in FP32, so D~ = (sum q_a q_b) / 2^16 and
v~ = 1 - 2 D~.  It lists every column with v~ <= x + delta8(x) and certifies a
row only when the exact second-best is below x, which is exact provided
|v~ - v| <= delta8(v) and v + delta8(v) increases with v, for
delta8(v) = c8 + k8 (1 + eps - v), k8 = 2u + u^2, eps = 5e-5, c8 = 4e-4 (the
BF16 form's 2e-4 plus 2e-4 for entries in E4M3's subnormal range).
"""
import zlib

import numpy as np
import pytest

import test_bf16_bound as BF

torch = pytest.importorskip("torch")
if not hasattr(torch, "float8_e4m3fn"):  # pragma: no cover
    pytest.skip("no float8_e4m3fn in this torch", allow_module_level=True)

U = 2.0 ** -4
K8 = 2 * U + U * U
EPS = 5e-5
C8 = 4e-4
SCALE = 256.0


def delta8(v):
    return C8 + K8 * (1 + EPS - v)


def _e4m3(x):
    q = torch.from_numpy(np.ascontiguousarray(x * np.float32(SCALE))).to(torch.float8_e4m3fn).float().numpy()
    assert np.isfinite(q).all() and q.max() <= 448.0
    return q


def _estimate(A, B):
    Aq, Bq = _e4m3(A), _e4m3(B)
    D = np.zeros((len(A), len(B)), np.float32)
    for k in range(128):
        D = (D + np.outer(Aq[:, k], Bq[:, k]).astype(np.float32)).astype(np.float32)
    return 1.0 - 2.0 * D.astype(np.float64) / (SCALE * SCALE)


def _small_entries(rng, n):
    # most entries far below 2^-14 (E4M3's subnormal range after the scale),
    # a few large ones carrying the norm
    d = np.abs(rng.standard_normal((n, 128))) * 1e-5
    d[:, :4] = np.abs(rng.standard_normal((n, 4)))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)


@pytest.mark.parametrize("kind", ["random", "near_duplicates", "duplicates", "sparse", "small_entries",
                                  "one_hot"])
def test_estimate_within_e4m3_bound(kind):
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    A = BF._descriptors(rng, 64, sparse=0.7 if kind == "sparse" else 0.0)
    if kind in ("random", "sparse"):
        B = BF._descriptors(rng, 96, sparse=0.7 if kind == "sparse" else 0.0)
    elif kind == "near_duplicates":
        B = np.abs(A + 0.01 * rng.standard_normal(A.shape)).astype(np.float32)
        B /= np.linalg.norm(B, axis=1, keepdims=True)
    elif kind == "duplicates":
        B = A.copy()
    elif kind == "small_entries":
        A = _small_entries(rng, 48)
        B = np.concatenate([A, _small_entries(rng, 48)])
    else:
        # a single entry of 1: the largest value the scale must keep below 448
        A = np.eye(128, dtype=np.float32)[:64]
        B = np.eye(128, dtype=np.float32)[rng.permutation(128)[:96]]
    v = BF._exact(A, B)
    err = np.abs(_estimate(A, B) - v)
    assert (err <= delta8(v)).all(), float((err - delta8(v)).max())
    if kind in ("near_duplicates", "duplicates"):
        diag = np.arange(len(A))
        assert err[diag, diag].max() > 1e-3         # E4M3 rounding is visible, and still inside the bound


def test_e4m3_window_top_is_monotone():
    v = np.linspace(-1.0 - EPS, 1.0 + EPS, 200001)
    top = v + delta8(v)
    assert (np.diff(top) > 0).all()
