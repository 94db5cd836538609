"""The BF16 filter's error bound, checked on the host.

The tensor-core matcher estimates v = |b|^2 - 2 a.b for unit descriptors a, b
(non-negative entries) as v~ = 1 - 2 D, with D the FP32 sum of the BF16-rounded
products.  It lists every column with v~ <= x + delta(x) and certifies a row
only when the exact second-best is below x.  That is exact provided
|v~ - v| <= delta(v) and v + delta(v) increases with v, for
delta(v) = c + k (1 + eps - v), k = 2u + u^2, u = 2^-8, eps = 5e-5, c = 2e-4.
These tests check both claims on random, near-duplicate, duplicate, sparse and
orthogonal descriptors shaped like the 128-d descriptors of Sec. 2.3 (entries
clamped at 0.2 and renormalised).
"""
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")

U = 2.0 ** -8
K = 2 * U + U * U
EPS = 5e-5
C = 2e-4


def delta(v):
    return C + K * (1 + EPS - v)


def _descriptors(rng, n, sparse=0.0):
    d = np.abs(rng.standard_normal((n, 128)))
    if sparse:
        d[rng.uniform(size=d.shape) < sparse] = 0.0
        d[:, 0] += 1e-3
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    d = np.minimum(d, 0.2)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d.astype(np.float32)


def _adversarial(rng, n):
    # 42 entries just above 2^-3 and 85 just above 2^-4, each 0.999 of the way
    # to the BF16 rounding midpoint, so every one rounds down by almost u; one
    # last entry brings the norm to 1.  BF16 products then fall short of the
    # exact ones by almost 2u each, the worst case the bound allows for.
    out = np.zeros((n, 128))
    for i in range(n):
        m = np.r_[np.full(42, 2.0 ** -3), np.full(85, 2.0 ** -4)]
        a = m * (1 + 0.999 * 2.0 ** -8)
        pos = rng.permutation(128)
        out[i, pos[:127]] = a
        out[i, pos[127]] = np.sqrt(1.0 - (a * a).sum())
    return out.astype(np.float32)


def _bf16(x):
    return torch.from_numpy(x).to(torch.bfloat16).float().numpy()


def _estimate(A, B):
    # FP32 sum over k of BF16 x BF16 products (each product exact in FP32)
    Ab, Bb = _bf16(A), _bf16(B)
    D = np.zeros((len(A), len(B)), np.float32)
    for k in range(128):
        D = (D + np.outer(Ab[:, k], Bb[:, k]).astype(np.float32)).astype(np.float32)
    return 1.0 - 2.0 * D.astype(np.float64)


def _exact(A, B):
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    return (B64 * B64).sum(1)[None, :] - 2.0 * A64 @ B64.T


@pytest.mark.parametrize("kind", ["random", "near_duplicates", "duplicates", "sparse", "disjoint_support",
                                  "adversarial_duplicates", "adversarial_pairs"])
def test_estimate_within_value_dependent_bound(kind):
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    A = _descriptors(rng, 64, sparse=0.7 if kind == "sparse" else 0.0)
    if kind == "random" or kind == "sparse":
        B = _descriptors(rng, 96, sparse=0.7 if kind == "sparse" else 0.0)
    elif kind == "near_duplicates":
        B = np.abs(A + 0.01 * rng.standard_normal(A.shape)).astype(np.float32)
        B /= np.linalg.norm(B, axis=1, keepdims=True)
    elif kind == "duplicates":
        B = A.copy()
    elif kind.startswith("adversarial"):
        A = _adversarial(rng, 32)
        B = A.copy() if kind == "adversarial_duplicates" else _adversarial(rng, 48)
    else:
        # a and b with disjoint supports: a.b = 0, v = 1 (orthogonal pairs)
        A = np.zeros((64, 128), np.float32)
        B = np.zeros((64, 128), np.float32)
        A[:, :64] = np.abs(rng.standard_normal((64, 64)))
        B[:, 64:] = np.abs(rng.standard_normal((64, 64)))
        A /= np.linalg.norm(A, axis=1, keepdims=True)
        B /= np.linalg.norm(B, axis=1, keepdims=True)
    assert np.abs(np.linalg.norm(B.astype(np.float64), axis=1) - 1).max() <= EPS
    v = _exact(A, B)
    err = np.abs(_estimate(A, B) - v)
    assert (err <= delta(v)).all(), float((err - delta(v)).max())
    # the bound is not loose by orders of magnitude where it matters (near duplicates),
    # and the adversarial rounding comes within 3% of it
    if kind in ("near_duplicates", "duplicates"):
        diag = np.arange(len(A))
        assert err[diag, diag].max() > 1e-4
    if kind == "adversarial_duplicates":
        assert (err / delta(v)).max() > 0.97


def test_window_top_is_monotone_and_covers_the_listed_range():
    v = np.linspace(-1.0 - EPS, 1.0 + EPS, 200001)
    top = v + delta(v)
    assert (np.diff(top) > 0).all()            # v <= x  =>  v + delta(v) <= x + delta(x)
    assert abs(delta(-1.0) - (C + K * (2 + EPS))) < 1e-15 and abs(delta(1.0) - (C + K * EPS)) < 1e-15
