"""lp_mosaic_plan (host code of liblp, no GPU) against the oracle's Sec. 4
rounds on random graphs of random homographies."""
import numpy as np
import pytest

import oracle
from paper_2405_08578_gb300 import lp


def _random_case(rng, n, p_edge):
    place = []
    for _ in range(n):
        H = np.eye(3)
        H[:2, :2] += 0.05 * rng.standard_normal((2, 2))
        H[:2, 2] = rng.uniform(-400, 400, 2)
        H[2, :2] = rng.uniform(-2e-5, 2e-5, 2)
        place.append(H)
    pairs, HM, valid = [], [], []
    for i in range(n):
        for j in range(i + 1, n):
            pairs.append((i, j))
            HM.append(np.linalg.inv(place[j]) @ place[i])
            valid.append(int(rng.uniform() < p_edge))
    sizes = [(int(rng.integers(50, 300)), int(rng.integers(50, 300))) for _ in range(n)]
    return pairs, np.array(HM), np.array(valid, np.uint8), sizes


@pytest.mark.parametrize("n,p_edge,seed", [(1, 0.0, 0), (2, 1.0, 1), (9, 0.3, 2), (9, 0.15, 3), (16, 0.2, 4),
                                           (30, 0.1, 5), (64, 0.05, 6)])
def test_plan_equals_oracle(n, p_edge, seed):
    rng = np.random.default_rng(seed)
    pairs, HM, valid, sizes = _random_case(rng, n, p_edge)
    if not pairs:
        pairs, HM, valid = np.zeros((0, 2), np.int32), np.zeros((0, 3, 3)), np.zeros(0, np.uint8)
    got = lp.lp_mosaic_plan(n, pairs, HM, valid, sizes)
    want = oracle.mosaic_plan(n, pairs, HM, valid, sizes)
    assert np.array_equal(got["round"], want["round"]) and np.array_equal(got["ref"], want["ref"])
    assert got["canvas"] == want["canvas"]
    assert np.allclose(got["G"], want["G"], rtol=1e-9, atol=1e-7)


def test_plan_rejects_bad_input():
    with pytest.raises(lp.LpError):
        lp.lp_mosaic_plan(65, [], np.zeros((0, 9)), [], [(10, 10)] * 65)
    with pytest.raises(lp.LpError):
        lp.lp_mosaic_plan(2, [(0, 2)], np.eye(3)[None], [1], [(10, 10)] * 2)
