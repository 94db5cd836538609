"""Pins for the oracle's Sec. 4 mosaic: round structure on hand-built graphs,
placements composed from exact homographies, and the render's closed forms."""
import numpy as np

import oracle


def T(tx, ty):
    return np.array([[1.0, 0, tx], [0, 1, ty], [0, 0, 1]])


def _hm_for(n, placement, valid_pairs):
    """Pairs i<j with H mapping i pixels to j pixels from known placements
    (image pixel -> world): H_ij = P_j^-1 P_i."""
    pairs, HM, valid = [], [], []
    for i in range(n):
        for j in range(i + 1, n):
            pairs.append((i, j))
            HM.append(np.linalg.inv(placement[j]) @ placement[i])
            valid.append(1 if (i, j) in valid_pairs else 0)
    return pairs, np.array(HM), np.array(valid, np.uint8)


def test_star_graph_is_one_round():
    n = 5
    place = [T(10 * k, -5 * k) for k in range(n)]
    pairs, HM, valid = _hm_for(n, place, {(2, 0), (0, 2), (1, 2), (2, 3), (2, 4)})
    plan = oracle.mosaic_plan(n, pairs, HM, valid, [(40, 50)] * n)
    assert plan["round"].tolist() == [0] * n and set(plan["ref"].tolist()) == {2}
    # placements relative to image 2, shifted into the canvas: all differences match the truth
    for k in range(n):
        want = np.linalg.inv(place[2]) @ place[k]          # image k pixels -> image 2 pixels
        assert np.allclose(np.linalg.inv(plan["G"][2]) @ plan["G"][k], want, atol=1e-9)


def test_chain_graph_rounds_and_references():
    # 0-1-2-3-4-5 chain plus 2-6: degrees 1,2,3,2,2,1,1 -> round 0 around 2 (1, 3, 6),
    # then the unmatched image of largest degree linked to a placed one: 4 (deg 2), then 0, then 5
    n = 7
    place = [T(7 * k, 3 * k) for k in range(n)]
    edges = {(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (2, 6)}
    pairs, HM, valid = _hm_for(n, place, edges)
    plan = oracle.mosaic_plan(n, pairs, HM, valid, [(30, 30)] * n)
    assert plan["round"].tolist() == [2, 0, 0, 0, 1, 1, 0]
    assert plan["ref"].tolist() == [0, 2, 2, 2, 4, 4, 2]
    for k in range(n):
        assert np.allclose(np.linalg.inv(plan["G"][2]) @ plan["G"][k], np.linalg.inv(place[2]) @ place[k], atol=1e-9)


def test_degree_tie_takes_the_lowest_index():
    # a 4-cycle: every image has degree 2, so image 0 is the first reference and
    # places 1 and 3; image 2 follows in round 1 as its own reference
    n = 4
    place = [T(9 * k, 4 * k) for k in range(n)]
    pairs, HM, valid = _hm_for(n, place, {(0, 1), (1, 2), (2, 3), (0, 3)})
    plan = oracle.mosaic_plan(n, pairs, HM, valid, [(30, 30)] * n)
    assert plan["round"].tolist() == [0, 0, 1, 0]
    assert plan["ref"].tolist() == [0, 0, 2, 0]


def test_disconnected_image_stays_unplaced_and_canvas_box():
    n = 3
    place = [T(0, 0), T(25, 10), T(500, 500)]
    pairs, HM, valid = _hm_for(n, place, {(0, 1)})
    plan = oracle.mosaic_plan(n, pairs, HM, valid, [(20, 30), (20, 30), (20, 30)])
    assert plan["round"].tolist() == [0, 0, -1] and not plan["G"][2].any()
    # image 0 at the origin, image 1 shifted by (25, 10): box 55 x 30
    assert plan["canvas"] == (30, 55)
    assert np.allclose(plan["G"][0], np.eye(3)) and np.allclose(plan["G"][1], T(25, 10))


def test_render_identity_and_integer_overlap():
    rng = np.random.default_rng(3)
    a = rng.integers(0, 256, (12, 17), dtype=np.uint8)
    canvas, cover = oracle.mosaic_render([a], [np.eye(3)], [0], (12, 17))
    assert np.array_equal(canvas, a) and (cover == 1).all()
    b = rng.integers(0, 256, (12, 17), dtype=np.uint8)
    canvas, cover = oracle.mosaic_render([a, b], [np.eye(3), T(5, 2)], [0, 0], (14, 22))
    want_overlap = np.floor((a[2:, 5:].astype(np.float64) + b[:10, :12]) / 2 + 0.5)
    assert np.array_equal(canvas[2:12, 5:17], want_overlap.astype(np.uint8))
    assert (cover[2:12, 5:17] == 2).all() and cover[0, 0] == 1 and cover[13, 0] == 0 and canvas[13, 0] == 0
    assert np.array_equal(canvas[:2, :17], a[:2]) and np.array_equal(canvas[12:, 5:], b[10:])


def test_render_half_pixel_shift_is_the_mean_of_neighbours():
    a = np.arange(40, dtype=np.uint8).reshape(5, 8) * 3
    canvas, cover = oracle.mosaic_render([a], [T(0.5, 0)], [0], (5, 9))
    # canvas x = u + 0.5: the sample at u = x - 0.5 is the mean of columns x-1 and x
    want = np.floor((a[:, :-1].astype(np.float64) + a[:, 1:]) / 2 + 0.5)
    assert np.array_equal(canvas[:, 1:8], want.astype(np.uint8))
    assert (cover[:, 0] == 0).all() and (cover[:, 8] == 0).all()
