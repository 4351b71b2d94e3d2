"""Pins of the block-based FAST oracle (Sec. 3.1.1) against facts fixed by
the segment test itself: uniform-contrast circles score their contrast,
arcs of 9 contiguous pixels are corners and arcs of 8 are not (at every
rotation of the arc), straight edges have no corners, scores scale exactly
with a power-of-two contrast, swap polarity under negation and rotate with
the image; block selection picks each block's strongest suppressed corner."""
import numpy as np
import pytest

import oracle

CIRCLE = [(0, -3), (1, -3), (2, -2), (3, -1), (3, 0), (3, 1), (2, 2), (1, 3),
          (0, 3), (-1, 3), (-2, 2), (-3, 1), (-3, 0), (-3, -1), (-2, -2), (-1, -3)]


@pytest.fixture(scope="module")
def orc():
    oracle.build()
    return oracle


def blank(v=0.5, n=15):
    return np.full((n, n), v, np.float32)


@pytest.mark.parametrize("sign", [1, -1])
def test_uniform_circle_scores_its_contrast(orc, sign):
    img = blank(0.5 + sign * 0.25)
    img[7, 7] = 0.5
    s = orc.fast_score(img, t=0.05)
    assert s[7, 7] == np.float32(0.25)


def test_score_must_exceed_the_threshold(orc):
    """A pixel is a corner when its score exceeds t (the segment test's
    strict inequality): a uniform circle of contrast exactly t is not one."""
    img = blank(0.75)
    img[7, 7] = 0.5                             # contrast 0.25, exact in FP32
    assert orc.fast_score(img, t=0.25)[7, 7] == 0.0
    assert orc.fast_score(img, t=0.2499)[7, 7] == np.float32(0.25)


@pytest.mark.parametrize("start", range(16))
@pytest.mark.parametrize("length,corner", [(9, True), (8, False), (12, True)])
def test_arcs(orc, start, length, corner):
    img = blank()
    for j in range(length):
        dx, dy = CIRCLE[(start + j) % 16]
        img[7 + dy, 7 + dx] = 0.75
    s = orc.fast_score(img, t=0.05)
    assert s[7, 7] == (np.float32(0.25) if corner else 0.0)


def test_straight_edges_have_no_corners(orc):
    img = np.zeros((40, 40), np.float32)
    img[:, 20:] = 1.0
    assert not orc.fast_score(img, t=0.05).any()
    assert not orc.fast_score(img.T.copy(), t=0.05).any()


def test_square_corners(orc):
    img = np.zeros((40, 40), np.float32)
    img[10:30, 10:30] = 1.0
    s = orc.fast_score(img, t=0.05)
    ys, xs = np.nonzero(s)
    # corner responses cluster at the four corners of the square only
    for y, x in zip(ys, xs):
        assert min(abs(y - 10), abs(y - 29)) <= 2 and min(abs(x - 10), abs(x - 29)) <= 2
    pts, sc = orc.fast_blocks(img, 0.05, 2, 2, 3)
    for (x, y), (cx, cy) in zip(pts, [(10, 10), (29, 10), (10, 29), (29, 29)]):   # block order: (0,0),(0,1),(1,0),(1,1)
        assert abs(x - cx) <= 3 and abs(y - cy) <= 3


def test_scale_negation_rotation(orc):
    rng = np.random.default_rng(3)
    img = rng.random((48, 52)).astype(np.float32)
    s = orc.fast_score(img, t=0.05)
    assert np.array_equal(orc.fast_score(2 * img, t=0.1), 2 * s)        # exact: power-of-two scaling
    assert np.array_equal(orc.fast_score(-img, t=0.05), s)             # bright <-> dark
    r = np.rot90(img).copy()
    assert np.array_equal(orc.fast_score(r, t=0.05), np.rot90(s))      # the circle maps onto itself


def test_blocks_pick_the_strongest(orc):
    img = blank(0.5, 64)
    # a centre 0.1 below the background inside a ring 0.5 + c: the centre
    # scores c + 0.1, any ring pixel at most c
    def spot(x, y, c):
        for dx, dy in CIRCLE:
            img[y + dy, x + dx] = 0.5 + c
        img[y, x] = 0.4
    spot(10, 12, 0.2); spot(20, 20, 0.3)      # block (0, 0): the 0.3 one
    spot(45, 10, 0.1)                         # block (0, 1)
    spot(12, 50, 0.25); spot(22, 40, 0.25)    # block (1, 0): equal scores -> smaller y
    pts, sc = orc.fast_blocks(img, 0.05, 2, 2, 3)
    assert tuple(pts[0]) == (20, 20) and sc[0] == np.float32(0.8) - np.float32(0.4)
    assert tuple(pts[1]) == (45, 10)
    assert tuple(pts[2]) == (22, 40)
    assert tuple(pts[3]) == (-1, -1) and sc[3] == 0


def test_suppression_tie_keeps_the_first(orc):
    s_img = blank(0.5, 30)
    # a dark two-pixel blob: each pixel sees a uniform circle, so both score
    # exactly 0.2 and would both be local maxima without the tie rule
    s_img[14, 12] = s_img[14, 13] = 0.3
    s = orc.fast_score(s_img, t=0.05)
    assert s[14, 12] == s[14, 13] == np.float32(0.5) - np.float32(0.3)
    assert np.count_nonzero(s) == 2
    pts, sc = orc.fast_blocks(s_img, 0.05, 1, 1, 3)
    assert tuple(pts[0]) == (12, 14)
    # the same tie across a block boundary (columns [0, 15) | [15, 30)): the
    # second pixel is suppressed, so the right block has no corner at all
    b_img = blank(0.5, 30)
    b_img[14, 14] = b_img[14, 15] = 0.3
    pts, sc = orc.fast_blocks(b_img, 0.05, 1, 2, 3)
    assert tuple(pts[0]) == (14, 14) and tuple(pts[1]) == (-1, -1) and sc[1] == 0


def test_flat_image_and_margin(orc):
    pts, sc = orc.fast_blocks(blank(0.3, 50), 0.05, 3, 3, 3)
    assert (pts == -1).all() and (sc == 0).all()
    img = np.zeros((40, 40), np.float32)
    img[2:8, 2:8] = 1.0                         # corners within 10 px of the border
    pts, _ = orc.fast_blocks(img, 0.05, 1, 1, 10)
    assert tuple(pts[0]) == (-1, -1)
    with pytest.raises(ValueError):
        orc.fast_blocks(img, 0.05, 0, 1, 3)


def test_blocks_partition_a_non_square_image(orc):
    """Block rows are [by H / grid_y, (by + 1) H / grid_y) and columns
    [bx W / grid_x, ...) (Sec. 3.1.1's partition): on a 30 x 60 image in
    3 x 2 blocks a single corner at (x, y) = (45, 25) is block 2 * 2 + 1."""
    img = np.full((30, 60), 0.5, np.float32)
    img[25, 45] = 0.25                          # a dark spot: every circle pixel is brighter
    pts, sc = orc.fast_blocks(img, 0.05, 3, 2, 3)
    assert tuple(pts[5]) == (45, 25) and sc[5] == np.float32(0.25)
    assert all(tuple(p) == (-1, -1) for k, p in enumerate(pts) if k != 5)
