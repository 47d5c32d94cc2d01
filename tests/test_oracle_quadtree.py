"""Pins for the contrast quadtree of the rendering branch (Sec. 3.5, Eq. 10, Algorithm 1).

Contrast is checked against closed forms (a region of two colours in proportions p, 1 - p has per-channel mean squared
deviation p (1 - p) (a - b)^2, in byte units); the subdivision against hand-counted trees and invariants that any
correct quadtree satisfies (its leaves tile the image; a threshold below zero splits to single pixels, one above the
largest possible contrast keeps the root)."""
import numpy as np
import pytest

import oracle

LUMA = np.array([0.2989, 0.5870, 0.1140])


def test_constant_region_has_zero_contrast():
    img = np.full((6, 9, 3), 77, np.uint8)
    assert oracle.qt_contrast(img, 0, 0, 9, 6) == 0.0


@pytest.mark.parametrize("p_num,a,b", [(1, (0, 0, 0), (255, 255, 255)), (3, (10, 200, 30), (250, 20, 90)),
                                       (5, (0, 128, 255), (0, 128, 0))])
def test_two_colour_region_matches_closed_form(p_num, a, b):
    # 8 x 8 region, the first p_num rows colour a, the rest b
    img = np.empty((8, 8, 3), np.uint8)
    img[:p_num] = a
    img[p_num:] = b
    p = p_num / 8
    var = p * (1 - p) * (np.array(a, float) - np.array(b, float)) ** 2
    assert abs(oracle.qt_contrast(img, 0, 0, 8, 8) - float(LUMA @ var)) < 1e-9


def test_black_white_halves_give_the_luma_sum_over_four():
    img = np.zeros((4, 4, 3), np.uint8)
    img[:, 2:] = 255
    assert abs(oracle.qt_contrast(img, 0, 0, 4, 4) - 0.25 * 255 ** 2 * LUMA.sum()) < 1e-9


def _tiles(leaves, w, h):
    cover = np.zeros((h, w), np.int32)
    for x, y, lw, lh in leaves:
        assert lw > 0 and lh > 0
        cover[y:y + lh, x:x + lw] += 1
    return cover


@pytest.mark.parametrize("w,h", [(13, 7), (16, 16), (5, 1)])
def test_negative_threshold_splits_to_single_pixels(w, h):
    img = np.random.default_rng(w * h).integers(0, 256, (h, w, 3), dtype=np.uint8)
    leaves = oracle.quadtree(img, threshold=-1.0, min_size=1)
    assert len(leaves) == w * h
    assert np.all(leaves[:, 2:] == 1)
    assert np.all(_tiles(leaves, w, h) == 1)


def test_threshold_above_the_maximum_keeps_the_root():
    img = np.random.default_rng(1).integers(0, 256, (48, 64, 3), dtype=np.uint8)
    leaves = oracle.quadtree(img, threshold=0.25 * 255 ** 2 * LUMA.sum() + 1e-6)
    assert leaves.tolist() == [[0, 0, 64, 48]]


def test_hand_counted_tree():
    """8 x 8 black image with a white 2 x 2 corner: root contrast (1/16)(15/16) 255^2 L (about 3809), L the luma sum.
    At 4000 the root stays; at 3000 it splits, its top-left 4 x 4 child (contrast (1/4)(3/4) 255^2 L) splits again into
    one white and three black 2 x 2 leaves, and the other three children are uniform: 7 leaves."""
    img = np.zeros((8, 8, 3), np.uint8)
    img[:2, :2] = 255
    L = LUMA.sum() * 255 ** 2
    assert abs(oracle.qt_contrast(img, 0, 0, 8, 8) - (1 / 16) * (15 / 16) * L) < 1e-9
    assert len(oracle.quadtree(img, 4000.0)) == 1
    leaves = oracle.quadtree(img, 3000.0)
    assert sorted(map(tuple, leaves.tolist())) == sorted([(0, 0, 2, 2), (2, 0, 2, 2), (0, 2, 2, 2), (2, 2, 2, 2),
                                                           (4, 0, 4, 4), (0, 4, 4, 4), (4, 4, 4, 4)])


def test_minimum_size_stops_the_split():
    img = np.random.default_rng(2).integers(0, 256, (16, 16, 3), dtype=np.uint8)
    leaves = oracle.quadtree(img, threshold=-1.0, min_size=4)
    assert len(leaves) == 16 and np.all(leaves[:, 2:] == 4)


def test_synthetic_frame_leaves_tile_and_respect_the_threshold():
    import synth
    wl = synth.rgbd()
    _, rgb, _ = synth.render_depth(wl, 0)
    leaves = oracle.quadtree(rgb, 0.1, 1)
    assert np.all(_tiles(leaves, wl.width, wl.height) == 1)
    # every leaf larger than one pixel is below the threshold
    big = leaves[(leaves[:, 2] > 1) | (leaves[:, 3] > 1)]
    for x, y, w, h in big[:: max(1, len(big) // 200)]:
        assert oracle.qt_contrast(rgb, x, y, w, h) <= 0.1
    assert 10000 < len(leaves) < wl.width * wl.height
