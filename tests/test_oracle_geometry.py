"""Pins for the oracle's segment -> cell sets (block allocation, Sec. 3.2; the LiDAR voxel walk, Sec. 3.1.1).

The oracle has two independent implementations (bounding-box test of every cell, ordered Amanatides-Woo walk); these
tests tie both to facts that do not come from either: closed-form cell counts, exact rational sample points of the
segment, hand-derived corner cases, and adjacency/monotonicity of the walk.
"""
import numpy as np
import pytest

import oracle

U = oracle.BLOCK_UNIT


def _set(cells):
    return {tuple(int(v) for v in c) for c in cells}


def test_axis_aligned_closed_form():
    # segment along +x from 0.25 U to 3.5 U at y = z = 0.5 U: cells 0..3
    cells = oracle.segment_cells([U // 4, U // 2, U // 2], [3 * U + U // 2, U // 2, U // 2], U)
    assert _set(cells) == {(0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0)}
    # along -y, ending exactly on a boundary: the end point belongs to the upper cell [c U, (c+1) U)
    cells = oracle.segment_cells([U // 2, 2 * U + 5, U // 2], [U // 2, U, U // 2], U, mode="walk")
    assert [tuple(c) for c in cells] == [(0, 2, 0), (0, 1, 0)]


def test_corner_crossings():
    h = U // 2
    # both axes upward through the corner (U, U): only the diagonal cells
    assert _set(oracle.segment_cells([h, h, h], [U + h, U + h, h], U)) == {(0, 0, 0), (1, 1, 0)}
    # both downward through the same corner: the corner point still lies in cell (1, 1)
    assert _set(oracle.segment_cells([U + h, U + h, h], [h, h, h], U)) == {(1, 1, 0), (0, 0, 0)}
    # x up, y down through (U, U): (0,1) -> corner in (1,1) -> (1,0)
    assert _set(oracle.segment_cells([h, U + h, h], [U + h, h, h], U)) == {(0, 1, 0), (1, 1, 0), (1, 0, 0)}
    walk = [tuple(c) for c in oracle.segment_cells([h, U + h, h], [U + h, h, h], U, mode="walk")]
    assert walk == [(0, 1, 0), (1, 1, 0), (1, 0, 0)]
    # all three axes up through (U, U, U)
    assert _set(oracle.segment_cells([h, h, h], [U + h, U + h, U + h], U)) == {(0, 0, 0), (1, 1, 1)}
    # a segment that only touches a face plane at its start: A on x = U moving down starts in cell 1
    assert _set(oracle.segment_cells([U, h, h], [U - 10, h, h], U)) == {(1, 0, 0), (0, 0, 0)}
    # degenerate zero-length segment
    assert _set(oracle.segment_cells([5, 7, -3], [5, 7, -3], U)) == {(0, 0, -1)}


def _rand_segments(rng, n, span, quantum=1):
    A = rng.integers(-span, span, (n, 3)) * quantum
    B = A + rng.integers(-span, span, (n, 3)) * quantum
    return A, B


def test_walk_equals_bruteforce_random():
    rng = np.random.default_rng(1234)
    # generic segments, and segments on a coarse lattice (quarter cells) where exact ties are frequent
    for quantum, span in ((1, 4 * U), (U // 4, 16)):
        A, B = _rand_segments(rng, 400, span, quantum)
        for a, b in zip(A, B):
            bf = oracle.segment_cells(a, b, U, mode="bruteforce")
            wk = oracle.segment_cells(a, b, U, mode="walk")
            assert _set(bf) == _set(wk)
            assert len(wk) == len(_set(wk))           # no cell visited twice
            steps = np.diff(wk, axis=0)
            assert np.all(np.abs(steps) <= 1)          # each step moves to a neighbour (face/edge/corner)
            d = np.sign(b - a)
            assert np.all(steps * d >= 0)              # monotone along the segment direction
            assert tuple(wk[0]) == tuple(np.floor_divide(a, U)) and tuple(wk[-1]) == tuple(np.floor_divide(b, U))


def test_generic_cell_count_closed_form():
    # without coinciding crossings a segment meets 1 + (number of boundary planes it crosses) cells
    rng = np.random.default_rng(7)
    A, B = _rand_segments(rng, 300, 5 * U)
    checked = 0
    for a, b in zip(A, B):
        ca, cb = np.floor_divide(a, U), np.floor_divide(b, U)
        cells = oracle.segment_cells(a, b, U)
        expected = 1 + int(np.abs(cb - ca).sum())
        if len(cells) != expected:
            # only allowed when two crossings coincide exactly; verify that with exact integer arithmetic
            d = b - a
            params = []
            for i in range(3):
                lo, hi = sorted((ca[i], cb[i]))
                for k in range(lo + 1, hi + 1):
                    params.append(((k * U - a[i]), d[i]))
            from fractions import Fraction
            fr = [Fraction(int(p), int(q)) for p, q in params]
            assert len(set(fr)) < len(fr)
        else:
            checked += 1
    assert checked > 250


def test_sample_points_are_covered():
    # exact rational points A + (j/64)(B - A) lie in cells of the set; cell = floor((64A + j(B-A)) / (64U))
    rng = np.random.default_rng(99)
    A, B = _rand_segments(rng, 200, 3 * U)
    for a, b in zip(A, B):
        s = _set(oracle.segment_cells(a, b, U))
        for j in range(65):
            p64 = 64 * a + j * (b - a)
            c = tuple(int(v) for v in np.floor_divide(p64, 64 * U))
            assert c in s


def test_voxel_unit_walk_matches_bruteforce():
    rng = np.random.default_rng(5)
    V = oracle.VOXEL_UNIT
    A, B = _rand_segments(rng, 200, 24 * V)
    for a, b in zip(A, B):
        assert _set(oracle.segment_cells(a, b, V, "walk")) == _set(oracle.segment_cells(a, b, V, "bruteforce"))


@pytest.mark.parametrize("x", [0.0, 1e-3, -0.3333, 0.1 + 2 ** -12, 65504.0, 2 ** -14, 3 * 2 ** -25, 1.0 + 2 ** -11])
def test_half_rounding_is_ieee(x):
    assert oracle.half_round(x) == float(np.float16(np.float32(x)))
