"""Pins of the oracle's parent frame and child prefix target (Sec. 3.4 bottom-up
generation with the prefix rule of Sec. 4.1).

Reading: a child's quantisation cube is [m_c, m_c + Q/s_c] (Q = 2^21 - 1); the parent
frame's minimum is the per-axis smallest child corner and its scale maps the largest
extent from there onto Q; a child is drawn with the shortest prefix reaching every child
surfel within one parent pixel step, 2^21/res parent units, i.e. (2^21/res) * (s_c/S)
child units, squared and truncated.  The cases below use dyadic corners and extents,
for which every double operation of the reading is exact, so the expected values are
closed forms; the random cases check what the frame is for (every child cube inside
[0, Q] of the parent, the largest touching Q).
"""
from fractions import Fraction

import numpy as np

import oracle

Q = 2**21 - 1


def _scale(extent):
    """Child scale whose cube side Q / s is exactly `extent` (a power of two)."""
    return Q / extent


def test_frame_closed_form_first_child_at_origin():
    fmin, s = oracle.parent_frame([[0, 0, 0], [1, 0, 0], [0.5, 2, 0]], [_scale(1), _scale(1), _scale(2)])
    assert fmin.tolist() == [0.0, 0.0, 0.0]
    assert s == Q / 4.0  # child 2 reaches y = 2 + 2 = 4


def test_frame_minimum_and_extent_from_later_children():
    # per-axis minima from children 1, 2 and 1; the extent (5.5 on z) from child 2
    mins = [[1, 1, 1], [0.25, 3, 0.5], [2, 0, 4]]
    fmin, s = oracle.parent_frame(mins, [_scale(1), _scale(0.5), _scale(2)])
    assert fmin.tolist() == [0.25, 0.0, 0.5]
    assert s == Q / 5.5


def test_frame_of_one_child_is_its_own():
    for m, e in [([0.125, -3.5, 7.0], 0.25), ([-1024.0, 0.0, 2.0], 512.0)]:
        fmin, s = oracle.parent_frame([m], [_scale(e)])
        assert fmin.tolist() == m and s == _scale(e)


def test_frame_holds_every_child_cube():
    g = np.random.default_rng(3)
    for _ in range(200):
        k = int(g.integers(1, 9))
        mins = g.uniform(-50, 50, size=(k, 3)).astype(np.float32)
        ext = np.exp(g.uniform(np.log(0.01), np.log(20), size=k))
        scales = Q / ext
        fmin, s = oracle.parent_frame(mins, scales)
        assert (fmin == mins.min(0)).all()
        lo = (mins.astype(np.float64) - fmin.astype(np.float64)) * s
        hi = (mins.astype(np.float64) + (Q / scales)[:, None] - fmin.astype(np.float64)) * s
        assert (lo >= 0).all()
        assert (hi <= Q * (1 + 1e-12)).all()
        assert abs(hi.max() - Q) <= Q * 1e-12


def test_child_target_closed_forms():
    # equal scales: one parent pixel = 2^21 / res child units
    assert oracle.child_target_r2(1000.0, 1000.0, 1024) == 2048**2
    assert oracle.child_target_r2(_scale(1), _scale(1), 4096) == 512**2
    # a child twice as finely quantised as the parent: twice as many child units
    assert oracle.child_target_r2(_scale(1), _scale(2), 1024) == 4096**2
    assert oracle.child_target_r2(_scale(2), _scale(1), 1024) == 1024**2
    # a non-dyadic ratio: the exact square truncated (no integer lies near it)
    want = int((Fraction(2**21, 1000) * Fraction(3, 2)) ** 2)
    assert oracle.child_target_r2(3.0, 2.0, 1000) == want == 9895604


def test_child_target_matches_the_parent_frame():
    """A parent over two unit cubes side by side at res 1024: its scale is Q / 2, so one
    parent pixel step is 4096 child units of a unit cube."""
    fmin, s = oracle.parent_frame([[0, 0, 0], [1, 0, 0]], [_scale(1), _scale(1)])
    assert s == Q / 2.0
    assert oracle.child_target_r2(_scale(1), s, 1024) == 4096**2
