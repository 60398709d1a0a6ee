"""Pins for the oracle's splat sampling: a parent node sampled from its children's surfels
drawn as oriented discs (Sec. 3.4's bottom-up generation, with Sec. 4.2's discs).

The checks come from geometry, not from the oracle's own formulas:
* a disc facing the camera covers exactly the pixels whose centres lie in its circle (a
  lattice-point count) and emits the pixel-centre points of its plane;
* a tilted disc covers the pixels whose rays hit the plane inside the disc, recomputed here
  with exact rational ray-plane intersections;
* the nearer disc wins a pixel, an edge-on disc is invisible, equal discs go to the lower
  index, and the frame change and radius scaling have closed forms for power-of-two scales.
"""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle

Q = 2**21 - 1
UP = np.array([[0, 0, 1]], np.int8)
DOWN = np.array([[0, 0, -1]], np.int8)


def _set(c, n, r2, rgb=None, bmin=(0.0, 0.0, 0.0), scale=1.0):
    c = np.atleast_2d(np.asarray(c, np.int64))
    return dict(key=oracle.pack(c), nrm=np.atleast_2d(np.asarray(n, np.int16)),
                rgb=None if rgb is None else np.atleast_2d(np.asarray(rgb, np.uint8)),
                bbox_min=np.asarray(bmin, np.float32), scale=scale, r2=r2)


def _splat(sets, dirs, res, fmin=(0.0, 0.0, 0.0), fscale=1.0):
    return oracle.sample_splats(sets, np.asarray(fmin, np.float32), fscale, dirs, res)


def _pixel_point(px, py, h):
    """Point of the +z view's pixel (px, py) centre in the quantised frame: the view's u
    axis is +y and its v axis is -x (the frame of Sec. 3.1's reading)."""
    return Q - (2 * py + 1) * h // 2, (2 * px + 1) * h // 2


@pytest.mark.parametrize("k", [0, 1, 2, 3, 5, 7])
def test_facing_disc_covers_its_lattice_circle(k):
    res, h = 64, 2**21 // 64
    a, b, cz = 20, 33, 777_777
    cx, cy = _pixel_point(a, b, h)
    r2 = k * k * h * h + h * h // 2  # between the k^2 and k^2 + 1 lattice shells
    out = _splat([_set([cx, cy, cz], [0, 0, 32767], r2)], UP, res)
    want = {(px, py) for px in range(res) for py in range(res) if (px - a) ** 2 + (py - b) ** 2 <= k * k}
    pts = oracle.unpack(out["key"])
    got = set()
    for x, y, z in pts:
        assert z == cz
        px, rem = divmod(int(y) - h // 2, h)
        assert rem == 0
        py = (Q - int(x) - h // 2) // h
        assert _pixel_point(px, py, h) == (x, y)
        got.add((px, py))
    assert got == want
    assert np.all(out["nrm"] == [0, 0, 32767])


def _exact_cover(c, n, r2, res, px, py):
    """Rational ray-plane hit of the +z view's pixel ray; covered iff within the disc."""
    h = F(2**21, res)
    x, y = F(Q) - (py + F(1, 2)) * h, (px + F(1, 2)) * h
    # plane n.(p - c) = 0 solved for z
    z = F(c[2]) - (n[0] * (x - c[0]) + n[1] * (y - c[1])) / F(n[2])
    d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
    return d2 <= r2, z


@pytest.mark.parametrize("n", [[0, -16000, 28000], [9000, 4000, 31000], [-20000, 20000, 12000]])
def test_tilted_disc_is_the_exact_ellipse(n):
    res, h = 32, 2**21 // 32
    c = [Q // 2 + 12345, Q // 2 - 54321, Q // 2 + 999]
    r2 = (7 * h) ** 2 + 17
    out = _splat([_set(c, n, r2)], UP, res)
    pts = oracle.unpack(out["key"])
    got = {}
    for x, y, z in pts:
        px = int(F(int(y)) / F(2**21, res))
        py = int((Q - F(int(x))) / F(2**21, res))
        got[(px, py)] = int(z)
    want = {}
    for px in range(res):
        for py in range(res):
            ok, z = _exact_cover(c, n, r2, res, px, py)
            if ok:
                want[(px, py)] = int(np.floor(float(z))) if z.denominator != 1 else int(z)
    assert set(got) == set(want)
    for k in want:
        assert got[k] == min(max(want[k], 0), Q), k
    # area: pi r^2 |n_z| / |n| in pixels, within the boundary pixels
    area = np.pi * r2 / h**2 * abs(n[2]) / np.linalg.norm(n)
    assert abs(len(want) - area) < 2 * np.pi * np.sqrt(r2) / h + 4


def test_nearer_disc_wins_each_view():
    res, h = 32, 2**21 // 32
    cx, cy = _pixel_point(10, 12, h)
    lo = _set([cx, cy, 1000], [0, 0, 32767], (4 * h) ** 2, rgb=[10, 0, 0])
    hi = _set([cx + h, cy, 900_000], [0, 0, 32767], (4 * h) ** 2, rgb=[20, 0, 0])
    for dirs, zwin in ((UP, 900_000), (DOWN, 1000)):
        out = _splat([lo, hi], dirs, res)
        pts = oracle.unpack(out["key"])
        # where the discs overlap the camera-side one wins; elsewhere each shows itself
        r2 = (4 * h) ** 2
        nboth = 0
        for x, y, z in pts:
            x, y = int(x), int(y)
            in_lo = (x - cx) ** 2 + (y - cy) ** 2 <= r2
            in_hi = (x - cx - h) ** 2 + (y - cy) ** 2 <= r2
            assert in_lo or in_hi
            if in_lo and in_hi:
                nboth += 1
                assert z == zwin
            else:
                assert z == (1000 if in_lo else 900_000)
        assert nboth > 10
        # normals face the camera
        assert np.all(out["nrm"][:, 2] * dirs[0, 2] > 0)


def test_edge_on_disc_is_invisible():
    res, h = 32, 2**21 // 32
    s = _set([Q // 2, Q // 2, Q // 2], [32767, 0, 0], (5 * h) ** 2)
    assert len(_splat([s], UP, res)["key"]) == 0
    assert len(_splat([s], np.array([[1, 0, 0]], np.int8), res)["key"]) > 0


def test_equal_discs_go_to_the_lower_index():
    res, h = 16, 2**21 // 16
    c = [Q // 3, Q // 3, Q // 3]
    a = _set([c, c], [[0, 0, 32767], [0, 0, 32767]], (3 * h) ** 2, rgb=[[1, 2, 3], [4, 5, 6]])
    out = _splat([a], UP, res)
    assert len(out["key"]) > 0 and np.all(out["rgb"] == [1, 2, 3])
    b = _set([c], [0, 0, 32767], (3 * h) ** 2, rgb=[7, 8, 9])
    out2 = _splat([b, _set([c], [0, 0, 32767], (3 * h) ** 2, rgb=[1, 1, 1])], UP, res)
    assert np.all(out2["rgb"] == [7, 8, 9])


def test_frame_change_and_radius_scaling_closed_form():
    """A set in a child frame (bbox_min, s_c) lands in the parent frame (fmin, s_p) at
    (bmin - fmin) s_p + q s_p / s_c; with power-of-two scales this is exact, and the disc
    radius scales by s_p / s_c."""
    res, h = 32, 2**21 // 32
    s_c, s_p = 2.0**20, 2.0**19
    bmin, fmin = (1.25, 2.0, 3.5), (0.25, 1.0, 2.5)
    q = np.array([400_000, 600_000, 123_456])
    child = _set(q, [0, 0, 32767], 4 * (3 * h) ** 2 + 4, bmin=bmin, scale=s_c)
    c = [int((b - f) * s_p + qq * s_p / s_c) for b, f, qq in zip(bmin, fmin, q)]
    direct = _set(c, [0, 0, 32767], (3 * h) ** 2 + 1, bmin=fmin, scale=s_p)  # already in the parent frame
    a = _splat([child], UP, res, fmin=fmin, fscale=s_p)
    b = _splat([direct], UP, res, fmin=fmin, fscale=s_p)
    assert len(a["key"]) > 0
    assert np.array_equal(a["key"], b["key"]) and np.array_equal(a["src"], b["src"])
    assert np.all(oracle.unpack(a["key"])[:, 2] == c[2])


def test_views_merge_keeping_the_first_emission():
    """The -z view's pixel grid is the +z grid mirrored (its u axis is -y), so the two views
    emit different points, each with its own emission index and camera-facing normal; a
    direction given twice emits the same points twice and the first emission is kept."""
    res, h = 16, 2**21 // 16
    cx, cy = _pixel_point(7, 8, h)
    s = _set([cx, cy, 5000], [0, 0, 32767], (2 * h) ** 2 + h)
    up = _splat([s], UP, res)
    down = _splat([s], DOWN, res)
    both = _splat([s], np.concatenate([UP, DOWN]), res)
    assert len(up["key"]) == 13 and not set(up["key"].tolist()) & set(down["key"].tolist())
    assert set(both["key"].tolist()) == set(up["key"].tolist()) | set(down["key"].tolist())
    ui = {k: i for i, k in enumerate(up["key"].tolist())}
    di = {k: i for i, k in enumerate(down["key"].tolist())}
    for i, k in enumerate(both["key"].tolist()):
        if k in ui:
            assert both["src"][i] == up["src"][ui[k]] and both["nrm"][i, 2] > 0
        else:
            assert both["src"][i] == down["src"][di[k]] + res * res and both["nrm"][i, 2] < 0
    twice = _splat([s], np.concatenate([UP, UP]), res)
    assert np.array_equal(twice["key"], up["key"]) and np.array_equal(twice["src"], up["src"])


def test_rejects_non_axis_directions():
    s = _set([Q // 2] * 3, [0, 0, 32767], 100)
    with pytest.raises(ValueError):
        _splat([s], np.array([[1, 1, 1]], np.int8), 8)


def test_crossing_discs_show_the_higher_hit_per_pixel():
    """Two tilted discs through the same region cross; from +z each pixel shows the disc
    whose ray hit is higher (exact rational hits), from -z the lower one."""
    res, h = 32, 2**21 // 32
    c1 = [Q // 2, Q // 2, Q // 2]
    c2 = [Q // 2 + 3 * h, Q // 2 - 2 * h, Q // 2 + 5000]
    n1, n2 = [0, -15000, 29000], [12000, 9000, 29000]
    r2 = (6 * h) ** 2
    out = _splat([_set(c1, n1, r2, rgb=[1, 0, 0]), _set(c2, n2, r2, rgb=[2, 0, 0])], UP, res)
    pts = oracle.unpack(out["key"])
    seen = 0
    for (x, y, z), col in zip(pts, out["rgb"][:, 0]):
        px = int(F(int(y)) / F(2**21, res))
        py = int((Q - F(int(x))) / F(2**21, res))
        a, za = _exact_cover(c1, n1, r2, res, px, py)
        b, zb = _exact_cover(c2, n2, r2, res, px, py)
        assert a or b
        if a and b and za != zb:
            seen += 1
            assert col == (1 if za > zb else 2), (px, py)
    assert seen > 20
