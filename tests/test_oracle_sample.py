"""Pins for the oracle's sampling half: quantiser, integer rasteriser, resolve, dedup.

Closed forms (pixel-aligned rectangles, whole cube faces, planes), watertightness
of meshes (every pixel centre covered exactly once), depth order, and a dedup
check rebuilt from single-direction runs.  Sec. 3.1 of the paper defines the
step: render the node from several directions and emit one surfel per covered
pixel with position, normal and colour.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1904_08225_gb300 import workloads as W

Q = (1 << 21) - 1
RES = 64  # with res=64 and an axis view, screen X = round(u / 128): u = a*2^15 is pixel boundary a


def _mesh_q(verts, tris):
    return np.asarray(verts, np.int32), np.asarray(tris, np.uint32)


def _ybound(a):  # u = y for the +z view
    return a * (1 << 15)


def _xbound(b):  # v = -x for the +z view: Y = (Q - x) / 128
    return Q - b * (1 << 15)


def test_frame_is_orthogonal_integer():
    for d in list(W.AXIS_DIRS) + list(W.CORNER_DIRS) + [np.array([1, 1, 0]), np.array([0, -1, 1])]:
        u, v = oracle.frame(d)
        d = np.asarray(d, np.int64)
        assert u @ d == 0 and v @ d == 0 and u @ v == 0
        assert np.abs(u).sum() > 0 and np.abs(v).sum() > 0
    u, v = oracle.frame([0, 0, 1])
    assert u.tolist() == [0, 1, 0] and v.tolist() == [-1, 0, 0]


def test_quantiser_closed_forms():
    xyz = np.array([[0, 0, 0], [2, 1, 1], [1, 0.5, 0.25]], np.float32)
    q, mn, s = oracle.quantise(xyz)
    assert s == Q / 2.0 and mn.tolist() == [0, 0, 0]
    assert q[0].tolist() == [0, 0, 0]
    assert q[1].tolist() == [Q, Q // 2, Q // 2]      # isotropic: y extent is half of x
    assert q[2].tolist() == [Q // 2, Q // 4, Q // 8]
    with pytest.raises(ValueError):
        oracle.quantise(np.array([[0, 0, 0], [np.nan, 1, 1]], np.float32))
    with pytest.raises(ValueError):
        oracle.quantise(np.array([[1, 1, 1], [1, 1, 1]], np.float32))
    with pytest.raises(ValueError):
        oracle.quantise(np.array([[0, 0, 0], [np.inf, 1, 1]], np.float32))


def test_raster_aligned_rectangle():
    """A quad with pixel-aligned edges covers exactly the pixels whose centres it contains."""
    a0, a1, b0, b1 = 5, 40, 12, 33
    z = 1000
    v = [[_xbound(b0), _ybound(a0), z], [_xbound(b0), _ybound(a1), z],
         [_xbound(b1), _ybound(a1), z], [_xbound(b1), _ybound(a0), z]]
    q, t = _mesh_q(v, [[0, 1, 2], [0, 2, 3]])
    depth, nf, cnt = oracle.raster_dir(q, t, [0, 0, 1], RES, counts=True)
    want = np.zeros((RES, RES), np.uint32)
    want[b0:b1, a0:a1] = 1  # rows = py (from v), cols = px (from u)
    assert np.array_equal(cnt, want)
    assert nf == (a1 - a0) * (b1 - b0)
    # depth of a plane z = const seen from +z: w = -z + Q
    assert np.all((depth[want == 1] >> np.uint64(32)) == Q - z)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_raster_watertight_jittered_grid(seed):
    """An n x n grid mesh with jittered interior vertices and random winding covers every
    pixel of its (aligned) outline exactly once: no holes, no double coverage."""
    g = np.random.default_rng(seed)
    a0, a1, b0, b1 = 3, 61, 2, 59
    n = 9
    ys = np.linspace(_ybound(a0), _ybound(a1), n + 1)
    xs = np.linspace(_xbound(b0), _xbound(b1), n + 1)
    verts = []
    for i in range(n + 1):
        for j in range(n + 1):
            x, y = xs[i], ys[j]
            if 0 < i < n:
                x += g.uniform(-0.3, 0.3) * (xs[1] - xs[0])
            if 0 < j < n:
                y += g.uniform(-0.3, 0.3) * (ys[1] - ys[0])
            verts.append([int(x), int(y), int(g.integers(0, Q))])
    tris = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = i * (n + 1) + j, (i + 1) * (n + 1) + j, (i + 1) * (n + 1) + j + 1, i * (n + 1) + j + 1
            for tri in ([a, b, c], [a, c, d]) if g.random() < 0.5 else ([a, b, d], [b, c, d]):
                tris.append(tri if g.random() < 0.5 else tri[::-1])
    q, t = _mesh_q(verts, tris)
    _, nf, cnt = oracle.raster_dir(q, t, [0, 0, 1], RES, counts=True)
    want = np.zeros((RES, RES), np.uint32)
    want[b0:b1, a0:a1] = 1
    assert np.array_equal(cnt, want)


def test_raster_fan_vertex_on_pixel_centre():
    """A triangle fan whose hub sits exactly on a pixel centre covers the hub pixel once."""
    a0, a1, b0, b1 = 10, 20, 30, 40
    hub = [Q - (256 * 35 + 128) * 128, (256 * 15 + 128) * 128, 0]
    ring = [[_xbound(b0), _ybound(a0)], [_xbound(b0), _ybound(15)], [_xbound(b0), _ybound(a1)],
            [_xbound(35), _ybound(a1)], [_xbound(b1), _ybound(a1)], [_xbound(b1), _ybound(15)],
            [_xbound(b1), _ybound(a0)], [_xbound(35), _ybound(a0)]]
    verts = [hub] + [[x, y, 0] for x, y in ring]
    tris = [[0, 1 + i, 1 + (i + 1) % 8] for i in range(8)]
    q, t = _mesh_q(verts, tris)
    _, _, cnt = oracle.raster_dir(q, t, [0, 0, 1], RES, counts=True)
    want = np.zeros((RES, RES), np.uint32)
    want[b0:b1, a0:a1] = 1
    assert np.array_equal(cnt, want)


def test_raster_nearer_quad_wins():
    """Two overlapping parallel quads seen from +z: the one with larger z (nearer) wins."""
    def quad(a0, a1, b0, b1, z):
        return [[_xbound(b0), _ybound(a0), z], [_xbound(b0), _ybound(a1), z],
                [_xbound(b1), _ybound(a1), z], [_xbound(b1), _ybound(a0), z]]
    v = quad(0, 40, 0, 40, 500) + quad(20, 60, 20, 60, 900)
    t = [[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]]
    q, t = _mesh_q(v, t)
    depth, _ = oracle.raster_dir(q, t, [0, 0, 1], RES)
    tid = (depth & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert set(np.unique(tid[20:40, 20:40]).tolist()) <= {2, 3}
    assert set(np.unique(tid[0:20, 0:20]).tolist()) <= {0, 1}
    # seen from -z the other quad is nearer
    depth2, _ = oracle.raster_dir(q, t, [0, 0, -1], RES)
    tid2 = (depth2 & np.uint64(0xFFFFFFFF)).astype(np.int64)
    covered = depth2 != np.uint64(2**64 - 1)
    assert covered.sum() == 40 * 40 * 2 - 20 * 20
    assert np.isin(tid2[covered], [0, 1, 2, 3]).all()
    assert (np.isin(tid2[covered], [0, 1])).sum() == 40 * 40


def test_cube_six_axis_views():
    """Unit cube: every axis view covers all res^2 pixels; the +z view sees z = Q with
    normal (0, 0, 32767); after merging, each position appears once."""
    m = W.cube(n=2)
    q, mn, s = oracle.quantise(m.xyz)
    res = 32
    for d in W.AXIS_DIRS:
        depth, _ = oracle.raster_dir(q, m.tri, d, res)
        assert (depth != np.uint64(2**64 - 1)).all()
    sv = oracle.sample_visible(q, m.tri, None, np.array([[0, 0, 1]], np.int8), res)
    P = oracle.unpack(sv["key"])
    assert len(P) == res * res and (P[:, 2] == Q).all()
    assert (sv["nrm"] == np.array([0, 0, 32767])).all()
    sv = oracle.sample_visible(q, m.tri, None, np.array([[0, 0, -1]], np.int8), res)
    assert (oracle.unpack(sv["key"])[:, 2] == 0).all()
    assert (sv["nrm"] == np.array([0, 0, -32767])).all()


def _morton_py(p):
    x, y, z = (int(v) for v in p)
    m = 0
    for i in range(21):
        m |= ((x >> i) & 1) << (3 * i) | ((y >> i) & 1) << (3 * i + 1) | ((z >> i) & 1) << (3 * i + 2)
    return m


def test_dedup_matches_single_direction_union():
    """Multi-direction result = union of single-direction results, keeping the smallest
    emission index e = dir*res^2 + py*res + px per position, ordered by Morton code."""
    m = W.torus(nu=48, nv=24, seed=3)
    q, mn, s = oracle.quantise(m.xyz)
    res = 48
    dirs = np.concatenate([W.AXIS_DIRS, W.DIAG_DIRS])
    best = {}
    for di, d in enumerate(dirs):
        sv = oracle.sample_visible(q, m.tri, m.rgb, d[None], res)
        for k, e, nr, c in zip(sv["key"].tolist(), sv["src"].tolist(), sv["nrm"].tolist(), sv["rgb"].tolist()):
            e2 = e + di * res * res
            if k not in best or e2 < best[k][0]:
                best[k] = (e2, nr, c)
    full = oracle.sample_visible(q, m.tri, m.rgb, dirs, res)
    assert len(full["key"]) == len(best)
    for k, e, nr, c in zip(full["key"].tolist(), full["src"].tolist(), full["nrm"].tolist(), full["rgb"].tolist()):
        assert best[k] == (e, nr, c)
    mort = [_morton_py(p) for p in oracle.unpack(full["key"])]
    assert all(a < b for a, b in zip(mort, mort[1:]))


def test_plane_positions_and_normals():
    """Surfels of a tilted plane z = x - 2y + c lie on it up to the floor rounding of
    each coordinate, and carry the plane's unit normal turned to the camera."""
    c = 900000
    pts2 = [(100000, 50000), (900000, 80000), (800000, 500000), (90000, 450000)]
    verts = [[x, y, x - 2 * y + c] for x, y in pts2]
    q, t = _mesh_q(verts, [[0, 1, 2], [0, 2, 3]])
    sv = oracle.sample_visible(q, t, None, np.array([[0, 0, 1]], np.int8), 128)
    P = oracle.unpack(sv["key"])
    assert len(P) > 1000
    resid = P[:, 2] - (P[:, 0] - 2 * P[:, 1] + c)
    assert np.abs(resid).max() < 1 + 1 + 2
    n = np.array([-1.0, 2.0, 1.0])  # normal of z - x + 2y = c, facing +z
    want = [int(round(32767.0 * v / math.sqrt(6.0))) for v in n]
    assert (sv["nrm"] == np.array(want)).all()


def test_torus_top_view_area():
    """Covered pixels of the top view match the annulus area 4*pi*R*r within the
    boundary-pixel count (sanity of scale and screen mapping)."""
    m = W.torus()
    q, mn, s = oracle.quantise(m.xyz)
    res = 128
    depth, _ = oracle.raster_dir(q, m.tri, [0, 0, 1], res)
    covered = int((depth != np.uint64(2**64 - 1)).sum())
    E = 2.6  # bbox side in x and y (largest extent)
    px = E / res
    want = 4 * math.pi * 1.0 * 0.3 / px**2
    boundary = 4 * math.pi * 1.0 / px
    assert abs(covered - want) < boundary / 2


def test_sample_edge_cases():
    q = np.array([[0, 0, 0], [10, 10, 10], [20, 20, 20]], np.int32)
    t = np.array([[0, 1, 2]], np.uint32)  # collinear: zero area in every view
    sv = oracle.sample_visible(q, t, None, W.AXIS_DIRS, 16)
    assert len(sv["key"]) == 0
    m = W.cube()
    qq, _, _ = oracle.quantise(m.xyz)
    sv = oracle.sample_visible(qq, m.tri, None, W.AXIS_DIRS, 1)
    assert len(sv["key"]) == 6  # one pixel per face
    with pytest.raises(ValueError):
        oracle.sample_visible(qq, m.tri, None, W.AXIS_DIRS, 0)
    with pytest.raises(ValueError):
        oracle.sample_visible(qq, m.tri, None, np.zeros((1, 3), np.int8), 8)


def test_torus_config_count():
    """The torus workload (R=1, r=0.3, 128x64 quads, 6 axis views at 128^2) gives ~30-50k surfels."""
    m = W.torus()
    sv, mn, s = oracle.sample_mesh(m, W.AXIS_DIRS, 128)
    assert 30000 <= len(sv["key"]) <= 50000
    assert m.ntris == 16384 and m.nverts == 8192


def test_quantiser_per_axis_minimum():
    """Each axis subtracts its own bbox minimum before scaling."""
    xyz = np.array([[1, -3, 10], [5, -1, 11], [3, -2, 10.5]], np.float32)
    q, mn, s = oracle.quantise(xyz)
    assert mn.tolist() == [1, -3, 10] and s == Q / 4.0
    assert q.tolist() == [[0, 0, 0], [Q, Q // 2, Q // 4], [Q // 2, Q // 4, Q // 8]]


def test_raster_tie_rule_closed_form():
    """Pixel centres exactly on an edge belong to the triangle that contains the
    centre shifted by an infinitesimal (+1, +eta) in screen (X, Y): a rectangle whose
    four edges pass through pixel centres covers columns a0..a1-1 and rows b0..b1-1
    (its left and lower edges are kept, its right and upper edges are not)."""
    a0, a1, b0, b1 = 4, 20, 7, 30
    def ub(a):  # u with X = 256a + 128 exactly (a pixel-centre column)
        return (256 * a + 128) * 128
    def xb(b):  # x with Y = 256b + 128 exactly
        return Q - (256 * b + 128) * 128
    z = 5
    v = [[xb(b0), ub(a0), z], [xb(b0), ub(a1), z], [xb(b1), ub(a1), z], [xb(b1), ub(a0), z]]
    for tris in ([[0, 1, 2], [0, 2, 3]], [[0, 2, 1], [0, 3, 2]], [[1, 2, 3], [1, 3, 0]]):
        q, t = _mesh_q(v, tris)
        _, _, cnt = oracle.raster_dir(q, t, [0, 0, 1], RES, counts=True)
        want = np.zeros((RES, RES), np.uint32)
        want[b0:b1, a0:a1] = 1
        assert np.array_equal(cnt, want)


def test_raster_snap_rounds_half_up():
    """Vertices snap to 1/256 pixel by rounding half up: an edge at X = 256a + 128.5
    snaps to 256a + 129, so the centre of column a (256a + 128) is left uncovered."""
    a0, a1, b0, b1 = 6, 30, 3, 40
    def ub(a):  # X = 256a + 128.5 before snapping
        return (256 * a + 128) * 128 + 64
    v = [[_xbound(b0), ub(a0), 9], [_xbound(b0), ub(a1), 9], [_xbound(b1), ub(a1), 9], [_xbound(b1), ub(a0), 9]]
    q, t = _mesh_q(v, [[0, 1, 2], [0, 2, 3]])
    _, _, cnt = oracle.raster_dir(q, t, [0, 0, 1], RES, counts=True)
    want = np.zeros((RES, RES), np.uint32)
    want[b0:b1, a0 + 1:a1 + 1] = 1
    assert np.array_equal(cnt, want)


def test_plane_both_windings():
    """Interpolation uses each vertex's own weight whatever the input winding."""
    c = 900000
    pts2 = [(100000, 50000), (900000, 80000), (800000, 500000), (90000, 450000)]
    verts = [[x, y, x - 2 * y + c] for x, y in pts2]
    q, _ = _mesh_q(verts, [[0, 1, 2]])
    out = []
    for tris in ([[0, 1, 2], [0, 2, 3]], [[0, 2, 1], [0, 3, 2]]):
        t = np.asarray(tris, np.uint32)
        sv = oracle.sample_visible(q, t, None, np.array([[0, 0, 1]], np.int8), 96)
        P = oracle.unpack(sv["key"])
        resid = P[:, 2] - (P[:, 0] - 2 * P[:, 1] + c)
        assert np.abs(resid).max() < 4
        lo = np.array(pts2).min(0)
        hi = np.array(pts2).max(0)
        assert (P[:, 0] >= lo[0]).all() and (P[:, 0] <= hi[0]).all()
        out.append(sv["key"])
    assert np.array_equal(out[0], out[1])


def test_dedup_keeps_lowest_emission_index():
    """A vertex that lands exactly on a pixel centre in both the +x and the +z view is
    emitted by both; the merged surfel keeps the +x row (direction 0, smaller e)."""
    res = RES
    p, p1, p2 = 20, 25, 40
    A = [Q - (1 << 15) * p1 - (1 << 14), (1 << 15) * p + (1 << 14), (1 << 15) * p2 + (1 << 14)]
    # a planar fan around A in the plane with normal (1, 0, 1): visible from both views,
    # and the pixel at A is covered by exactly one fan triangle in each
    L = 200000
    ring = [[A[0] + r * L, A[1] + s_ * L, A[2] - r * L] for s_, r in ((1, 1), (-1, 1), (-1, -1), (1, -1))]
    q, t = _mesh_q([A] + ring, [[0, 1 + i, 1 + (i + 1) % 4] for i in range(4)])
    dirs = np.array([[1, 0, 0], [0, 0, 1]], np.int8)
    keyA = int(oracle.pack(np.array(A)))
    rows = []
    for di, d in enumerate(dirs):
        sv = oracle.sample_visible(q, t, None, d[None], res)
        hit = np.where(sv["key"] == np.uint64(keyA))[0]
        assert len(hit) == 1, di
        rows.append(int(sv["src"][hit[0]]) + di * res * res)
    both = oracle.sample_visible(q, t, None, dirs, res)
    hit = np.where(both["key"] == np.uint64(keyA))[0]
    assert len(hit) == 1
    assert int(both["src"][hit[0]]) == min(rows) < res * res


def test_quantiser_negative_zero_minimum():
    """A bbox minimum of -0.0 is reported as +0.0; the quantised positions are unchanged."""
    xyz = np.array([[-0.0, 0, 0], [1, 1, 1], [0.0, 0.5, 0.5]], np.float32)
    q, mn, s = oracle.quantise(xyz)
    assert not np.signbit(mn).any()
    assert q[0].tolist() == [0, 0, 0] and q[2].tolist() == [0, Q // 2, Q // 2]
