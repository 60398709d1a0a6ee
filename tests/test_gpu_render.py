"""Headless renders (no window, no graphics API: the image is a device buffer) and the
image-space coverage check of Sec. 4.1: the shortest prefix of an exact ordering that
reaches every surfel within r, drawn as the oriented discs of Sec. 4.2 with radius r,
covers the object's pixels.  Images are bit-compared with the oracle's depth passes."""
import numpy as np
import pytest

import oracle
from paper_1904_08225_gb300 import workloads as W

pytestmark = pytest.mark.gpu
EMPTY = np.uint64(2**64 - 1)


@pytest.fixture(scope="module")
def bs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs as _bs
    _bs.load()
    return _bs


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _img(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("d", [[0, 0, 1], [-1, 0, 0], [0, 1, 0], [1, 1, 1], [0, -1, 1]])
@pytest.mark.parametrize("res", [64, 101])
def test_render_mesh_matches_oracle(bs, d, res):
    m = W.torus(nu=48, nv=24, seed=3, rot=W.CUBE_ROTATIONS[7])
    q, _, _ = oracle.quantise(m.xyz)
    ref, _ = oracle.raster_dir(q, m.tri, np.array(d, np.int8), res)
    got = bs.render_mesh(_dev(m.xyz), _dev(m.tri.view(np.int32)), d, res)
    assert np.array_equal(_img(got), ref)


def _child(bs, mesh, res, seed=0):
    """A part sampled and ordered by the oracle (oracle side) and by the GPU (product side)."""
    sv, mn, sc = oracle.sample_mesh(mesh, W.AXIS_DIRS, res)
    operm, orad2 = oracle.greedy(sv["key"], oracle.start_index(len(sv["key"]), seed=seed))
    g = bs.sample_visible(_dev(mesh.xyz), _dev(mesh.tri.view(np.int32)), None, W.AXIS_DIRS, res)
    perm, rad2, _ = bs.order(g["key"], seed=seed, scale=g["scale"])
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), operm)
    return sv, mn, sc, operm, orad2, g, perm


@pytest.mark.parametrize("k", [1, 2, 4])
def test_render_prefix_discs_matches_oracle(bs, k):
    res = 48
    mesh = W.torus(nu=32, nv=16, seed=5)
    sv, mn, sc, operm, orad2, g, perm = _child(bs, mesh, res)
    h = 2**21 // res
    p = oracle.prefix_for_radius(orad2, (k * h) ** 2)
    hs = dict(key=sv["key"][operm[:p]], nrm=sv["nrm"][operm[:p]], bbox_min=mn, scale=sc, r2=(k * h) ** 2)
    gs = dict(key=g["key"], nrm=g["nrm"], rgb=None, perm=perm[:p], n=p, bbox_min=list(g["bbox_min"]),
              scale=g["scale"], r2=(k * h) ** 2)
    for d in W.AXIS_DIRS:
        ref = oracle.render_splats([hs], mn, sc, d, res)
        got = bs.render_splats([gs], (mn, sc, res), d)
        assert np.array_equal(_img(got), ref), d


@pytest.mark.parametrize("name,k", [("torus", 1), ("torus", 2), ("torus", 4), ("cad", 2)])
def test_prefix_for_radius_covers_the_object(bs, name, k):
    """Sec. 4.1: the prefix that reaches every surfel within r = k pixel steps, drawn with
    radius r, covers (nearly) every pixel the mesh covers, from every axis direction; the
    paper's estimate p(r) = pm (rm / r)^2 is measured beside it."""
    res = 128
    mesh = W.torus(nu=96, nv=48, seed=1) if name == "torus" else W.cad_part(seed=2, nboxes=60, ncyl=15)
    xyz, tri = _dev(mesh.xyz), _dev(mesh.tri.view(np.int32))
    g = bs.sample_visible(xyz, tri, None, W.AXIS_DIRS, res)
    perm, rad2, _ = bs.order(g["key"], seed=0, scale=g["scale"])
    h = 2**21 / res
    r2 = int((k * h) ** 2)
    p = bs.prefix_for_radius(rad2, r2)
    pm = min(1000, g["n"])
    rm2 = bs.prefix_median_nn(g["key"], perm, pm)
    p_est = int(min(g["n"], max(1, round(bs.prefix_estimate(pm, rm2, r2)))))
    cover = {}
    for tag, pp in (("exact", p), ("estimate", p_est)):
        s = dict(key=g["key"], nrm=g["nrm"], rgb=None, perm=perm[:pp], n=pp, bbox_min=list(g["bbox_min"]),
                 scale=g["scale"], r2=r2)
        tot = hit = 0
        for d in W.AXIS_DIRS:
            mimg = _img(bs.render_mesh(xyz, tri, d, res)) != EMPTY
            simg = _img(bs.render_splats([s], (g["bbox_min"], g["scale"], res), d)) != EMPTY
            tot += int(mimg.sum())
            hit += int((mimg & simg).sum())
        cover[tag] = hit / tot
    assert p < g["n"] and cover["exact"] >= 0.98, (p, cover)
    print(f"{name} r={k}px: exact prefix {p} covers {cover['exact']:.4f}; estimate {p_est} covers "
          f"{cover['estimate']:.4f} of {g['n']} surfels")
