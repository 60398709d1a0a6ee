"""Splat sampling on the GPU (bs_sample_splats) against the oracle, bit for bit: parent
nodes rendered from their children's surfels drawn as oriented discs (Sec. 3.4 bottom-up
generation, Sec. 4.2 discs)."""
import numpy as np
import pytest

import oracle
from paper_1904_08225_gb300 import workloads as W

pytestmark = pytest.mark.gpu
Q = 2**21 - 1
UP = np.array([[0, 0, 1]], np.int8)


@pytest.fixture(scope="module")
def bs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs as _bs
    _bs.load()
    return _bs


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.view(dtype) if dtype is not None else t).cuda()


def _gpu_sets(host_sets, nodes_of=None):
    """Oracle-style set dicts -> device descriptors (optionally with a perm over a longer array)."""
    import torch
    out = []
    for i, st in enumerate(host_sets):
        key = np.asarray(st["key"], np.uint64)
        d = dict(key=_dev(key.view(np.int64)), nrm=_dev(np.asarray(st["nrm"], np.int16).reshape(-1, 3)),
                 rgb=None if st.get("rgb") is None else _dev(np.asarray(st["rgb"], np.uint8).reshape(-1, 3)),
                 perm=None, n=len(key), bbox_min=[float(x) for x in st["bbox_min"]], scale=float(st["scale"]),
                 r2=int(st["r2"]), node=0 if nodes_of is None else nodes_of[i])
        out.append(d)
    return out


def _check(got, ref):
    assert got["n"] == len(ref["key"])
    assert np.array_equal(got["key"].cpu().numpy().view(np.uint64), ref["key"])
    assert np.array_equal(got["nrm"].cpu().numpy(), ref["nrm"])
    assert np.array_equal(got["rgb"].cpu().numpy(), ref["rgb"])
    assert np.array_equal(got["src"].cpu().numpy().view(np.uint32), ref["src"])


def _pin_sets():
    h = 2**21 // 32
    c = [Q // 2, Q // 2, Q // 2]
    mk = lambda cc, n, r2, rgb: dict(key=oracle.pack(np.atleast_2d(np.asarray(cc, np.int64))),
                                     nrm=np.atleast_2d(np.asarray(n, np.int16)),
                                     rgb=np.atleast_2d(np.asarray(rgb, np.uint8)),
                                     bbox_min=np.zeros(3, np.float32), scale=1.0, r2=r2)
    return [
        [mk(c, [0, 0, 32767], (5 * h) ** 2 + h, [1, 2, 3])],                      # facing
        [mk(c, [0, -16000, 28000], (7 * h) ** 2 + 17, [4, 5, 6])],                 # tilted
        [mk(c, [0, -15000, 29000], (6 * h) ** 2, [1, 0, 0]),                       # crossing
         mk([c[0] + 3 * h, c[1] - 2 * h, c[2] + 5000], [12000, 9000, 29000], (6 * h) ** 2, [2, 0, 0])],
        [mk(c, [32767, 0, 0], (5 * h) ** 2, [7, 7, 7])],                          # edge-on from +z
        [mk([c, c], [[0, 0, 32767], [0, 0, 32767]], (3 * h) ** 2, [[1, 2, 3], [4, 5, 6]])],  # tie
        [mk([100, 200, 300], [0, 0, -32767], (40 * h) ** 2, [9, 9, 9])],           # big disc at the corner
    ]


@pytest.mark.parametrize("case", range(6))
def test_pin_cases_match_oracle(bs, case):
    sets = _pin_sets()[case]
    for dirs in (UP, W.AXIS_DIRS):
        for res in (32, 37):
            ref = oracle.sample_splats(sets, np.zeros(3, np.float32), 1.0, dirs, res)
            got = bs.sample_splats(_gpu_sets(sets), [((0.0, 0.0, 0.0), 1.0, res)], dirs)[0]
            _check(got, ref)


def _meshes(seeds=(1, 2, 3)):
    out = []
    for j, sd in enumerate(seeds):
        m = W.torus(nu=48, nv=24, seed=sd, rot=W.CUBE_ROTATIONS[sd % 24])
        m.xyz = m.xyz * np.float32(0.5 + 0.25 * j) + np.float32([1.5 * j, 0.3 * j, -0.2 * j])
        out.append(m)
    return out


def _children(bs, res=64, seeds=(1, 2, 3)):
    """Child parts sampled and ordered twice: by the oracle (the oracle side's inputs) and
    by the GPU (the product side's inputs); the two must already agree."""
    kids = []
    for sd, m in zip(seeds, _meshes(seeds)):
        sv, mn, sc = oracle.sample_mesh(m, W.AXIS_DIRS, res)
        st = oracle.start_index(len(sv["key"]), seed=sd)
        operm, orad2 = oracle.greedy(sv["key"], st)
        g = bs.sample_visible(_dev(m.xyz), _dev(m.tri.view(np.int32)), _dev(m.rgb), W.AXIS_DIRS, res)
        perm, rad2, _ = bs.order(g["key"], seed=sd, scale=g["scale"])
        assert np.array_equal(g["key"].cpu().numpy().view(np.uint64), sv["key"])
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), operm)
        assert g["scale"] == sc and np.array_equal(g["bbox_min"], mn)
        kids.append(dict(g=g, perm=perm, sv=sv, operm=operm, orad2=orad2, mn=mn, sc=sc))
    return kids


def _parent_frame(kids):
    return oracle.parent_frame([k["mn"] for k in kids], [k["sc"] for k in kids])


def test_children_prefixes_match_oracle(bs):
    """Prefixes of real child orderings (every set through perm), several nodes per call."""
    kids = _children(bs)
    fmin, fscale = _parent_frame(kids)
    host_sets, gsets = [], []
    for j, k in enumerate(kids):
        p = [50, 400, 1500][j]
        r2 = int(k["orad2"][p])
        pi = k["operm"][:p]
        sv = k["sv"]
        host_sets.append(dict(key=sv["key"][pi], nrm=sv["nrm"][pi], rgb=sv["rgb"][pi], bbox_min=k["mn"],
                              scale=k["sc"], r2=r2))
        g = k["g"]
        gsets.append(dict(key=g["key"], nrm=g["nrm"], rgb=g["rgb"], perm=k["perm"][:p], n=p,
                          bbox_min=list(g["bbox_min"]), scale=g["scale"], r2=r2, node=j % 2))
    # node 0 gets children 0 and 2, node 1 gets child 1; a third node gets all three again
    gsets += [dict(s, node=2) for s in gsets]
    nodes = [(fmin, fscale, 96), (fmin, fscale, 64), (fmin, fscale, 128)]
    got = bs.sample_splats(gsets, nodes, W.AXIS_DIRS)
    for ni, members in ((0, [0, 2]), (1, [1]), (2, [0, 1, 2])):
        ref = oracle.sample_splats([host_sets[i] for i in members], fmin, fscale, W.AXIS_DIRS, nodes[ni][2])
        assert len(ref["key"]) > 100
        _check(got[ni], ref)
        assert np.allclose(got[ni]["bbox_min"], fmin) and got[ni]["scale"] == fscale


def test_rejects_bad_arguments(bs):
    sets = _gpu_sets(_pin_sets()[0])
    with pytest.raises(bs.BsError):
        bs.sample_splats(sets, [((0.0, 0.0, 0.0), 1.0, 32)], np.array([[1, 1, 0]], np.int8))
    with pytest.raises(bs.BsError):
        bs.sample_splats([dict(sets[0], node=3)], [((0.0, 0.0, 0.0), 1.0, 32)], UP)
    with pytest.raises(bs.BsError):
        bs.sample_splats(sets, [((0.0, 0.0, 0.0), -1.0, 32)], UP)


def test_empty_sets_give_empty_nodes(bs):
    got = bs.sample_splats([], [((0.0, 0.0, 0.0), 1.0, 16), ((1.0, 1.0, 1.0), 2.0, 8)], W.AXIS_DIRS)
    assert [g["n"] for g in got] == [0, 0]
