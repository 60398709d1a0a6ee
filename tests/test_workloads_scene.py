"""Host checks of the production-line scene generator (the synthetic stand-in for the
paper's evaluation scene, Sec. 5): every primitive is a closed surface of the stated
size, the Philox words are the published generator's, and the node hierarchy follows
Sec. 3.4's rule (nodes of more than 10k triangles)."""
import numpy as np
import pytest

from paper_1904_08225_gb300 import workloads as W


def _closed(v, tri):
    """With vertices merged by position, every directed edge appears once and its reverse
    once (a closed, consistently wound surface)."""
    _, inv = np.unique(v, axis=0, return_inverse=True)
    tri = inv.reshape(-1)[tri]
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]).astype(np.int64)
    fwd = set(map(tuple, e.tolist()))
    assert len(fwd) == len(e)
    assert all((b, a) in fwd for a, b in fwd)


def _volume(v, tri):
    a, b, c = (v[tri[:, k]].astype(np.float64) for k in range(3))
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


@pytest.mark.parametrize("part,line,slot", [(0, 0, 0), (123, 4, 77), (2**33 + 1, 19, 2499)])
def test_scene_part_primitives_are_closed_boxes_and_cylinders(part, line, slot):
    nb, nc = 12, 4
    m = W.scene_part(7, part, line, slot, nb, nc)
    assert m.xyz.shape == (nb * W.BOX_VERTS + nc * W.CYL_VERTS, 3)
    assert m.tri.shape == (nb * W.BOX_TRIS + nc * W.CYL_TRIS, 3) and m.rgb.shape == m.tri.shape
    off = np.array([np.float32(slot) * W.SCENE_DX, np.float32(line) * W.SCENE_DY, 0], np.float64)
    vols = []
    for b in range(nb):
        t = m.tri[b * 48:(b + 1) * 48].astype(np.int64) - b * 54
        v = m.xyz[b * 54:(b + 1) * 54]
        assert t.min() == 0 and t.max() == 53
        _closed(v, t)
        lo, hi = v.min(0), v.max(0)
        # every vertex on the box surface, 9 per face, the six faces in x-lo, x-hi, y-lo, y-hi, z-lo, z-hi order
        for f, (ax, at) in enumerate([(0, lo), (0, hi), (1, lo), (1, hi), (2, lo), (2, hi)]):
            assert np.all(v[f * 9:(f + 1) * 9, ax] == at[ax]), (b, f)
        # the box is centred in the unit cube cell of its part and at most 0.3 on a side
        c = (lo.astype(np.float64) + hi) / 2 - off
        assert np.all(c > -0.16) and np.all(c < 1.16) and np.all(hi - lo <= 0.3001)
        vol = _volume(v, t)
        assert abs(abs(vol) - np.prod((hi - lo).astype(np.float64))) < 1e-3 * np.prod(hi - lo) + 1e-9
        vols.append(np.sign(vol))
        # one colour per face
        col = m.rgb[b * 48:(b + 1) * 48].reshape(6, 8, 3)
        assert np.all(col == col[:, :1])
    for q in range(nc):
        t = m.tri[nb * 48 + q * 192: nb * 48 + (q + 1) * 192].astype(np.int64) - (nb * 54 + q * 98)
        v = m.xyz[nb * 54 + q * 98: nb * 54 + (q + 1) * 98].astype(np.float64)
        assert t.min() == 0 and t.max() == 97
        _closed(v, t)
        vols.append(np.sign(_volume(v, t)))
    assert len(set(vols)) == 1  # boxes and cylinders wound the same way


def test_philox_words_match_known_answers():
    """The vectorised Philox of the generator against the published known-answer vectors."""
    rows = []
    for line in open(__file__.replace("test_workloads_scene.py", "golden/philox4x32_10_kat.txt")):
        line = line.split("#")[0].split()
        if len(line) == 10:
            rows.append([int(x, 16) for x in line])
    assert rows
    for r in rows:
        got = W.philox4x32_10(r[0], r[1], r[2], r[3], r[4], r[5])
        assert [int(x) for x in got] == r[6:10]


def test_scene_nodes_hierarchy():
    nodes = W.scene_nodes(lines=3, per_line=120, group=50)
    lv = [n.level for n in nodes]
    assert lv.count(0) == 360 and lv.count(1) == 9 and lv.count(2) == 3
    tris = W.BOX_TRIS * 200 + W.CYL_TRIS * 50
    assert tris == 19_200 and all(n.count * tris > 10_000 for n in nodes)
    for l in range(3):
        grp = [n for n in nodes if n.line == l and n.level == 1]
        assert [(g.first, g.count) for g in grp] == [(0, 50), (50, 50), (100, 20)]
        assert [p[0] for p in nodes[[i for i, n in enumerate(nodes) if n.line == l and n.level == 2][0]].parts(120)] == \
            list(range(l * 120, (l + 1) * 120))


def test_node_mesh_concatenates_parts():
    nd = W.SceneNode(1, 3, 2, 1)
    m = W.scene_node_mesh(3, nd, 10, 4, 1)
    a, b = W.scene_part(3, 13, 1, 3, 4, 1), W.scene_part(3, 14, 1, 4, 4, 1)
    assert np.array_equal(m.xyz, np.concatenate([a.xyz, b.xyz]))
    assert np.array_equal(m.tri, np.concatenate([a.tri, b.tri + np.uint32(a.nverts)]))
    assert np.array_equal(m.rgb, np.concatenate([a.rgb, b.rgb]))


def test_cad_primitives_closed():
    """The single-part CAD generator's box and cylinder are closed and wound alike."""
    v, t = W._box((0.1, 0.2, 0.3), (0.4, 0.25, 0.9))
    _closed(v, t.astype(np.int64))
    vb = _volume(v, t)
    assert abs(abs(vb) - 0.3 * 0.05 * 0.6) < 1e-9
    v, t = W._cylinder((0.5, 0.5, 0.5), 1, 0.1, 0.4)
    _closed(v, t.astype(np.int64))
    vc = _volume(v, t)
    # a 32-gon prism: area 16 sin(2 pi / 32) r^2 times the length
    assert abs(abs(vc) - 16 * np.sin(2 * np.pi / 32) * 0.01 * 0.4) < 1e-9
    assert np.sign(vb) == np.sign(vc)
