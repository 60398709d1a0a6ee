"""Scene scale on the GPU: the device generator against its host mirror, and every level of
node of a scene sampled and ordered against the oracle.

Scenes are production lines of parts; nodes are single parts, groups of consecutive parts and
whole lines (Sec. 3.4's hierarchy).  Each node keeps min(200k, triangles / 2) surfels, the
bound of the paper's evaluation (Sec. 5).
"""
import numpy as np
import pytest

import oracle
from paper_1904_08225_gb300 import workloads as W

pytestmark = pytest.mark.gpu
I64MAX = np.iinfo(np.int64).max


@pytest.fixture(scope="module")
def bs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs as _bs
    _bs.load()
    return _bs


def _host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("nboxes,ncyl", [(200, 50), (7, 3), (0, 4), (5, 0)])
def test_generator_matches_host_mirror(bs, nboxes, ncyl):
    seed = 0x1234_5678_9ABC
    parts = [(0, 0, 0), (2_499, 0, 2_499), (31_337, 12, 1_337), (2**40 + 5, 3, 17)]
    xyz, tri, rgb = bs.scene_generate(seed, parts, nboxes, ncyl)
    xyz_l, tri_l, rgb_l = bs.scene_generate(seed, parts, nboxes, ncyl, local_indices=True)
    vp = W.BOX_VERTS * nboxes + W.CYL_VERTS * ncyl
    tp = W.BOX_TRIS * nboxes + W.CYL_TRIS * ncyl
    assert xyz.shape == (vp * len(parts), 3) and tri.shape == (tp * len(parts), 3)
    X, T, Rg = _host(xyz), _host(tri).view(np.uint32), _host(rgb)
    TL = _host(tri_l).view(np.uint32)
    assert np.array_equal(_host(xyz_l).view(np.uint32), X.view(np.uint32))
    assert np.array_equal(_host(rgb_l), Rg)
    for q, (p, l, s) in enumerate(parts):
        m = W.scene_part(seed, p, l, s, nboxes, ncyl)
        assert np.array_equal(X[q * vp:(q + 1) * vp].view(np.uint32), m.xyz.view(np.uint32)), q
        assert np.array_equal(T[q * tp:(q + 1) * tp], m.tri + np.uint32(q * vp)), q
        assert np.array_equal(TL[q * tp:(q + 1) * tp], m.tri), q
        assert np.array_equal(Rg[q * tp:(q + 1) * tp], m.rgb), q


def test_generator_node_mesh(bs):
    nodes = W.scene_nodes(lines=2, per_line=12, group=5)
    for nd in [n for n in nodes if n.level > 0][:3]:
        xyz, tri, rgb = bs.scene_generate(9, nd.parts(12), 30, 10)
        m = W.scene_node_mesh(9, nd, 12, 30, 10)
        assert np.array_equal(_host(xyz).view(np.uint32), m.xyz.view(np.uint32))
        assert np.array_equal(_host(tri).view(np.uint32), m.tri)
        assert np.array_equal(_host(rgb), m.rgb)


def test_generator_rejects_bad_arguments(bs):
    with pytest.raises(bs.BsError):
        bs.scene_generate(0, [(0, 0, 0)], 0, 0)


def _check_node(seed, idx, node, per_line, nboxes, ncyl, res, got):
    """Oracle of one node: host mesh -> Sec. 3.1 sampling -> exact ordering with the node bound."""
    from paper_1904_08225_gb300 import scene
    m = W.scene_node_mesh(seed, node, per_line, nboxes, ncyl)
    sv, _, _ = oracle.sample_mesh(m, W.AXIS_DIRS, res)
    key, perm, rad2 = got
    assert np.array_equal(key, sv["key"]), idx
    mc = scene.node_bound(m.ntris, len(key))
    st = oracle.start_index(len(key), seed=seed, part_id=idx)
    p, r = oracle.greedy(sv["key"], st, max_count=mc)
    assert np.array_equal(perm, p), idx
    assert np.array_equal(rad2, r), idx
    return len(key), mc


def test_reduced_scene_every_node(bs):
    """Every node of a 2-line scene (leaves, groups, lines) against the oracle."""
    from paper_1904_08225_gb300 import scene
    seed, lines, per_line, group, nb, nc = 21, 2, 7, 3, 20, 5
    level_res = {0: 96, 1: 256, 2: 1024}
    nodes = W.scene_nodes(lines, per_line, group)
    out = scene.run(seed, lines, per_line, group, nb, nc, keep=range(len(nodes)), leaf_wave=5, group_wave=2,
                    level_res=level_res)
    assert out.nodes == len(nodes) and sorted(out.kept) == list(range(len(nodes)))
    assert set(out.per_level) == {0, 1, 2}
    for i, nd in enumerate(nodes):
        _check_node(seed, i, nd, per_line, nb, nc, level_res[nd.level], out.kept[i])


def test_scene_lpt_shards_cover_every_node_once(bs):
    """The scene's nodes split over two ranks by LPT (run here one rank after the other on
    one GPU; ranks share nothing): the shards are disjoint, cover every node, and each
    node's output equals the unsharded run's."""
    from paper_1904_08225_gb300 import scene
    seed, lines, per_line, group, nb, nc = 21, 2, 7, 3, 20, 5
    level_res = {0: 96, 1: 256, 2: 1024}
    nodes = W.scene_nodes(lines, per_line, group)
    full = scene.run(seed, lines, per_line, group, nb, nc, keep=range(len(nodes)), leaf_wave=5, group_wave=2,
                     level_res=level_res)
    parts = [scene.run(seed, lines, per_line, group, nb, nc, keep=range(len(nodes)), leaf_wave=5, group_wave=2,
                       level_res=level_res, world=2, rank=r) for r in range(2)]
    assert parts[0].nodes > 0 and parts[1].nodes > 0
    assert not set(parts[0].kept) & set(parts[1].kept)
    assert sorted(list(parts[0].kept) + list(parts[1].kept)) == list(range(len(nodes)))
    assert parts[0].surfels_ordered + parts[1].surfels_ordered == full.surfels_ordered
    for pr in parts:
        for i, (key, perm, rad2) in pr.kept.items():
            fk, fp, fr = full.kept[i]
            assert np.array_equal(key, fk) and np.array_equal(perm, fp) and np.array_equal(rad2, fr), i


def _invariants(key, perm, rad2, picks):
    P = oracle.unpack(key[perm])
    assert len(np.unique(perm)) == len(perm) and perm.max() < len(key)
    assert rad2[0] == I64MAX and np.all(np.diff(rad2[1:]) <= 0)
    for k in picks:
        assert rad2[k] == ((P[:k] - P[k]) ** 2).sum(1).min(), k


def test_full_scene_seeded_subset(bs):
    """The 20-line x 2,500-part scene (~1G triangles): a seeded subset of leaves and groups
    against the oracle, every line node against the ordering invariants."""
    from paper_1904_08225_gb300 import scene
    seed, lines, per_line, group = 5, 20, 2500, 50
    nodes = W.scene_nodes(lines, per_line, group)
    g = np.random.default_rng(seed)
    leaves = [i for i, n in enumerate(nodes) if n.level == 0]
    groups = [i for i, n in enumerate(nodes) if n.level == 1]
    line_ids = [i for i, n in enumerate(nodes) if n.level == 2]
    pick_leaves = sorted(g.choice(leaves, 40, replace=False).tolist())
    pick_groups = sorted(g.choice(groups, 2, replace=False).tolist())
    out = scene.run(seed, lines, per_line, group, keep=pick_leaves + pick_groups + line_ids)
    assert out.nodes == len(nodes)
    assert out.per_level[0]["nodes"] == lines * per_line
    assert out.triangles == sum(n.count for n in nodes) * (W.BOX_TRIS * 200 + W.CYL_TRIS * 50)
    for i in pick_leaves + pick_groups:
        _check_node(seed, i, nodes[i], per_line, 200, 50, scene.LEVEL_RES[nodes[i].level], out.kept[i])
    for i in line_ids:
        key, perm, rad2 = out.kept[i]
        assert len(perm) == scene.node_bound(nodes[i].count * 19_200, len(key))
        _invariants(key, perm, rad2, [1, 2, 17, len(perm) // 2, len(perm) - 1])


def test_packed_bindings_match_list_bindings(bs):
    """sample_visible_packed / order_packed (pointer arrays built with numpy) give the same
    surfels and orderings as the per-part list bindings."""
    import torch
    parts = [(p, 0, p) for p in range(5)]
    nb, nc = 10, 3
    vp, tp = nb * W.BOX_VERTS + nc * W.CYL_VERTS, nb * W.BOX_TRIS + nc * W.CYL_TRIS
    xyz, tri, rgb = bs.scene_generate(3, parts, nb, nc, local_indices=True)
    P = len(parts)
    res = [64, 96, 128, 80, 64]
    sv = bs.sample_visible_packed(xyz, tri, rgb, np.arange(P) * vp, [vp] * P, np.arange(P) * tp, [tp] * P, res,
                                  W.AXIS_DIRS)
    meshes = [(xyz[q * vp:(q + 1) * vp], tri[q * tp:(q + 1) * tp], rgb[q * tp:(q + 1) * tp]) for q in range(P)]
    ref = bs.sample_visible_batched(meshes, res, W.AXIS_DIRS)
    for q in range(P):
        a, n = int(sv["ofs"][q]), int(sv["n"][q])
        assert n == ref[q]["n"] and sv["scale"][q] == ref[q]["scale"]
        for f in ("key", "nrm", "rgb", "src"):
            assert torch.equal(sv[f][a:a + n], ref[q][f]), (q, f)
    mc = [0, 100, 5, 10**9, 1]
    perm, rad2, radius, mofs = bs.order_packed(sv["key"], sv["ofs"], sv["n"], max_counts=mc, seeds=11,
                                               part_ids=[7, 8, 9, 10, 11], scales=sv["scale"])
    got = bs.order_batched([r["key"] for r in ref], seeds=[11] * P, part_ids=[7, 8, 9, 10, 11], max_counts=mc,
                           scales=[r["scale"] for r in ref])
    for q in range(P):
        lo, hi = int(mofs[q]), int(mofs[q + 1])
        assert torch.equal(perm[lo:hi], got[q][0]) and torch.equal(rad2[lo:hi], got[q][1])
        assert torch.equal(radius[lo:hi], got[q][2])


# ---- bottom-up generation (groups from parts' surfels, lines from groups') ----

Q = 2**21 - 1


def _oracle_leaf(seed, idx, node, per_line, nb, nc, res):
    m = W.scene_node_mesh(seed, node, per_line, nb, nc)
    sv, mn, sc = oracle.sample_mesh(m, W.AXIS_DIRS, res)
    mc = min(200_000, m.ntris // 2, len(sv["key"]))
    st = oracle.start_index(len(sv["key"]), seed=seed, part_id=idx)
    p, r = oracle.greedy(sv["key"], st, max_count=mc)
    return dict(sv=sv, mn=mn, sc=sc, perm=p, rad2=r, m=mc)


def _oracle_parent(children, seed, idx, res, ntris):
    """A parent from its children's prefixes: the frame holding the children's cubes, each
    child's shortest prefix reaching its surfels within one parent pixel step (Sec. 4.1),
    its discs drawn (Sec. 3.4 / 4.2), then the exact ordering with the node bound."""
    fmin, fs = oracle.parent_frame([c["mn"] for c in children], [c["sc"] for c in children])
    sets = []
    for c in children:
        p = oracle.prefix_for_radius(c["rad2"], oracle.child_target_r2(c["sc"], fs, res))
        pi = c["perm"][:p]
        sets.append(dict(key=c["sv"]["key"][pi], nrm=c["sv"]["nrm"][pi], rgb=c["sv"]["rgb"][pi], bbox_min=c["mn"],
                         scale=c["sc"], r2=int(c["rad2"][min(p, c["m"] - 1)])))
    sv = oracle.sample_splats(sets, fmin, fs, W.AXIS_DIRS, res)
    mc = min(200_000, ntris // 2, len(sv["key"]))
    st = oracle.start_index(len(sv["key"]), seed=seed, part_id=idx)
    p, r = oracle.greedy(sv["key"], st, max_count=mc)
    return dict(sv=sv, mn=fmin, sc=fs, perm=p, rad2=r, m=mc)


def test_bottom_up_reduced_scene_every_node(bs):
    """Every node of a 2-line scene generated bottom-up against the oracle chain (parts from
    triangles, groups from parts' discs, lines from groups' discs)."""
    from paper_1904_08225_gb300 import scene
    seed, lines, per_line, group, nb, nc = 23, 2, 7, 3, 20, 5
    level_res = {0: 96, 1: 256, 2: 1024}
    nodes = W.scene_nodes(lines, per_line, group)
    out = scene.run_hierarchical(seed, lines, per_line, group, nb, nc, keep=range(len(nodes)), groups_per_wave=2,
                                 level_res=level_res)
    assert out.nodes == len(nodes) and sorted(out.kept) == list(range(len(nodes)))
    tp = W.BOX_TRIS * nb + W.CYL_TRIS * nc
    ref = {}
    for i, nd in enumerate(nodes):
        if nd.level == 0:
            ref[i] = _oracle_leaf(seed, i, nd, per_line, nb, nc, level_res[0])
    for i, nd in enumerate(nodes):
        if nd.level == 1:
            kids = [ref[j] for j, c in enumerate(nodes) if c.level == 0 and c.line == nd.line
                    and nd.first <= c.first < nd.first + nd.count]
            ref[i] = _oracle_parent(kids, seed, i, level_res[1], nd.count * tp)
    for i, nd in enumerate(nodes):
        if nd.level == 2:
            kids = [ref[j] for j, c in enumerate(nodes) if c.level == 1 and c.line == nd.line]
            ref[i] = _oracle_parent(kids, seed, i, level_res[2], nd.count * tp)
    for i, nd in enumerate(nodes):
        key, perm, rad2 = out.kept[i]
        assert np.array_equal(key, ref[i]["sv"]["key"]), (i, nd.level)
        assert np.array_equal(perm, ref[i]["perm"]), (i, nd.level)
        assert np.array_equal(rad2, ref[i]["rad2"]), (i, nd.level)
    assert out.per_level[1]["splats"] > 0 and out.per_level[2]["splats"] > 0


def test_parent_frames_match_oracle(bs):
    """bs_parent_frames (the frames and child prefix targets of the bottom-up generation)
    equals the oracle's parent_frame / child_target_r2 bit for bit: random child frames,
    dyadic ones, parents of one child and children sharing no corner."""
    g = np.random.default_rng(12)
    mins, scales, kids, res = [], [], [], []
    c = 0
    for k in range(60):
        nk = int(g.integers(1, 12))
        if k % 3 == 0:
            m = g.integers(-8, 8, size=(nk, 3)).astype(np.float32) / 4
            sc = Q / 2.0 ** g.integers(-3, 4, size=nk)
        else:
            m = g.uniform(-100, 100, size=(nk, 3)).astype(np.float32)
            sc = Q / np.exp(g.uniform(np.log(0.01), np.log(50), size=nk))
        mins.append(m)
        scales.append(sc)
        kids.append(list(range(c, c + nk)))
        c += nk
        res.append(int(g.choice([96, 128, 256, 1000, 1024, 4096])))
    mins, scales = np.concatenate(mins), np.concatenate(scales)
    fmin, fs, r2 = bs.parent_frames(mins, scales, kids, res)
    j = 0
    for k, cs in enumerate(kids):
        om, os_ = oracle.parent_frame(mins[cs], scales[cs])
        assert np.array_equal(fmin[k].view(np.uint32), om.view(np.uint32)) and fs[k] == os_, k
        for ci in cs:
            assert r2[j] == oracle.child_target_r2(scales[ci], os_, res[k]), (k, ci)
            j += 1
    with pytest.raises(bs.BsError):
        bs.parent_frames(mins[:2], scales[:2], [[]], [128])
    with pytest.raises(bs.BsError):
        bs.parent_frames(mins[:2], np.array([1.0, -1.0]), [[0, 1]], [128])


def test_prefix_for_radius_batched(bs):
    import torch
    g = np.random.default_rng(4)
    rad2s, ms, r2s, want = [], [], [], []
    for i in range(40):
        pts = np.unique(g.integers(0, 1 << 16, size=(int(g.integers(2, 3000)), 3)), axis=0)
        key = oracle.pack(pts)
        m = int(g.integers(1, len(key) + 1))
        _, r = oracle.greedy(key, 0, max_count=m)
        r2 = int(g.choice([0, r[min(1, m - 1)], r[m // 2], r[-1], 10**12, int(g.integers(0, 1 << 30))]))
        r2s.append(max(r2, 0))
        ms.append(m)
        rad2s.append(torch.from_numpy(r).cuda())
        p = oracle.prefix_for_radius(r, r2s[-1])
        want.append((p, int(r[min(p, m - 1)])))
    p, at = bs.prefix_for_radius_batched(rad2s, ms, r2s)
    assert [(int(a), int(b)) for a, b in zip(p, at)] == want
    for i in (0, 7, 39):
        assert bs.prefix_for_radius(rad2s[i], r2s[i]) == want[i][0]
