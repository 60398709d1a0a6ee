"""Scene-scale driver: every node of a production-line scene sampled and ordered on the GPU.

The scene (workloads.scene_nodes) has one node per part, one per group of consecutive
parts and one per line; each node's triangles are regenerated on the device from the
scene seed (bs_scene_generate) when its wave runs, so the scene's triangles are never
all resident.  A node is sampled from the six axis directions at a resolution set by
its level and ordered exactly, keeping the first min(200k, triangles / 2) surfels -- the
per-object bound of the paper's evaluation (Sec. 5).  Waves of nodes go through
bs_sample_visible_batched and bs_order_batched on two alternating streams, so one wave's
ordering overlaps the next wave's generation and sampling.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import bs
from . import shard
from . import workloads as W

# Raster resolution per node level.  Node images are squares over the node's cube extent
# (the quantisation is isotropic), so a level-1 group (50 parts in a row) gets 1024 pixels
# and a whole line 4096, the most one call takes.
LEVEL_RES = {0: 128, 1: 1024, 2: 4096}
NODE_BOUND = 200_000


@dataclass
class SceneResult:
    nodes: int = 0
    triangles: int = 0
    surfels_sampled: int = 0
    surfels_ordered: int = 0
    seconds: float = 0.0
    per_level: dict = field(default_factory=dict)
    kept: dict = field(default_factory=dict)  # node index -> (keys, perm, rad2) on the host


def node_bound(ntris: int, nsampled: int) -> int:
    """Surfels kept for a node: min(200k, triangles / 2), at most what was sampled (Sec. 5)."""
    return min(NODE_BOUND, ntris // 2, nsampled)


def _tris_per_part(nboxes, ncyl):
    return W.BOX_TRIS * nboxes + W.CYL_TRIS * ncyl


def _verts_per_part(nboxes, ncyl):
    return W.BOX_VERTS * nboxes + W.CYL_VERTS * ncyl


def run(seed: int = 0, lines: int = 20, per_line: int = 2500, group: int = 50, nboxes: int = 200, ncyl: int = 50,
        keep=(), leaf_wave: int = 2048, group_wave: int = 32, levels=(0, 1, 2), level_res=None, world: int = 1,
        rank: int = 0) -> SceneResult:
    """Samples and orders every node; returns totals and the outputs of the nodes in `keep`.

    Node i's ordering starts from the Philox start of (seed, part_id=i), so a node's result
    does not depend on which rank orders it.  With world > 1 this rank takes only its
    share of each level's nodes: the longest-processing-time assignment by triangle count
    (shard.lpt_assign), no collective on the data path."""
    import torch
    dirs = W.AXIS_DIRS
    nodes = W.scene_nodes(lines, per_line, group)
    keep = set(keep)
    res = SceneResult()
    tp = _tris_per_part(nboxes, ncyl)
    vp = _verts_per_part(nboxes, ncyl)
    lres = {**LEVEL_RES, **(level_res or {})}
    torch.cuda.synchronize()
    t0 = time.perf_counter()

    def wave(level, idx, counts):
        """Generates the nodes idx (node j holds counts[j] parts) into one packed mesh, then
        samples and orders them with one batched call each."""
        counts = np.asarray(counts, np.int64)
        pstart = np.concatenate([[0], np.cumsum(counts)])
        tot = int(pstart[-1])
        dev = torch.device("cuda")
        xyz = torch.empty((tot * vp, 3), dtype=torch.float32, device=dev)
        tri = torch.empty((tot * tp, 3), dtype=torch.int32, device=dev)
        rgb = torch.empty((tot * tp, 3), dtype=torch.uint8, device=dev)
        if np.all(counts == 1):
            bs.scene_generate(seed, [nodes[i].parts(per_line)[0] for i in idx], nboxes, ncyl, local_indices=True,
                              out=(xyz, tri, rgb))
        else:
            for j, i in enumerate(idx):  # node-local vertex indices: one call per node
                a, b = int(pstart[j]), int(pstart[j + 1])
                bs.scene_generate(seed, nodes[i].parts(per_line), nboxes, ncyl,
                                  out=(xyz[a * vp:b * vp], tri[a * tp:b * tp], rgb[a * tp:b * tp]))
        ntris = counts * tp
        sv = bs.sample_visible_packed(xyz, tri, rgb, pstart[:-1] * vp, counts * vp, pstart[:-1] * tp, ntris,
                                      lres[level], dirs)
        del xyz, tri, rgb
        n = sv["n"]
        mc = np.minimum(np.minimum(NODE_BOUND, ntris // 2), n)
        live = np.nonzero(mc > 0)[0]
        idx = np.asarray(idx, np.int64)
        perm, rad2, _, mofs = bs.order_packed(sv["key"], sv["ofs"][live], n[live], max_counts=mc[live], seeds=seed,
                                              part_ids=idx[live], scales=sv["scale"][live])
        lv = res.per_level.setdefault(level, {"nodes": 0, "sampled": 0, "ordered": 0, "triangles": 0})
        lv["nodes"] += len(idx)
        lv["sampled"] += int(n.sum())
        lv["ordered"] += int(mc.sum())
        lv["triangles"] += int(ntris.sum())
        res.nodes += len(idx)
        res.surfels_sampled += int(n.sum())
        res.surfels_ordered += int(mc.sum())
        res.triangles += int(ntris.sum())
        slot = {int(j): k for k, j in enumerate(live)}
        for j, i in enumerate(idx.tolist()):
            if i in keep:
                a = int(sv["ofs"][j])
                key = sv["key"][a:a + int(n[j])].cpu().numpy().view(np.uint64)
                if j in slot:
                    lo, hi = int(mofs[slot[j]]), int(mofs[slot[j] + 1])
                    res.kept[i] = (key, perm[lo:hi].cpu().numpy().view(np.uint32), rad2[lo:hi].cpu().numpy())
                else:
                    res.kept[i] = (key, None, None)

    by_level = {0: [], 1: [], 2: []}
    for i, nd in enumerate(nodes):
        by_level[nd.level].append(i)
    if world > 1:
        for lv_, ids_ in by_level.items():
            by_level[lv_] = [ids_[j] for j in shard.shard([nodes[i].count * tp for i in ids_], world, rank)]
    # leaves in waves of single parts, groups in waves of nodes, one line at a time.  Waves
    # alternate between two streams: a wave's sampling call returns once its surfels exist
    # and its ordering then runs on the GPU while the next wave is generated and sampled.
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for st in streams:
        st.wait_stream(torch.cuda.current_stream())
    for level, wsize in ((0, leaf_wave), (1, group_wave), (2, 1)):
        if level not in levels:
            continue
        tl = time.perf_counter()
        ids = by_level[level]
        for w in range(0, len(ids), wsize):
            idx = ids[w:w + wsize]
            with torch.cuda.stream(streams[(w // wsize) % 2]):
                wave(level, idx, [nodes[i].count for i in idx])
        torch.cuda.synchronize()
        if level in res.per_level:
            res.per_level[level]["seconds"] = time.perf_counter() - tl
    torch.cuda.synchronize()
    res.seconds = time.perf_counter() - t0
    return res


# ---------------------------------------------------------------------------
# Bottom-up generation (Sec. 3.4): groups are sampled from their parts' surfels and
# lines from their groups' surfels, each surfel drawn as an oriented disc
# (bs_sample_splats), instead of from triangles.
# ---------------------------------------------------------------------------
def _splat_level(children, nodes_children, level, seed, node_ids, res, ntris, out_res: SceneResult, keep):
    """Samples parent nodes from child outputs and orders them; returns the parents' outputs.

    children: list of dicts (key, nrm, rgb, perm, rad2, m, bbox_min, scale); nodes_children:
    per parent the indices of its children."""
    # the parents' frames and each child's prefix target, from the library (Sec. 3.4 / 4.1)
    listed = sorted({c for cs in nodes_children for c in cs})
    cmin = np.zeros((len(children), 3), np.float32)
    cscale = np.ones(len(children), np.float64)
    for c in listed:
        cmin[c] = children[c]["bbox_min"]
        cscale[c] = children[c]["scale"]
    fmin, fscale, targets = bs.parent_frames(cmin, cscale, nodes_children, [res] * len(nodes_children))
    frames = [(fmin[k], float(fscale[k])) for k in range(len(nodes_children))]
    order_c = [(k, c) for k, cs in enumerate(nodes_children) for c in cs]
    p, r2_at = bs.prefix_for_radius_batched([children[c]["rad2"] for _, c in order_c],
                                            [children[c]["m"] for _, c in order_c], targets)
    sets = []
    for (k, c), pk, rk in zip(order_c, p, r2_at):
        ch = children[c]
        sets.append(dict(key=ch["key"], nrm=ch["nrm"], rgb=ch["rgb"], perm=ch["perm"], n=int(pk),
                         bbox_min=list(ch["bbox_min"]), scale=ch["scale"], r2=int(rk), node=k))
    sv = bs.sample_splats(sets, [(f[0], f[1], res) for f in frames], W.AXIS_DIRS)
    mc = [node_bound(t, s["n"]) for t, s in zip(ntris, sv)]
    live = [k for k in range(len(sv)) if mc[k] > 0]
    got = bs.order_batched([sv[k]["key"] for k in live], seeds=[seed] * len(live),
                           part_ids=[node_ids[k] for k in live], max_counts=[mc[k] for k in live],
                           scales=[sv[k]["scale"] for k in live])
    outs = [None] * len(sv)
    for k, o in zip(live, got):
        outs[k] = dict(key=sv[k]["key"], nrm=sv[k]["nrm"], rgb=sv[k]["rgb"], perm=o[0], rad2=o[1], m=mc[k],
                       bbox_min=sv[k]["bbox_min"], scale=sv[k]["scale"])
    lv = out_res.per_level.setdefault(level, {"nodes": 0, "sampled": 0, "ordered": 0, "triangles": 0, "splats": 0})
    lv["nodes"] += len(sv)
    lv["sampled"] += sum(s["n"] for s in sv)
    lv["ordered"] += sum(mc)
    lv["triangles"] += sum(ntris)
    lv["splats"] += int(np.sum(p))
    out_res.nodes += len(sv)
    out_res.surfels_sampled += sum(s["n"] for s in sv)
    out_res.surfels_ordered += sum(mc)
    out_res.triangles += sum(ntris)
    for k, i in enumerate(node_ids):
        if i in keep:
            key = sv[k]["key"].cpu().numpy().view(np.uint64)
            if outs[k] is not None:
                out_res.kept[i] = (key, outs[k]["perm"].cpu().numpy().view(np.uint32), outs[k]["rad2"].cpu().numpy())
            else:
                out_res.kept[i] = (key, None, None)
    return outs


def run_hierarchical(seed: int = 0, lines: int = 20, per_line: int = 2500, group: int = 50, nboxes: int = 200,
                     ncyl: int = 50, keep=(), groups_per_wave: int = 25, level_res=None) -> SceneResult:
    """The scene of run() generated bottom-up: parts from their triangles (as in run()),
    every group from its parts' surfel prefixes and every line from its groups' prefixes,
    drawn as oriented discs.  A child contributes the shortest prefix of its ordering that
    reaches all its surfels within one pixel step of the parent's raster, each surfel a
    disc of that prefix's covering radius.  Waves of parts alternate between two streams:
    a wave's parts are ordered while the next wave's parts are generated and sampled, and
    its groups are drawn while the next wave's parts are ordered."""
    import torch
    nodes = W.scene_nodes(lines, per_line, group)
    keep = set(keep)
    res = SceneResult()
    tp = _tris_per_part(nboxes, ncyl)
    vp = _verts_per_part(nboxes, ncyl)
    lres = {**LEVEL_RES, **(level_res or {})}
    index = {(nd.line, nd.first, nd.count, nd.level): i for i, nd in enumerate(nodes)}
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for st in streams:
        st.wait_stream(torch.cuda.current_stream())
    waves = []
    for l in range(lines):
        groups = [(s0, min(group, per_line - s0)) for s0 in range(0, per_line, group)]
        for w in range(0, len(groups), groups_per_wave):
            waves.append((l, groups[w:w + groups_per_wave]))
    waves_left = {l: sum(1 for wl, _ in waves if wl == l) for l in range(lines)}
    line_groups = {l: [] for l in range(lines)}

    def leaf_stage(l, gw):
        """Parts of the wave from triangles: generated, sampled (returns once sampled) and
        ordered (left running on the current stream)."""
        slots = [s0 for g0, cnt in gw for s0 in range(g0, g0 + cnt)]
        leaf_ids = [index[(l, s0, 1, 0)] for s0 in slots]
        npart = len(slots)
        dev = torch.device("cuda")
        xyz = torch.empty((npart * vp, 3), dtype=torch.float32, device=dev)
        tri = torch.empty((npart * tp, 3), dtype=torch.int32, device=dev)
        rgb = torch.empty((npart * tp, 3), dtype=torch.uint8, device=dev)
        bs.scene_generate(seed, [(l * per_line + s0, l, s0) for s0 in slots], nboxes, ncyl, local_indices=True,
                          out=(xyz, tri, rgb))
        q = np.arange(npart, dtype=np.int64)
        sv = bs.sample_visible_packed(xyz, tri, rgb, q * vp, [vp] * npart, q * tp, [tp] * npart, lres[0],
                                      W.AXIS_DIRS)
        del xyz, tri, rgb
        n = sv["n"]
        mc = np.minimum(np.minimum(NODE_BOUND, tp // 2), n)
        perm, rad2, _, mofs = bs.order_packed(sv["key"], sv["ofs"], n, max_counts=mc, seeds=seed,
                                              part_ids=leaf_ids, scales=sv["scale"])
        lv = res.per_level.setdefault(0, {"nodes": 0, "sampled": 0, "ordered": 0, "triangles": 0})
        lv["nodes"] += npart
        lv["sampled"] += int(n.sum())
        lv["ordered"] += int(mc.sum())
        lv["triangles"] += npart * tp
        res.nodes += npart
        res.surfels_sampled += int(n.sum())
        res.surfels_ordered += int(mc.sum())
        res.triangles += npart * tp
        leaves = []
        for j in range(npart):
            a, b = int(sv["ofs"][j]), int(sv["ofs"][j]) + int(n[j])
            lo, hi = int(mofs[j]), int(mofs[j + 1])
            leaves.append(dict(key=sv["key"][a:b], nrm=sv["nrm"][a:b], rgb=sv["rgb"][a:b], perm=perm[lo:hi],
                               rad2=rad2[lo:hi], m=int(mc[j]), bbox_min=sv["bbox_min"][j], scale=float(sv["scale"][j])))
        return dict(l=l, gw=gw, leaves=leaves, leaf_ids=leaf_ids, stream=torch.cuda.current_stream())

    def group_stage(wv):
        """Groups of a wave from its parts' discs; the line once all its groups exist."""
        l, gw, leaves = wv["l"], wv["gw"], wv["leaves"]
        for j, i in enumerate(wv["leaf_ids"]):
            if i in keep:
                res.kept[i] = (leaves[j]["key"].cpu().numpy().view(np.uint64),
                               leaves[j]["perm"].cpu().numpy().view(np.uint32), leaves[j]["rad2"].cpu().numpy())
        members, j0 = [], 0
        for g0, cnt in gw:  # parts with no surfels have nothing to draw
            members.append([j for j in range(j0, j0 + cnt) if leaves[j]["m"] > 0])
            j0 += cnt
        group_ids = [index[(l, g0, cnt, 1)] for g0, cnt in gw]
        line_groups[l] += _splat_level(leaves, members, 1, seed, group_ids, lres[1], [cnt * tp for _, cnt in gw],
                                       res, keep)
        waves_left[l] -= 1
        if waves_left[l] == 0:
            kids = [g for g in line_groups.pop(l) if g is not None]
            # the line's groups were ordered on both streams: wait for them, and keep their
            # memory from being reused before this stream is done with it
            cur = torch.cuda.current_stream()
            for st in streams:
                if st != cur:
                    cur.wait_stream(st)
            for g in kids:
                for f in ("key", "nrm", "rgb", "perm", "rad2"):
                    g[f].record_stream(cur)
            _splat_level(kids, [list(range(len(kids)))], 2, seed, [index[(l, 0, per_line, 2)]], lres[2],
                         [per_line * tp], res, keep)

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pending = None
    for w, (l, gw) in enumerate(waves):
        with torch.cuda.stream(streams[w % 2]):
            cur = leaf_stage(l, gw)
        if pending is not None:
            with torch.cuda.stream(pending["stream"]):
                group_stage(pending)
        pending = cur
    if pending is not None:
        with torch.cuda.stream(pending["stream"]):
            group_stage(pending)
    torch.cuda.synchronize()
    res.seconds = time.perf_counter() - t0
    return res
