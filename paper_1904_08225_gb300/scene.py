"""Scene-scale driver: every node of a production-line scene sampled and ordered on the GPU.

The scene (workloads.scene_nodes) has one node per part, one per group of consecutive
parts and one per line; each node's triangles are regenerated on the device from the
scene seed (bs_scene_generate) when its wave runs, so the scene's triangles are never
all resident.  A node is sampled from the six axis directions at a resolution set by
its level and ordered exactly, keeping the first min(200k, triangles / 2) surfels -- the
per-object bound of the paper's evaluation (Sec. 5).  Waves of nodes go through
bs_sample_visible_batched and bs_order_batched.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import bs
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
        keep=(), leaf_wave: int = 2048, group_wave: int = 32, levels=(0, 1, 2), level_res=None) -> SceneResult:
    """Samples and orders every node; returns totals and the outputs of the nodes in `keep`.

    Node i's ordering starts from the Philox start of (seed, part_id=i)."""
    import torch
    dirs = W.AXIS_DIRS
    nodes = W.scene_nodes(lines, per_line, group)
    keep = set(keep)
    res = SceneResult()
    tp = _tris_per_part(nboxes, ncyl)
    vp = _verts_per_part(nboxes, ncyl)
    torch.cuda.synchronize()
    t0 = time.perf_counter()

    lres = {**LEVEL_RES, **(level_res or {})}

    def finish(idx_list, meshes, level):
        r = lres[level]
        sv = bs.sample_visible_batched(meshes, [r] * len(meshes), dirs)
        ntri = [int(m[1].shape[0]) for m in meshes]
        mc = [node_bound(t, s["n"]) for t, s in zip(ntri, sv)]
        live = [j for j in range(len(sv)) if mc[j] > 0]
        orders = [None] * len(sv)
        got = bs.order_batched([sv[j]["key"] for j in live], seeds=[seed] * len(live),
                               part_ids=[idx_list[j] for j in live], max_counts=[mc[j] for j in live],
                               scales=[sv[j]["scale"] for j in live])
        for j, o in zip(live, got):
            orders[j] = o
        lv = res.per_level.setdefault(level, {"nodes": 0, "sampled": 0, "ordered": 0, "triangles": 0})
        for i, s, o, m, t in zip(idx_list, sv, orders, mc, ntri):
            res.surfels_sampled += s["n"]
            res.surfels_ordered += m
            res.triangles += t
            lv["nodes"] += 1
            lv["sampled"] += s["n"]
            lv["ordered"] += m
            lv["triangles"] += t
            if i in keep:
                perm, rad2 = (o[0].cpu().numpy().view(np.uint32), o[1].cpu().numpy()) if o else (None, None)
                res.kept[i] = (s["key"].cpu().numpy().view(np.uint64), perm, rad2)
        res.nodes += len(idx_list)

    by_level = {0: [], 1: [], 2: []}
    for i, nd in enumerate(nodes):
        by_level[nd.level].append(i)
    def level_done(level, t):
        torch.cuda.synchronize()
        if level in res.per_level:
            res.per_level[level]["seconds"] = time.perf_counter() - t

    if 0 in levels:
        tl = time.perf_counter()
        leaves = by_level[0]
        for w in range(0, len(leaves), leaf_wave):
            idx = leaves[w:w + leaf_wave]
            parts = [nodes[i].parts(per_line)[0] for i in idx]
            xyz, tri, rgb = bs.scene_generate(seed, parts, nboxes, ncyl, local_indices=True)
            meshes = [(xyz[q * vp:(q + 1) * vp], tri[q * tp:(q + 1) * tp], rgb[q * tp:(q + 1) * tp])
                      for q in range(len(idx))]
            finish(idx, meshes, 0)
            del xyz, tri, rgb, meshes
        level_done(0, tl)
    for level, wave in ((1, group_wave), (2, 1)):
        if level not in levels:
            continue
        tl = time.perf_counter()
        ids = by_level[level]
        for w in range(0, len(ids), wave):
            idx = ids[w:w + wave]
            meshes = [bs.scene_generate(seed, nodes[i].parts(per_line), nboxes, ncyl) for i in idx]
            finish(idx, meshes, level)
            del meshes
        level_done(level, tl)
    torch.cuda.synchronize()
    res.seconds = time.perf_counter() - t0
    return res
