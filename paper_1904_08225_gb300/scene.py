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
