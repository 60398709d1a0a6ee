#!/usr/bin/env python3
"""Benchmark: surfels sampled and progressively ordered per second on one GB300.

Workload (the batched-ordering configuration): 4096 seeded tori with lognormal
triangle counts (2k-50k) and lognormal target surfel counts (median 20k, 1k-500k,
about 100M surfels in total), each sampled from the 6 axis directions at a
per-part resolution and then ordered exactly.  One step = one bs_sample_visible_batched
call over every part followed by one bs_order_batched over all parts (every row of
the hot path: quantise, raster, resolve, dedup, ordering, radius).

Printed JSON line (rank 0):
  value      surfels/s of the device-resident step (inputs already in HBM)
  e2e        the same with the meshes copied from pinned host memory and the
             ordered surfels read back inside the timed region
  order_only batched vs plain (one bs_order launch per part) ordering throughput
  served     p50/p99/p999 latency of a short Poisson request trace through bs_server
  roofline   the ordering loop kernel's algorithmic bytes / its event-timed duration
  cpu_baseline  the CPU oracle on a bounded sample of the same workload
With --impl reference the CPU oracle is the timed arm (same metric and config).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1904_08225_gb300 import workloads as W  # noqa: E402

METRIC = "surfels ordered/s (sample + exact greedy order, batched)"
UNIT = "surfels/s"

# Algorithmic work of the exact ordering, per part of N surfels (the update sweep
# must examine every unchosen point inside the new point's ball): visits/N and
# improved/N fitted as a + b*ln(N) over seeded torus parts of the batch generator
# by oracle/fit_visits.py (exact counts from the O(N^2) oracle).
VISITS_FIT = (-4.25, 2.06)
IMPROVED_FIT = (-1.06, 0.74)
BYTES_PER_VISIT = 16   # 8 B key + 8 B D read
BYTES_PER_IMPROVE = 8  # 8 B D write
BYTES_OUT = 16         # perm 4 + rad2 8 + radius 4
# DRAM bytes (read + write) per surfel ordered of the dominant launch (the ordering of the
# non-lead parts, k_order_rounds<1024, 1>), from an ncu capture of that launch in the
# full-size bench step: profiles/k_order_rounds_traffic_bench4096_rest.md.  Must be
# re-measured (or set to None) whenever k_order_rounds changes.
DRAM_BYTES_PER_SURFEL = 2013.6


def band_layout(ns, thresholds):
    """Bands of parts by surfel count and the layout that makes each band contiguous.

    thresholds: descending surfel counts; band j (j < len(thresholds)) holds the parts with
    thresholds[j] <= n < thresholds[j - 1] (no upper bound for j = 0), the last band the
    rest.  Returns (orig, band): orig[i] = seeded index of the part at position i (band
    order, seeded order within a band), band[i] = its band (non-decreasing)."""
    ns = np.asarray(ns)
    bounds = [float("inf")] + list(thresholds)
    band0 = np.array([next((j for j in range(len(thresholds)) if bounds[j + 1] <= n < bounds[j]), len(thresholds))
                      for n in ns], np.int64)
    orig = np.array(sorted(range(len(ns)), key=lambda i: (band0[i], i)), np.int64)
    return orig, band0[orig]


def seeded_positions(orig):
    """at[s] = position of the part whose seeded index is s (the inverse of orig)."""
    orig = np.asarray(orig)
    at = np.empty(len(orig), np.int64)
    at[orig] = np.arange(len(orig))
    return at


def algorithmic_bytes(n: int) -> float:
    """Bytes the ordering of an N-surfel part must move (init sweep + update sweeps + outputs)."""
    if n <= 1:
        return float(BYTES_OUT * n + BYTES_PER_VISIT * n)
    ln = math.log(n)
    visits = max(0.0, VISITS_FIT[0] + VISITS_FIT[1] * ln) * n
    improved = max(0.0, IMPROVED_FIT[0] + IMPROVED_FIT[1] * ln) * n
    return BYTES_PER_VISIT * (visits + n) + BYTES_PER_IMPROVE * improved + BYTES_OUT * n


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_specs(nparts: int, seed: int, rank: int):
    """Each rank orders its own seeded batch (weak scaling: parts are independent, no
    data-path collective)."""
    return W.batch_parts(nparts, seed=seed + 7919 * rank)


def max_over_ranks(ms: float, dist, device) -> float:
    """The step time the job is charged: the slowest rank's."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle as it stands, on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample_parts(specs, budget_s: float, seed: int):
    """A seeded sample of parts whose estimated oracle time (O(N^2) greedy, about
    9 ns per point pair per core) fits budget_s seconds; parts too big alone are skipped."""
    g = np.random.default_rng(seed)
    cores = max(1, os.cpu_count() or 1)

    def cost(n):
        return 9e-9 * n * n / cores + 0.05

    picked, est = [], 0.0
    for i in g.permutation(len(specs)):
        c = cost(specs[i].n_target)
        if est + c > budget_s:
            continue
        picked.append(int(i))
        est += c
    if not picked:
        picked = [int(np.argmin([sp.n_target for sp in specs]))]
    return picked


def run_oracle_parts(specs, idx, nthreads):
    import oracle
    tot = 0
    t0 = time.perf_counter()
    for i in idx:
        sp = specs[i]
        m = sp.mesh()
        sv, mn, s = oracle.sample_mesh(m, W.AXIS_DIRS, sp.res)
        k = sv["key"]
        st = oracle.start_index(len(k), seed=0, part_id=i)
        oracle.greedy(k, st, nthreads=nthreads)
        tot += len(k)
    return tot, time.perf_counter() - t0


def reference_arm(args, specs, world, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    nthreads = oracle.num_threads()
    idx = oracle_sample_parts(specs, args.cpu_budget_s, seed=args.seed)
    for _ in range(args.warmup):
        run_oracle_parts(specs, idx[:1], nthreads)
    tot, dt = 0, 0.0
    for _ in range(args.steps):
        n, t = run_oracle_parts(specs, idx, nthreads)
        tot += n
        dt += t
    v = tot / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": config_dict(args, specs),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": f"{len(idx)} of {len(specs)} parts (seeded), {tot // args.steps} surfels per step; "
                                   f"oracle sample_visible + O(N^2) greedy, OpenMP"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(args, specs):
    return {"workload": f"batched ordering: {len(specs)} tori, lognormal tris 2k-50k, lognormal surfels "
                        f"(median 20k, 1k-500k), 6 axis views at 16^2-1024^2, exact greedy order",
            "parts": len(specs), "seed": args.seed, "dirs": 6,
            "l2": "inputs larger than L2 (meshes + keys ~ GBs, no flush needed)"} | \
        ({"tuning": dict(kv.split("=") for kv in args.tune)} if args.tune else {})


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--parts", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--plain-parts", type=int, default=512, help="parts timed one launch each for the plain path")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[500.0, 1000.0, 2000.0, 4000.0, 8000.0])
    ap.add_argument("--serve-window", type=float, default=2.0, help="seconds of arrivals per offered rate")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true", help="skip plain / served / cpu baseline legs")
    ap.add_argument("--legs", default="order_only,autotune,served,table2,scene,cpu_baseline",
                    help="comma list of the extra legs to run (order_only, autotune, served, table2, scene, "
                         "cpu_baseline)")
    ap.add_argument("--scene-lines", type=int, default=20, help="production lines of the scene leg (0 skips it)")
    ap.add_argument("--scene-per-line", type=int, default=2500)
    ap.add_argument("--lead-min", type=int, nargs="+", default=[350_000, 150_000],
                    help="surfel-count thresholds, largest first: the parts of at least each threshold (and below "
                         "the previous one) are sampled and then ordered on a stream of their own, largest group "
                         "first, before the rest (0 = one sample call and one order call for all parts)")
    ap.add_argument("--tune", action="append", default=[], metavar="KNOB=VALUE",
                    help="bs_set_tuning launch-shape knob for the run (repeatable)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    specs = rank_specs(args.parts, args.seed, rank)
    if args.impl == "reference":
        return reference_arm(args, specs, world, rank)

    import torch
    from paper_1904_08225_gb300 import bs
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = bs.load()
    for kv in args.tune:
        name, val = kv.split("=")
        bs.set_tuning(name, int(val))
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)

    # ---- inputs: all meshes packed in one buffer (host pinned + device copy) ----
    specs0 = specs
    meshes = [sp.mesh() for sp in specs]

    def pack(meshes):
        vofs = np.cumsum([0] + [m.nverts for m in meshes])
        tofs = np.cumsum([0] + [m.ntris for m in meshes])
        xyz_h = torch.from_numpy(np.concatenate([m.xyz for m in meshes])).pin_memory()
        tri_h = torch.from_numpy(np.concatenate([m.tri for m in meshes]).view(np.int32)).pin_memory()
        rgb_h = torch.from_numpy(np.concatenate([m.rgb for m in meshes])).pin_memory()
        return vofs, tofs, xyz_h, tri_h, rgb_h, xyz_h.to(dev), tri_h.to(dev), rgb_h.to(dev)

    vofs, tofs, xyz_h, tri_h, rgb_h, xyz_d, tri_d, rgb_d = pack(meshes)
    h2d_bytes = xyz_h.numel() * 4 + tri_h.numel() * 4 + rgb_h.numel()
    dirs = (bs.Dir * 6)(*[bs.Dir(int(a), int(b), int(c)) for a, b, c in W.AXIS_DIRS])

    # first pass learns each part's surfel count (deterministic) to size the outputs
    caps = [6 * sp.res * sp.res for sp in specs]
    coff = np.cumsum([0] + caps)
    key_all = torch.empty(int(coff[-1]), dtype=torch.int64, device=dev)
    nrm_all = torch.empty((int(coff[-1]), 3), dtype=torch.int16, device=dev)
    rgb_all = torch.empty((int(coff[-1]), 3), dtype=torch.uint8, device=dev)
    src_all = torch.empty(int(coff[-1]), dtype=torch.int32, device=dev)
    import ctypes as C
    cs = C.c_void_p(stream.cuda_stream)
    mesh_structs, out_structs = [], []
    for i, sp in enumerate(specs):
        mesh_structs.append(bs.Mesh(xyz_d.data_ptr() + int(vofs[i]) * 12, meshes[i].nverts,
                                    tri_d.data_ptr() + int(tofs[i]) * 12, meshes[i].ntris,
                                    rgb_d.data_ptr() + int(tofs[i]) * 3, 1))
        o = int(coff[i])
        out_structs.append(bs.Surfels(key_all.data_ptr() + 8 * o, nrm_all.data_ptr() + 6 * o,
                                      rgb_all.data_ptr() + 3 * o, src_all.data_ptr() + 4 * o, 0, caps[i],
                                      (C.c_float * 3)(), 0.0))

    mesh_arr = (bs.Mesh * len(specs))(*mesh_structs)
    out_arr = (bs.Surfels * len(specs))(*out_structs)
    res_arr = (C.c_int * len(specs))(*[sp.res for sp in specs])

    def sample_all():
        st = lib.bs_sample_visible_batched(mesh_arr, res_arr, len(specs), dirs, 6, out_arr, cs)
        if st != bs.BS_OK:
            raise bs.BsError(st, "bs_sample_visible_batched", bs.last_error())

    sample_all()
    ns = np.array([out_arr[i].n for i in range(len(specs))], np.int64)
    total = int(ns.sum())
    # Parts in band order (the largest-band parts first, then the next band, then the
    # rest; index order within a band): each band's meshes, sampled records and ordered
    # outputs are then contiguous, so the end-to-end step moves them band by band and
    # overlaps the copies with the other bands' work.  orig[i] = the part's seeded index.
    thresholds = sorted([t for t in args.lead_min if t > 0], reverse=True)
    orig, band = band_layout(ns, thresholds)
    if not np.array_equal(orig, np.arange(len(specs))):
        specs = [specs[i] for i in orig]
        meshes = [meshes[i] for i in orig]
        ns = ns[orig]
        del xyz_d, tri_d, rgb_d
        vofs, tofs, xyz_h, tri_h, rgb_h, xyz_d, tri_d, rgb_d = pack(meshes)
        mesh_structs = [bs.Mesh(xyz_d.data_ptr() + int(vofs[i]) * 12, meshes[i].nverts,
                                tri_d.data_ptr() + int(tofs[i]) * 12, meshes[i].ntris,
                                rgb_d.data_ptr() + int(tofs[i]) * 3, 1) for i in range(len(specs))]
        mesh_arr = (bs.Mesh * len(specs))(*mesh_structs)
        res_arr = (C.c_int * len(specs))(*[sp.res for sp in specs])
    # the counts are deterministic: size every part's outputs exactly, so the surfel records
    # of all parts form one contiguous array (one copy per field for the e2e read-back)
    coff = np.cumsum([0] + list(ns))
    key_all = torch.empty(total, dtype=torch.int64, device=dev)
    nrm_all = torch.empty((total, 3), dtype=torch.int16, device=dev)
    rgb_all = torch.empty((total, 3), dtype=torch.uint8, device=dev)
    src_all = torch.empty(total, dtype=torch.int32, device=dev)
    out_arr = (bs.Surfels * len(specs))(*[
        bs.Surfels(key_all.data_ptr() + 8 * int(coff[i]), nrm_all.data_ptr() + 6 * int(coff[i]),
                   rgb_all.data_ptr() + 3 * int(coff[i]), src_all.data_ptr() + 4 * int(coff[i]), 0, int(ns[i]),
                   (C.c_float * 3)(), 0.0) for i in range(len(specs))])
    sample_all()
    out_structs = [out_arr[i] for i in range(len(specs))]
    assert np.array_equal(np.array([o.n for o in out_structs], np.int64), ns)
    pofs = np.cumsum([0] + list(ns))
    perm_all = torch.empty(total, dtype=torch.int32, device=dev)
    rad2_all = torch.empty(total, dtype=torch.int64, device=dev)
    radius_all = torch.empty(total, dtype=torch.float32, device=dev)
    P = len(specs)
    parts = (bs.Surfels * P)()
    opts = (bs.OrderOpts * P)()
    pp, rp, fp = (C.c_void_p * P)(), (C.c_void_p * P)(), (C.c_void_p * P)()
    for i in range(P):
        o = out_structs[i]
        parts[i] = bs.Surfels(o.key, None, None, None, o.n, o.n, (C.c_float * 3)(), o.scale)
        opts[i] = bs.OrderOpts(0, int(orig[i]), -1, 0)
        pp[i] = perm_all.data_ptr() + 4 * int(pofs[i])
        rp[i] = rad2_all.data_ptr() + 8 * int(pofs[i])
        fp[i] = radius_all.data_ptr() + 4 * int(pofs[i])

    def order_all():
        st = lib.bs_order_batched(parts, P, opts, C.cast(pp, C.c_void_p), C.cast(rp, C.c_void_p),
                                  C.cast(fp, C.c_void_p), cs)
        if st != bs.BS_OK:
            raise bs.BsError(st, "bs_order_batched", bs.last_error())

    # Pipelined step: the parts of at least --lead-min surfels (whose ordering is the
    # longest single chain) are sampled first and ordered on a second stream while the
    # others are sampled and ordered on the main stream.  Every part is sampled and
    # ordered exactly once per step; both streams join the main stream at the end.
    leads = [[i for i in range(P) if band[i] == j] for j in range(len(thresholds))]
    rest = [i for i in range(P) if band[i] == len(thresholds)]

    def subset(idx):
        k = len(idx)
        return dict(k=k, mesh=(bs.Mesh * k)(*[mesh_structs[i] for i in idx]),
                    res=(C.c_int * k)(*[specs[i].res for i in idx]),
                    out=(bs.Surfels * k)(*[out_structs[i] for i in idx]),
                    parts=(bs.Surfels * k)(*[parts[i] for i in idx]),
                    opts=(bs.OrderOpts * k)(*[opts[i] for i in idx]),
                    pp=(C.c_void_p * k)(*[pp[i] for i in idx]), rp=(C.c_void_p * k)(*[rp[i] for i in idx]),
                    fp=(C.c_void_p * k)(*[fp[i] for i in idx]))
    sub_leads, sub_rest = [subset(grp) for grp in leads], subset(rest)
    lead_streams = [torch.cuda.Stream(device=dev) for _ in leads]
    cs_leads = [C.c_void_p(st_.cuda_stream) for st_ in lead_streams]

    marks = {}

    def run_subset(sb, csx, tag, tstream, ready=None):
        if sb["k"] == 0:
            return
        if ready is not None:
            tstream.wait_event(ready)
        st = lib.bs_sample_visible_batched(sb["mesh"], sb["res"], sb["k"], dirs, 6, sb["out"], csx)
        if st != bs.BS_OK:
            raise bs.BsError(st, "bs_sample_visible_batched", bs.last_error())
        marks[tag + "_sampled"] = torch.cuda.Event(enable_timing=True)
        marks[tag + "_sampled"].record(tstream)
        st = lib.bs_order_batched(sb["parts"], sb["k"], sb["opts"], C.cast(sb["pp"], C.c_void_p),
                                  C.cast(sb["rp"], C.c_void_p), C.cast(sb["fp"], C.c_void_p), csx)
        if st != bs.BS_OK:
            raise bs.BsError(st, "bs_order_batched", bs.last_error())

    def step(ready=None):
        """One step; ready[j] (optional) = event after which band j's meshes are on the device."""
        marks["start"] = torch.cuda.Event(enable_timing=True)
        marks["start"].record(stream)
        # each call returns once its parts are sampled; their ordering runs on while the
        # next groups are sampled and ordered
        for j, (sb, csx, st_) in enumerate(zip(sub_leads, cs_leads, lead_streams)):
            st_.wait_stream(stream)
            run_subset(sb, csx, f"lead{j}", st_, ready[j] if ready else None)
        run_subset(sub_rest, cs, "rest", stream, ready[-1] if ready else None)
        for tag, st_ in [(f"lead{j}_ordered", x) for j, x in enumerate(lead_streams)] + [("rest_ordered", stream)]:
            marks[tag] = torch.cuda.Event(enable_timing=True)
            marks[tag].record(st_)
        for st_ in lead_streams:
            stream.wait_stream(st_)

    def step_breakdown():
        """ms from the step's start to each milestone of the last step (CUDA events)."""
        torch.cuda.synchronize()
        return {k: round(marks["start"].elapsed_time(v), 2) for k, v in marks.items() if k != "start"}

    # e2e: host meshes in, ordered surfels out (perm, rad2, radius, key, nrm, rgb), through
    # the C ABI: bs_sample_order_batched uploads the (pinned, packed) host meshes itself and
    # writes every result into pinned host arrays; one call per band, each on its own
    # stream from its own host thread, so the bands overlap as in the device-resident step
    res_h = {
        "perm": torch.empty(total, dtype=torch.int32).pin_memory(),
        "rad2": torch.empty(total, dtype=torch.int64).pin_memory(),
        "radius": torch.empty(total, dtype=torch.float32).pin_memory(),
        "key": torch.empty(total, dtype=torch.int64).pin_memory(),
        "nrm": torch.empty((total, 3), dtype=torch.int16).pin_memory(),
        "rgb": torch.empty((total, 3), dtype=torch.uint8).pin_memory(),
    }
    d2h_bytes = total * (4 + 8 + 4) + total * (8 + 6 + 3)
    band_rng = [(int(np.searchsorted(band, j, "left")), int(np.searchsorted(band, j, "right")))
                for j in range(len(thresholds) + 1)]
    band_cs = cs_leads + [cs]
    e2e_calls = []
    for (p0, p1), csx in zip(band_rng, band_cs):
        k = p1 - p0
        if k == 0:
            continue
        hm = (bs.Mesh * k)(*[bs.Mesh(xyz_h.data_ptr() + int(vofs[i]) * 12, meshes[i].nverts,
                                     tri_h.data_ptr() + int(tofs[i]) * 12, meshes[i].ntris,
                                     rgb_h.data_ptr() + int(tofs[i]) * 3, 0) for i in range(p0, p1)])
        ho = (bs.PartResult * k)()
        for j, i in enumerate(range(p0, p1)):
            o = int(coff[i])
            ho[j] = bs.PartResult(res_h["key"].data_ptr() + 8 * o, res_h["nrm"].data_ptr() + 6 * o,
                                  res_h["rgb"].data_ptr() + 3 * o, None, res_h["perm"].data_ptr() + 4 * o,
                                  res_h["rad2"].data_ptr() + 8 * o, res_h["radius"].data_ptr() + 4 * o, int(ns[i]))
        e2e_calls.append((hm, (C.c_int * k)(*[specs[i].res for i in range(p0, p1)]), k,
                          (bs.OrderOpts * k)(*[opts[i] for i in range(p0, p1)]), ho, csx))

    def step_e2e():
        errs = []

        def call(args):
            hm, hres, k, hopts, ho, csx = args
            st = lib.bs_sample_order_batched(hm, hres, k, dirs, 6, hopts, ho, 0, csx)
            if st != bs.BS_OK:
                errs.append(bs.BsError(st, "bs_sample_order_batched", bs.last_error()))
        th = [threading.Thread(target=call, args=(a,)) for a in e2e_calls]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errs:
            raise errs[0]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist, dev)

    for _ in range(args.warmup):
        step()
    bs.set_tuning("kernel_timing", 1)
    clocks = Clocks(local)
    clocks.start()
    # dominant kernel (ordering loop) timed per launch with events on its own stream
    loop_ms = []
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
        loop_ms.append(bs.last_launch_ms("order_loop"))
    e1.record(stream)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    breakdown = step_breakdown()
    clk = clocks.stop()
    bs.set_tuning("kernel_timing", 0)
    ms_step = ms / args.steps
    value = world * total / (ms_step / 1e3)

    # e2e through the public API with host buffers
    step_e2e()
    # the host path gives the device-resident step's results, array for array
    torch.cuda.synchronize()
    for name, dv in (("perm", perm_all), ("rad2", rad2_all), ("radius", radius_all), ("key", key_all),
                     ("nrm", nrm_all), ("rgb", rgb_all)):
        if not torch.equal(res_h[name].view(torch.uint8), dv.cpu().view(torch.uint8)):
            raise RuntimeError(f"e2e {name} differs from the device-resident step")
    ms_e2e = timed(step_e2e, args.steps) / args.steps
    e2e_value = world * total / (ms_e2e / 1e3)

    extras = {}
    legs = set(args.legs.split(",")) if not args.no_extras else set()
    if legs and rank == 0:
        if "order_only" in legs:
            # ordering only: batched (one launch) vs plain (one launch per part) on a seeded subset
            ms_b = timed(order_all, 2) / 2
            g = np.random.default_rng(args.seed)
            at = seeded_positions(orig)  # the subset is drawn by seeded part index, whatever the layout
            sub = np.sort(at[g.choice(P, size=min(args.plain_parts, P), replace=False)])
            sub_n = int(ns[sub].sum())

            def plain():
                for i in sub:
                    st = lib.bs_order(C.byref(parts[i]), C.byref(opts[i]), C.c_void_p(pp[i]), C.c_void_p(rp[i]),
                                      C.c_void_p(fp[i]), cs)
                    if st != bs.BS_OK:
                        raise bs.BsError(st, "bs_order", bs.last_error())
            plain()
            ms_p = timed(plain, 1)
            sub_parts = (bs.Surfels * len(sub))(*[parts[i] for i in sub])
            sub_opts = (bs.OrderOpts * len(sub))(*[opts[i] for i in sub])
            spp = (C.c_void_p * len(sub))(*[pp[i] for i in sub])
            srp = (C.c_void_p * len(sub))(*[rp[i] for i in sub])
            sfp = (C.c_void_p * len(sub))(*[fp[i] for i in sub])

            def batched_sub():
                lib.bs_order_batched(sub_parts, len(sub), sub_opts, C.cast(spp, C.c_void_p), C.cast(srp, C.c_void_p),
                                     C.cast(sfp, C.c_void_p), cs)
            batched_sub()
            ms_bs = timed(batched_sub, 1)
            extras["order_only"] = {
                "batched_all_parts": total / (ms_b / 1e3),
                "batched_subset": sub_n / (ms_bs / 1e3),
                "plain_subset": sub_n / (ms_p / 1e3),
                "batched_over_plain": (sub_n / (ms_bs / 1e3)) / (sub_n / (ms_p / 1e3)),
                "subset": f"{len(sub)} seeded parts, {sub_n} surfels, one bs_order launch each on one stream",
                "unit": UNIT,
            }
        if "autotune" in legs:
            # the autotuner over the batch's ordering launch (all parts in one launch)
            from paper_1904_08225_gb300 import autotune
            keys_t = [key_all[int(coff[i]):int(coff[i]) + int(ns[i])] for i in range(P)]
            best, times = autotune.autotune(keys_t, repeats=1, apply=False)
            extras["autotune"] = {"best": {"order_threads": best[0], "order_quarters": best[1],
                                           "order_full_parts": best[2]},
                                  "ms": {f"threads={c[0]},quarters={c[1]},full_parts={c[2]}": round(t, 2)
                                         for c, t in times.items()},
                                  "launch": f"bs_order_batched over all {P} parts"}
        if "served" in legs:
            extras["served"] = serve_leg(bs, key_all, coff, ns, out_structs, args, orig)
        if "table2" in legs:
            extras["paper_table2_shape"] = table2_leg(bs, timed)
        if "scene" in legs and args.scene_lines > 0:
            extras["scene"] = scene_leg(args)
        if "cpu_baseline" in legs:
            extras["cpu_baseline"] = cpu_baseline(specs0, args)

    if rank == 0:
        peak, peak_src = measured_peaks()
        # the dominant launch: the ordering of the non-lead parts (the last timed launch)
        bytes_launch = float(sum(algorithmic_bytes(int(ns[i])) for i in rest))
        loop_avg = float(np.mean(loop_ms))
        achieved = bytes_launch / (loop_avg / 1e3) / 1e9
        # one sampling call: bbox, quantise, setup, raster, cover count, 1-3 scan kernels,
        # resolve, 10 radix passes x (hist, 1-3 scan kernels, scatter), part keys,
        # unique count, scan, 2 unique passes; ordering: init, loop, radius
        nsample_kernels = 64
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": config_dict(args, specs) | {"surfels_per_gpu": total,
                                                  "pipeline": f"parts in surfel-count bands {thresholds} "
                                                              f"({[len(g) for g in leads]} parts) sampled first, "
                                                              f"largest band first, each ordered on its own stream",
                                                  "step_milestones_ms": breakdown},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d_bytes),
                    "d2h_bytes_per_step": int(d2h_bytes)},
            "gpu_launches": args.steps * (nsample_kernels + 3) * (1 + sum(1 for g in leads if g)),
            "roofline": {"bound": "hbm", "kernel": "k_order_rounds", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": (DRAM_BYTES_PER_SURFEL * float(ns[rest].sum())) if DRAM_BYTES_PER_SURFEL else None,
                         "traffic_source": "ncu dram__bytes_read+write of this launch in the full-size step, per surfel",
                         "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback 6800 GB/s",
                         "algorithmic_bytes_per_launch": bytes_launch, "loop_ms_per_launch": loop_avg,
                         "launch": f"bs_order_batched over the {len(rest)} non-lead parts ({int(ns[rest].sum())} surfels)"},
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def serve_leg(bs, key_all, coff, ns, out_structs, args, orig=None):
    """Poisson arrivals of ordering requests (surfel arrays of the sampled parts with
    1k-1M surfels, each with its own seed) through bs_server at several offered rates;
    latency = device completion - submit, on the server's clock.  Requests are drawn by
    the parts' seeded indices (orig[i] = seeded index of the part at position i), so the
    trace does not depend on how the parts are laid out."""
    g = np.random.default_rng(args.seed + 1)
    orig = np.arange(len(ns)) if orig is None else np.asarray(orig)
    at = seeded_positions(orig)  # seeded index -> position
    ns_seeded = ns[at]
    pool = np.where((ns_seeded >= 1000) & (ns_seeded <= 1_000_000))[0]
    keys = {}
    sweep = []
    for rate in args.serve_rates:
        # enough requests that arrivals last serve_window seconds: the tail of the largest
        # requests then weighs little in the sustained rate
        nreq = max(args.serve_requests, int(rate * args.serve_window))
        pick = at[g.choice(pool, size=nreq)]
        for i in np.unique(pick):
            if int(i) not in keys:
                keys[int(i)] = key_all[int(coff[i]):int(coff[i]) + int(ns[i])].cpu().numpy().view(np.uint64)
        arr = np.cumsum(g.exponential(1.0 / rate, nreq))
        srv = bs.Server(budget_bytes=64 << 30)
        tickets = []
        t0 = time.perf_counter()
        for r in range(nreq):
            now = time.perf_counter() - t0
            if arr[r] > now:
                time.sleep(arr[r] - now)
            i = int(pick[r])
            tickets.append((srv.submit(keys[i], scale=out_structs[i].scale, seed=r, part_id=int(orig[i])),
                            int(ns[i])))
        lat, done, t_first, t_last = [], 0, None, 0.0
        pending = list(tickets)
        while pending:
            rest = []
            for t, n in pending:
                if srv.poll(t) is None:
                    rest.append((t, n))
                    continue
                ts = srv.times(t)
                lat.append((ts[2] - ts[0]) * 1e3)
                t_first = ts[0] if t_first is None else min(t_first, ts[0])
                t_last = max(t_last, ts[2])
                done += n
            pending = rest
            if pending:
                time.sleep(0.0005)
        srv.close()
        lat = np.array(lat)
        offered = float(ns[pick].sum() / arr[-1])
        sweep.append({"offered_rate_hz": rate, "requests": nreq, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "p999_ms": float(np.percentile(lat, 99.9)),
                      "offered_surfels_per_s": offered,
                      "sustained_surfels_per_s": done / max(1e-9, t_last - t_first)})
    ok = [x for x in sweep if x["sustained_surfels_per_s"] >= 0.9 * x["offered_surfels_per_s"]]
    head = max(ok, key=lambda x: x["offered_rate_hz"]) if ok else sweep[0]
    return {"headline_rate_hz": head["offered_rate_hz"], "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
            "p999_ms": head["p999_ms"], "sustained_surfels_per_s": head["sustained_surfels_per_s"],
            "sweep": sweep,
            "requests_from": "surfel arrays of the batch parts with 1k-1M surfels, seeded choice and start",
            "headline": "highest offered rate the server keeps up with (>= 90% of offered surfels/s)"}


def scene_leg(args):
    """Scene scale: every node of a production-line scene (one per part, per group of 50
    parts and per line) regenerated on the device, sampled from the 6 axis directions and
    ordered with the min(200k, triangles / 2) bound; end-to-end wall time of the whole scene
    (one run, after a one-line warm-up), from triangles at every level and bottom-up."""
    from paper_1904_08225_gb300 import scene
    scene.run(args.seed, lines=1, per_line=min(args.scene_per_line, 100))
    r = scene.run(args.seed, lines=args.scene_lines, per_line=args.scene_per_line)
    out = {"lines": args.scene_lines, "parts": args.scene_lines * args.scene_per_line, "nodes": r.nodes,
           "triangles": r.triangles, "surfels_sampled": r.surfels_sampled, "surfels_ordered": r.surfels_ordered,
           "seconds": r.seconds, "ordered_per_s": r.surfels_ordered / r.seconds,
           "per_level": {str(k): v for k, v in sorted(r.per_level.items())},
           "level_res": scene.LEVEL_RES, "dirs": "6 axis"}
    # bottom-up: groups from their parts' surfel discs, lines from their groups' (Sec. 3.4)
    scene.run_hierarchical(args.seed, lines=1, per_line=min(args.scene_per_line, 100))
    h = scene.run_hierarchical(args.seed, lines=args.scene_lines, per_line=args.scene_per_line)
    out["bottom_up"] = {"nodes": h.nodes, "seconds": h.seconds, "surfels_sampled": h.surfels_sampled,
                        "surfels_ordered": h.surfels_ordered,
                        "per_level": {str(k): v for k, v in sorted(h.per_level.items())}}
    return out


def table2_leg(bs, timed):
    """The shape of the paper's Table 2 (one CAD object, 8 views at 1024^2, prefixes of
    10k/50k/100k surfels ordered by the randomised sampler with 200 samples per round and
    k = 500): here the CAD-like part.  Context only -- the paper's 12 ms render + 82 ms
    initial set + 105/311/592 ms sampling are a GTX 1060 and one i7-6700 thread."""
    import torch
    m = W.cad_part(seed=0)
    dirs = np.concatenate([W.AXIS_DIRS, W.DIAG_DIRS])
    xyz, tri, rgb = (torch.from_numpy(m.xyz).cuda(), torch.from_numpy(m.tri.view(np.int32)).cuda(),
                     torch.from_numpy(m.rgb).cuda())
    g = bs.sample_visible(xyz, tri, rgb, dirs, 1024)
    ms_sample = timed(lambda: bs.sample_visible(xyz, tri, rgb, dirs, 1024), 3) / 3
    out = {"surfels": g["n"], "sample_visible_ms": ms_sample, "triangles": m.ntris}
    for mc in (10_000, 50_000, 100_000):
        bs.order(g["key"], seed=0, max_count=mc, variant=1, sample_size=200, sample_step=500)
        out[f"sampler_{mc // 1000}k_ms"] = timed(lambda: bs.order(g["key"], seed=0, max_count=mc, variant=1,
                                                                  sample_size=200, sample_step=500), 1)
        out[f"exact_{mc // 1000}k_ms"] = timed(lambda: bs.order(g["key"], seed=0, max_count=mc), 1)
    out["paper"] = "GTX 1060 + i7-6700 1 thread: render 12 ms, initial set 82 ms, sampling 105/311/592 ms (10k/50k/100k of 1.75M)"
    return out


def cpu_baseline(specs, args):
    import oracle
    oracle.build()
    nthreads = oracle.num_threads()
    idx = oracle_sample_parts(specs, args.cpu_budget_s, seed=args.seed)
    tot, dt = run_oracle_parts(specs, idx, nthreads)
    return {"value": tot / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{len(idx)} of {len(specs)} parts (seeded), {tot} surfels, {dt:.1f} s; oracle "
                      f"sample_visible + O(N^2) greedy"}


if __name__ == "__main__":
    sys.exit(main())
