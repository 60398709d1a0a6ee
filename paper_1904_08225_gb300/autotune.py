"""Autotuner for the batched ordering launch.

Times bs_order_batched on the caller's own batch under each candidate launch shape --
CTA size, whether the CTAs split into part slots after their whole-CTA parts, how many of
the largest parts run on whole CTAs, and how many parts a CTA orders at once (2, 4 or 8
slots) -- and keeps the fastest through bs_set_tuning.  Each candidate is timed `repeats`
times (median).  The knobs change how the work is spread over the GPU, never the result:
every candidate gives the same permutations and radii, and the tuner checks that on the
batch it times.  (The grid cell of the ordering -- a bucket of 32 consecutive points, one
warp -- is fixed by the kernel's data layout and is not a knob.)
"""
from __future__ import annotations

import itertools

from . import bs

NAMES = ("order_threads", "order_quarters", "order_full_parts", "order_slots")

# (order_threads, order_quarters, order_full_parts, order_slots); 0 lets the library decide
DEFAULT_CANDIDATES = [
    (0, 0, 0, 0),        # the library's own choice (cost model, four slots per CTA)
    (512, 1, 0, 0),      # whole 512-thread CTAs, one part each
    (1024, 1, 0, 0),     # whole 1024-thread CTAs
    (0, 2, 0, 0),        # quarters for every part that fits one
    (0, 0, 0, 2),        # two 512-thread slots per CTA (cost model for the whole-CTA parts)
    (0, 0, 0, 8),        # eight 128-thread slots per CTA
] + [(0, 2, k, 0) for k in (4, 16, 64)]  # quarters after the k largest parts on whole CTAs


def autotune(keys, starts=None, seeds=None, max_counts=None, scales=None, candidates=None, repeats: int = 3,
             apply: bool = True):
    """Returns (best candidate, {candidate: median ms}); with apply, leaves the best one set.

    keys: list of CUDA int64 key tensors (the batch to tune on)."""
    import torch
    cands = candidates or DEFAULT_CANDIDATES
    times, spread, ref = {}, {}, None
    try:
        for cand in cands:
            for n, v in zip(NAMES, cand):
                bs.set_tuning(n, v)
            out = bs.order_batched(keys, starts=starts, seeds=seeds, max_counts=max_counts, scales=scales)
            torch.cuda.synchronize()
            perms = [o[0] for o in out]
            if ref is None:
                ref = perms
            elif not all(torch.equal(a, b) for a, b in zip(ref, perms)):
                raise RuntimeError(f"autotune: launch shape {cand} changed a result")
            ms = []
            for _ in range(max(1, repeats)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                bs.order_batched(keys, starts=starts, seeds=seeds, max_counts=max_counts, scales=scales)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            ms.sort()
            times[cand] = ms[len(ms) // 2]
            spread[cand] = (ms[0], ms[-1])
    finally:
        for n in NAMES:
            bs.set_tuning(n, 0)
    best = min(times, key=times.get)
    if apply:
        for n, v in zip(NAMES, best):
            bs.set_tuning(n, v)
    autotune.last_spread = spread
    return best, times


def candidates_grid(threads=(0, 512, 1024), quarters=(0, 1, 2), full_parts=(0, 16), slots=(0, 2, 8)):
    """A wider candidate grid (every combination)."""
    return list(itertools.product(threads, quarters, full_parts, slots))
