"""Autotuner for the batched ordering launch.

Times bs_order_batched on the caller's own batch under each candidate launch shape (CTA
size, quarter mode on or off, how many of the largest parts run on whole CTAs) and
keeps the fastest through bs_set_tuning.  The knobs change how the work is spread over
the GPU, never the result: every candidate gives the same permutations and radii, and
the tuner checks that on the batch it times.
"""
from __future__ import annotations

import itertools

from . import bs

# (order_threads, order_quarters, order_full_parts); 0 lets the library decide
DEFAULT_CANDIDATES = [
    (0, 0, 0),        # the library's own choice (cost model)
    (512, 1, 0),      # whole 512-thread CTAs, one part each
    (1024, 1, 0),     # whole 1024-thread CTAs
    (0, 2, 0),        # quarters for every part that fits one
] + [(0, 2, k) for k in (4, 16, 64)]  # quarters after the k largest parts on whole CTAs


def autotune(keys, starts=None, seeds=None, max_counts=None, scales=None, candidates=None, repeats: int = 2,
             apply: bool = True):
    """Returns (best candidate, {candidate: ms}); with apply, leaves the best one set.

    keys: list of CUDA int64 key tensors (the batch to tune on)."""
    import torch
    cands = candidates or DEFAULT_CANDIDATES
    names = ("order_threads", "order_quarters", "order_full_parts")
    times, ref = {}, None
    try:
        for cand in cands:
            for n, v in zip(names, cand):
                bs.set_tuning(n, v)
            out = bs.order_batched(keys, starts=starts, seeds=seeds, max_counts=max_counts, scales=scales)
            torch.cuda.synchronize()
            perms = [o[0] for o in out]
            if ref is None:
                ref = perms
            elif not all(torch.equal(a, b) for a, b in zip(ref, perms)):
                raise RuntimeError(f"autotune: launch shape {cand} changed a result")
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(repeats):
                bs.order_batched(keys, starts=starts, seeds=seeds, max_counts=max_counts, scales=scales)
            e1.record()
            torch.cuda.synchronize()
            times[cand] = e0.elapsed_time(e1) / repeats
    finally:
        for n in names:
            bs.set_tuning(n, 0)
    best = min(times, key=times.get)
    if apply:
        for n, v in zip(names, best):
            bs.set_tuning(n, v)
    return best, times


def candidates_grid(threads=(0, 512, 1024), quarters=(0, 1, 2), full_parts=(0, 16)):
    """A wider candidate grid (every combination)."""
    return list(itertools.product(threads, quarters, full_parts))
