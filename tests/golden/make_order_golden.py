"""Write the stored expected orderings of the full-size parts (test fixture generator).

The GPU parity tests compare whole orderings of parts too large for the O(N^2) oracle
to redo inside a test run: the CAD-like part of 5,423,479 surfels (2000 boxes + 500
cylinders, seed 0, 6 axis + 2 diagonal views at 1024^2) and the three largest parts of
the 4096-torus batch (seed 0).  This script computes them with the oracle only --
``oracle.sample_mesh`` for the initial surfel set of Sec. 3.1 and ``oracle.greedy`` for
the exact greedy permutation of Sec. 3.2/3.3 with the random start of Sec. 3.2 and the
per-prefix radius of Sec. 4.1 -- and stores, per part, SHA-256 digests of the surfel
keys and of the complete perm / rad2 / radius arrays plus the values at fixed indices.

Usage (from the repository root; the CAD part takes hours on 8 host cores):

    python tests/golden/make_order_golden.py batch [--threads T]
    python tests/golden/make_order_golden.py cad [--threads T]

Digest convention: SHA-256 of the arrays' little-endian bytes -- keys uint64, perm uint32,
rad2 int64, radius float32 bit patterns.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
from paper_1904_08225_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
CAD_FILE = os.path.join(HERE, "cad_part_seed0_order.txt")
BATCH_FILE = os.path.join(HERE, "batch4096_largest_order.txt")
SAMPLE_AT = (0, 1, 2, 1000, 100_000, 400_000)


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes()).hexdigest()


def record(name: str, part_id: int, key: np.ndarray, scale: float, threads: int) -> list[str]:
    n = len(key)
    st = oracle.start_index(n, seed=0, part_id=part_id)
    t = time.time()
    perm, rad2 = oracle.greedy(key, st, nthreads=threads)
    rad = oracle.radius(rad2, scale)
    dt = time.time() - t
    lines = [f"part {name} id {part_id} n {n} start {st} scale {scale!r} oracle_seconds {dt:.0f} threads {threads}",
             f"  key_sha256 {sha(key)}",
             f"  perm_sha256 {sha(perm)}",
             f"  rad2_sha256 {sha(rad2)}",
             f"  radius_sha256 {sha(rad.view(np.uint32))}"]
    for k in SAMPLE_AT + (n - 1,):
        if k < n:
            lines.append(f"  at {k} perm {int(perm[k])} rad2 {int(rad2[k])}")
    print("\n".join(lines), flush=True)
    return lines


def write(path: str, header: list[str], body: list[str]) -> None:
    with open(path + ".tmp", "w") as f:
        f.write("\n".join(header + body) + "\n")
    os.replace(path + ".tmp", path)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["batch", "cad"])
    ap.add_argument("--threads", type=int, default=oracle.num_threads())
    a = ap.parse_args()
    common = ["# Written by tests/golden/make_order_golden.py from the oracle alone (oracle.sample_mesh,",
              "# oracle.start_index with seed 0, oracle.greedy over every surfel, oracle.radius).",
              "# Exact greedy permutation of Sec. 3.2/3.3, random start of Sec. 3.2, per-prefix radius",
              "# of Sec. 4.1.  Digests: SHA-256 of little-endian key u64 / perm u32 / rad2 i64 / radius f32 bits."]
    if a.which == "cad":
        m = W.cad_part(seed=0)
        dirs = np.concatenate([W.AXIS_DIRS, W.DIAG_DIRS])
        ref, mn, s = oracle.sample_mesh(m, dirs, 1024)
        body = record("cad_seed0_8dirs_1024", 0, ref["key"], s, a.threads)
        write(CAD_FILE, common + ["# CAD-like part: workloads.cad_part(seed=0), 6 axis + 2 diagonal views at 1024^2."], body)
    else:
        specs = W.batch_parts(4096, seed=0)
        nt = np.array([sp.n_target for sp in specs])
        cand = [int(i) for i in np.argsort(-nt, kind="stable")[:16]]
        sized = []
        for i in cand:
            ref, mn, s = oracle.sample_mesh(specs[i].mesh(), W.AXIS_DIRS, specs[i].res)
            sized.append((len(ref["key"]), i, ref["key"], s))
        sized.sort(key=lambda t: (-t[0], t[1]))
        body = []
        for n, i, key, s in sized[:3]:
            body += record(f"batch4096_seed0_part{i}", i, key, s, a.threads)
        write(BATCH_FILE, common + ["# The three largest (by oracle surfel count, among the 16 largest targets) parts of",
                                    "# workloads.batch_parts(4096, seed=0), 6 axis views at each part's resolution;",
                                    "# part id = batch index (the Philox start uses part_id = batch index)."], body)


if __name__ == "__main__":
    main()
