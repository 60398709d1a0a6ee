"""Fits the algorithmic work of the exact greedy ordering per surfel (test infrastructure).

For seeded torus parts of the batched-ordering generator, the oracle counts
exactly how many unchosen points lie strictly inside each new point's ball
(visits: what any correct pruned min-update must examine, plus the initial
sweep) and how many distances each update lowers (improved).  Both grow like
N ln N on a 2-manifold (ball of radius ~ spacing * sqrt(N/k) holds ~ c N/k
points), so visits/N and improved/N are fitted as a + b ln N.

Run:  python -m oracle.fit_visits   (prints the fit and the per-part residuals)
"""
from __future__ import annotations

import math
import sys

import numpy as np

import oracle
from paper_1904_08225_gb300 import workloads as W


def measure(nparts: int = 24, seed: int = 11, n_max: int = 40_000):
    specs = W.batch_parts(400, seed=seed, n_median=8000)
    rows = []
    for sp in specs:
        if len(rows) >= nparts:
            break
        m = sp.mesh()
        sv, mn, s = oracle.sample_mesh(m, W.AXIS_DIRS, sp.res)
        n = len(sv["key"])
        if n < 500 or n > n_max:
            continue
        st = oracle.start_index(n, seed=0)
        _, _, vis, imp = oracle.greedy(sv["key"], st, nthreads=oracle.num_threads(), stats=True)
        rows.append((n, vis, imp))
    return np.array(rows, dtype=np.float64)


def fit(rows):
    n = rows[:, 0]
    A = np.stack([np.ones_like(n), np.log(n)], 1)
    cv, *_ = np.linalg.lstsq(A, rows[:, 1] / n, rcond=None)
    ci, *_ = np.linalg.lstsq(A, rows[:, 2] / n, rcond=None)
    return cv, ci


def main():
    rows = measure()
    cv, ci = fit(rows)
    print(f"parts={len(rows)} N in [{int(rows[:, 0].min())}, {int(rows[:, 0].max())}]")
    print(f"VISITS_FIT = ({cv[0]:.2f}, {cv[1]:.2f})   # visits/N = a + b ln N")
    print(f"IMPROVED_FIT = ({ci[0]:.2f}, {ci[1]:.2f})")
    for n, v, i in rows:
        pv = cv[0] + cv[1] * math.log(n)
        pi = ci[0] + ci[1] * math.log(n)
        print(f"  N={int(n):7d} visits/N={v / n:7.2f} (fit {pv:7.2f})  improved/N={i / n:6.2f} (fit {pi:6.2f})")
    return 0


if __name__ == "__main__":
    sys.exit(main())
