"""Pins for the oracle's prefix selection (Sec. 4.1): median nearest-neighbour distance
of a prefix and the shortest prefix covering a part within a radius."""
import numpy as np

import oracle


def test_line_closed_forms():
    """2^m + 1 collinear points, spacing h, from one end: the prefix of 2^j + 1 points is
    the evenly spaced subset with gap 2^(m-j) h, so every NN distance is that gap; the
    shortest prefix reaching every point within r = 2^(m-j) h is 2^j + 1."""
    m, h = 8, 3
    n = 2**m + 1
    p = np.zeros((n, 3), np.int64)
    p[:, 0] = np.arange(n) * h
    key = oracle.pack(p)
    perm, rad2 = oracle.greedy(key, 0)
    for j in range(1, m + 1):
        pm = 2**j + 1
        gap = 2 ** (m - j) * h
        assert oracle.prefix_median_nn(key, perm, pm) == gap * gap
        assert oracle.prefix_for_radius(rad2, gap * gap) == 2 ** (j - 1) + 1
        assert oracle.prefix_for_radius(rad2, gap * gap - 1) == (pm if j < m else n)
    assert oracle.prefix_for_radius(rad2, 0) == n
    assert oracle.prefix_for_radius(rad2, 10**12) == 1


def test_median_brute_force_and_covering():
    g = np.random.default_rng(2)
    pts = np.unique(g.integers(0, 5000, size=(700, 3)), axis=0)
    key = oracle.pack(pts)
    perm, rad2 = oracle.greedy(key, 0)
    for pm in [2, 3, 10, 101, 400]:
        P = pts[perm[:pm]]
        d = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
        np.fill_diagonal(d, np.iinfo(np.int64).max)
        nn = np.sort(d.min(1))
        assert oracle.prefix_median_nn(key, perm, pm) == nn[(pm + 1) // 2 - 1]
    for r2 in [0, 1, 1000, 50000, 10**6, 10**9]:
        p = oracle.prefix_for_radius(rad2, r2)
        # the prefix reaches every point within r and no shorter prefix does
        P = pts[perm[:p]]
        reach = ((pts[:, None, :] - P[None, :, :]) ** 2).sum(-1).min(1).max()
        assert reach <= r2 or p == len(pts)
        if p > 1:
            Q = pts[perm[:p - 1]]
            assert ((pts[:, None, :] - Q[None, :, :]) ** 2).sum(-1).min(1).max() > r2
    assert oracle.prefix_median_nn(key, perm, 1) == 0
