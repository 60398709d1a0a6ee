"""Pins for the oracle's randomised progressive sampler (Sec. 3.2 of the paper).

* With the whole remaining set as the sample and one pick per round, the sampler is
  the greedy permutation itself.
* Every pick of round t is the farthest (from the surfels chosen before the round)
  of that round's random subset, re-drawn here from the Philox stream (itself pinned
  by the published known-answer vectors) and the remaining set rebuilt from the picks.
* Round sizes follow 1 + t // step; rad2 is the distance to all earlier picks.
* Quality, as the paper reports it (Sec. 3.3): the median nearest-neighbour distance of a
  prefix is close to the greedy permutation's and well above a random order's.
"""
import numpy as np
import pytest

import oracle
from paper_1904_08225_gb300 import workloads as W

I64MAX = np.iinfo(np.int64).max


def _pts(n, seed, span=1 << 21):
    g = np.random.default_rng(seed)
    return np.unique(g.integers(0, span, size=(n + 50, 3)), axis=0)[:n]


@pytest.mark.parametrize("seed,span", [(0, 1 << 21), (1, 40), (2, 1 << 12)])
def test_whole_sample_is_the_greedy_permutation(seed, span):
    pts = _pts(1500, seed, span)
    key = oracle.pack(pts)
    s = oracle.start_index(len(key), seed=seed)
    a = oracle.greedy(key, s)
    b = oracle.sampled(key, s, sample_size=0, step=0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_picks_are_the_farthest_of_their_sample():
    pts = _pts(2000, 3)
    key = oracle.pack(pts)
    n = len(key)
    seed, part, S, step = 77, 5, 50, 40
    s = oracle.start_index(n, seed=seed, part_id=part)
    perm, rad2, rnd = oracle.sampled(key, s, max_count=900, seed=seed, part_id=part, sample_size=S, step=step,
                                     rounds=True)
    R = list(range(n))
    pos = list(range(n))

    def remove(x):
        p, y = pos[x], R[-1]
        R[p] = y
        pos[y] = p
        R.pop()
    remove(int(perm[0]))
    D = ((pts - pts[perm[0]]) ** 2).sum(1)
    k = 1
    t = 0
    while k < len(perm):
        L = len(R)
        sample = []
        for u in range(S):
            w = int(oracle.philox4x32_10([part, t, u, 1], [seed & 0xffffffff, seed >> 32])[0])
            c = R[(w * L) >> 32]
            if c not in sample:
                sample.append(c)
        mt = 1 + t // step
        want = sorted(sample, key=lambda c: (-int(D[c]), c))[:mt]
        got = [int(x) for x in perm[k:k + len(want)]]
        assert got == want[:len(got)], t
        assert (rnd[k:k + len(got)] == t).all()
        for c in got:
            remove(c)
        for c in got:
            D = np.minimum(D, ((pts - pts[c]) ** 2).sum(1))
        k += len(got)
        t += 1


def test_round_sizes_and_radii():
    pts = _pts(3000, 4)
    key = oracle.pack(pts)
    perm, rad2, rnd = oracle.sampled(key, 11, max_count=2500, sample_size=200, step=100, rounds=True)
    assert len(set(perm.tolist())) == len(perm)
    counts = np.bincount(rnd[1:])
    for t, c in enumerate(counts):
        assert c == 1 + t // 100 or t == len(counts) - 1
    P = pts[perm]
    for k in [1, 2, 10, 500, 2499]:
        assert rad2[k] == ((P[:k] - P[k]) ** 2).sum(1).min()
    assert rad2[0] == I64MAX
    # truncation keeps the prefix
    p2, r2 = oracle.sampled(key, 11, max_count=700, sample_size=200, step=100)
    assert np.array_equal(p2, perm[:700]) and np.array_equal(r2, rad2[:700])


def _median_nn(P):
    d = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1).astype(np.float64)
    np.fill_diagonal(d, np.inf)
    return float(np.median(np.sqrt(d.min(1))))


def test_quality_between_random_and_greedy():
    """Sec. 3.3: the sampled prefix is nearly as even as the greedy permutation's and far
    more even than a random subset (median nearest-neighbour distance of 1000 points)."""
    m = W.torus(nu=96, nv=48)
    sv, mn, s = oracle.sample_mesh(m, W.AXIS_DIRS, 96)
    key = sv["key"]
    pts = oracle.unpack(key)
    st = oracle.start_index(len(key), seed=0)
    gp, _ = oracle.greedy(key, st, max_count=1000)
    sp, _ = oracle.sampled(key, st, max_count=1000, sample_size=200, step=500)
    rnd = np.random.default_rng(0).permutation(len(key))[:1000]
    mg, ms, mr = _median_nn(pts[gp]), _median_nn(pts[sp]), _median_nn(pts[rnd])
    assert ms >= 0.8 * mg and ms >= 1.5 * mr


def test_tiny_inputs():
    key = oracle.pack(np.array([[0, 0, 0]]))
    p, r = oracle.sampled(key, 0)
    assert p.tolist() == [0] and r.tolist() == [I64MAX]
    key = oracle.pack(np.array([[0, 0, 0], [3, 4, 0]]))
    p, r = oracle.sampled(key, 1)
    assert p.tolist() == [1, 0] and r.tolist() == [I64MAX, 25]
