"""Pins for the oracle's ordering half: Philox, start index, greedy permutation.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, an exhaustive search over all permutations,
from-scratch recomputation, and the r-net property of greedy prefixes (Sec. 4.1).
"""
import itertools

import numpy as np
import pytest

import oracle
from tests.conftest import golden_path

I64MAX = np.iinfo(np.int64).max


def _read_kat():
    rows = []
    with open(golden_path("philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    """Philox4x32-10 equals the Random123 / SC'11 known-answer vectors."""
    rows = _read_kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert oracle.philox4x32_10(ctr, key).tolist() == want


def test_start_index_from_seed():
    """Random start of Sec. 3.2: s = (word0 * N) >> 32 with word0 from the KAT table."""
    word0 = 0x6627E8D5  # Philox4x32-10(ctr=0, key=0) word 0, from the published vectors
    for n in [1, 2, 7, 1000, 32920, 3_000_000, 2**32 - 1]:
        assert oracle.start_index(n, seed=0, part_id=0) == (word0 * n) >> 32
    assert oracle.start_index(10, start=3) == 3
    with pytest.raises(ValueError):
        oracle.start_index(10, start=10)


def _morton_py(x, y, z):
    m = 0
    for i in range(21):
        m |= ((x >> i) & 1) << (3 * i) | ((y >> i) & 1) << (3 * i + 1) | ((z >> i) & 1) << (3 * i + 2)
    return m


def test_morton_small_cases():
    assert oracle.morton3(1, 0, 0) == 1
    assert oracle.morton3(0, 1, 0) == 2
    assert oracle.morton3(0, 0, 1) == 4
    assert oracle.morton3(2, 0, 0) == 8
    q = (1 << 21) - 1
    assert oracle.morton3(q, q, q) == (1 << 63) - 1
    g = np.random.default_rng(5)
    for _ in range(200):
        x, y, z = (int(v) for v in g.integers(0, 1 << 21, 3))
        assert oracle.morton3(x, y, z) == _morton_py(x, y, z)


def _d2(a, b):
    return int(((a - b) ** 2).sum())


def _from_scratch(pts, perm):
    """rad2 of a given permutation, each entry recomputed from its definition."""
    out = [I64MAX]
    for k in range(1, len(perm)):
        out.append(min(_d2(pts[perm[k]], pts[perm[j]]) for j in range(k)))
    return out


def _exhaustive_greedy(pts, s):
    """Lexicographic maximum over ALL permutations starting at s of the sequence
    ((rad2_1, -p_1), (rad2_2, -p_2), ...) -- the greedy permutation by definition
    of "each next point as far as possible from all previous ones"."""
    n = len(pts)
    rest = [i for i in range(n) if i != s]
    best, best_seq = None, None
    for tail in itertools.permutations(rest):
        perm = (s,) + tail
        r = _from_scratch(pts, perm)
        seq = [(r[k], -perm[k]) for k in range(1, n)]
        if best is None or seq > best:
            best, best_seq = seq, perm
    return list(best_seq)


@pytest.mark.parametrize("n,seed", [(2, 0), (5, 1), (6, 2), (7, 3), (7, 4), (7, 5)])
def test_greedy_exhaustive_tiny(n, seed):
    """Oracle equals the exhaustive lexicographic maximum on N <= 7 (ties included)."""
    g = np.random.default_rng(seed)
    pts = g.integers(0, 6, size=(n, 3)).astype(np.int64)  # small range: many equal distances
    # distinct points only (canonical surfel arrays are deduplicated)
    pts = np.unique(pts, axis=0)
    n = len(pts)
    key = oracle.pack(pts)
    s = int(g.integers(0, n))
    perm, rad2 = oracle.greedy(key, s)
    assert perm.tolist() == _exhaustive_greedy(pts, s)
    assert rad2.tolist() == _from_scratch(pts, perm.tolist())


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("m,h", [(3, 1), (6, 5), (9, 1000)])
def test_greedy_line_closed_form(axis, m, h):
    """2^m+1 equally spaced points from one end: the far end, then dyadic midpoints
    level by level, lowest index first; level j (j>=1) has 2^(j-1) entries of
    squared radius (2^(m-j) h)^2."""
    n = 2**m + 1
    p = np.zeros((n, 3), np.int64)
    p[:, axis] = np.arange(n) * h
    perm, rad2 = oracle.greedy(oracle.pack(p), 0)
    want_perm = [0, n - 1]
    want_rad = [I64MAX, ((n - 1) * h) ** 2]
    for j in range(1, m + 1):
        step = 2 ** (m - j)
        mids = list(range(step, n - 1, 2 * step))
        assert len(mids) == 2 ** (j - 1)
        want_perm += mids
        want_rad += [(step * h) ** 2] * len(mids)
    assert perm.tolist() == want_perm
    assert rad2.tolist() == want_rad


def _rnet_check(pts, perm, rad2, ks):
    """r-net property (Sec. 4.1): prefix k is rad2[k-1]-separated (min pairwise d^2
    equals rad2[k-1]) and rad2[k]-covering (max distance^2 to the prefix)."""
    n = len(pts)
    P = pts[perm]
    for k in ks:
        pre = P[:k]
        if k >= 2:
            dd = ((pre[:, None, :] - pre[None, :, :]) ** 2).sum(-1)
            dd[np.arange(k), np.arange(k)] = I64MAX
            assert dd.min() == rad2[k - 1], k
        cov = ((pts[:, None, :] - pre[None, :, :]) ** 2).sum(-1).min(1).max()
        assert cov == (rad2[k] if k < n else 0), k


def test_greedy_rnet_invariants_random():
    g = np.random.default_rng(11)
    pts = np.unique(g.integers(0, 1 << 21, size=(600, 3)), axis=0)
    key = oracle.pack(pts)
    perm, rad2 = oracle.greedy(key, 17)
    assert sorted(perm.tolist()) == list(range(len(pts)))
    assert np.all(np.diff(rad2[1:]) <= 0)
    _rnet_check(pts, perm, rad2, [1, 2, 3, 5, 10, 50, 100, 299, 598, len(pts)])
    assert rad2.tolist() == _from_scratch(pts, perm.tolist())


def test_greedy_grid_invariants():
    """A 2-D (2^3+1)^2 grid from a corner: from-scratch radii, r-net at every prefix."""
    m = 3
    n1 = 2**m + 1
    X, Y = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    pts = np.stack([X.ravel() * 7, Y.ravel() * 7, np.zeros(n1 * n1, np.int64)], -1)
    order = np.argsort([oracle.morton3(*map(int, p)) for p in pts], kind="stable")
    pts = pts[order]
    key = oracle.pack(pts)
    s = int(np.where((pts == 0).all(1))[0][0])
    perm, rad2 = oracle.greedy(key, s)
    assert rad2.tolist() == _from_scratch(pts, perm.tolist())
    _rnet_check(pts, perm, rad2, range(1, len(pts) + 1))
    # every squared radius of a grid with spacing 7 is 49 * (a^2 + b^2)
    assert all(r % 49 == 0 for r in rad2[1:])


def test_greedy_truncation_is_prefix():
    g = np.random.default_rng(3)
    pts = np.unique(g.integers(0, 5000, size=(3000, 3)), axis=0)
    key = oracle.pack(pts)
    pf, rf = oracle.greedy(key, 5)
    for m in [1, 2, 17, 500]:
        pt, rt = oracle.greedy(key, 5, max_count=m)
        assert pt.tolist() == pf[:m].tolist() and rt.tolist() == rf[:m].tolist()


def test_greedy_duplicates_come_last():
    """With repeated keys the remaining copies have distance 0 and come last, in index order."""
    pts = np.array([[0, 0, 0], [10, 0, 0], [10, 0, 0], [0, 0, 0], [5, 0, 0]], np.int64)
    perm, rad2 = oracle.greedy(oracle.pack(pts), 0)
    assert perm.tolist() == [0, 1, 4, 2, 3]
    assert rad2.tolist() == [I64MAX, 100, 25, 0, 0]


def test_greedy_threads_agree():
    g = np.random.default_rng(8)
    pts = np.unique(g.integers(0, 300, size=(4000, 3)), axis=0)
    key = oracle.pack(pts)
    a = oracle.greedy(key, 0, nthreads=1)
    b = oracle.greedy(key, 0, nthreads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_visit_count_brute_force():
    """visits = N + sum_k #{unchosen i : d^2(i, perm[k]) < rad2[k]}, counted here directly."""
    g = np.random.default_rng(4)
    pts = np.unique(g.integers(0, 1000, size=(300, 3)), axis=0)
    perm, rad2, vis, imp = oracle.greedy(oracle.pack(pts), 2, stats=True)
    n = len(pts)
    want = n
    chosen = np.zeros(n, bool)
    chosen[perm[0]] = True
    for k in range(1, n):
        j = perm[k]
        chosen[j] = True
        d = ((pts - pts[j]) ** 2).sum(1)
        want += int(((d < rad2[k]) & ~chosen).sum())
    assert vis == want
    assert 0 < imp <= want


def test_radius_output():
    """Splat radius sqrt(rad2)/S as float32; +inf for the first entry."""
    r = oracle.radius(np.array([I64MAX, 4, 2, 0], np.int64), 2.0)
    assert np.isinf(r[0]) and r[1] == np.float32(1.0) and r[3] == 0.0
    assert r[2] == np.float32(np.sqrt(2.0) / 2.0)
