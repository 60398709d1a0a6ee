"""Cluster mode: the exact ordering of one part split over the CTAs of a thread-block
cluster (Sec. 3.2 greedy permutation, Sec. 4.1 radius), against the oracle and against
the one-CTA-per-part path (itself oracle-checked), bit for bit.

Each CTA of the cluster owns a range of super-groups; candidates are gathered into the
leader's shared memory through distributed shared memory and the leader runs the
candidate greedy, so the cases below cover: cluster sizes 2..16 (including sizes that
do not divide the part's super-groups), ties whose tie window spans CTAs (a regular
grid), truncation, radii, a batch mixing cluster parts with ordinary ones (side
stream), and server requests large enough for a cluster.
"""
import time

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs as _bs
    _bs.load()
    yield _bs
    _bs.set_tuning("order_cluster", 1)
    _bs.set_tuning("order_cluster_min", 262144)


def _morton_sorted(pts):
    return oracle.pack(pts[np.argsort(_morton(pts), kind="stable")])


def _morton(pts):
    """Vectorised Morton code of (N, 3) coordinates (x in bit 0 of each triple)."""
    out = np.zeros(len(pts), np.uint64)
    p = pts.astype(np.uint64)
    for b in range(21):
        for a in range(3):
            out |= ((p[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return out


def _surface(n, seed):
    """n distinct points on a wavy sheet (a 2-manifold, like a sampled surface)."""
    g = np.random.default_rng(seed)
    uv = g.integers(0, 1 << 20, size=(n + n // 4 + 16, 2))
    z = ((np.sin(uv[:, 0] / 90000.0) + np.cos(uv[:, 1] / 70000.0)) * 200000 + 600000).astype(np.int64)
    pts = np.unique(np.stack([uv[:, 0], uv[:, 1], z], -1), axis=0)[:n]
    return _morton_sorted(pts)


def _dev(key):
    return torch.from_numpy(np.ascontiguousarray(key).view(np.int64)).cuda()


def _run(bs, key, cluster, **kw):
    try:
        bs.set_tuning("order_cluster_min", 1)
        bs.set_tuning("order_cluster", cluster)
        out = bs.order(key, **kw)
        torch.cuda.synchronize()
    finally:
        bs.set_tuning("order_cluster", 1)
        bs.set_tuning("order_cluster_min", 262144)
    return [t.cpu().numpy() for t in out]


def _same(a, b):
    return all(np.array_equal(x.view(np.uint32) if x.dtype == np.float32 else x,
                              y.view(np.uint32) if y.dtype == np.float32 else y) for x, y in zip(a, b))


def test_cluster_matches_oracle_on_a_surface(bs):
    """A 120k-point sheet (4 super-groups) on clusters of 2, 3 and 4: the oracle's ordering."""
    key = _surface(120_000, 1)
    kd = _dev(key)
    st = oracle.start_index(len(key), seed=3, part_id=9)
    rp, rr = oracle.greedy(key, st, nthreads=oracle.num_threads())
    rrad = oracle.radius(rr, 2.5)
    for c in (2, 3, 4):
        perm, rad2, radius = _run(bs, kd, c, seed=3, part_id=9, scale=2.5)
        assert np.array_equal(perm.view(np.uint32), rp), c
        assert np.array_equal(rad2, rr), c
        assert np.array_equal(radius.view(np.uint32), rrad.view(np.uint32)), c


def test_cluster_ties_span_ctas(bs):
    """A 257 x 257 grid (66,049 points, 3 super-groups) from its corner: many equal
    distances, tie windows that cross CTA boundaries; lowest index wins (oracle)."""
    n1 = 257
    X, Y = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    pts = np.stack([X.ravel() * 512, Y.ravel() * 512, np.full(n1 * n1, 7)], -1)
    key = _morton_sorted(pts)
    rp, rr = oracle.greedy(key, 0, nthreads=oracle.num_threads())
    kd = _dev(key)
    for c in (2, 3):
        perm, rad2, _ = _run(bs, kd, c, start=0)
        assert np.array_equal(perm.view(np.uint32), rp), c
        assert np.array_equal(rad2, rr), c


@pytest.fixture(scope="module")
def sheet600k(bs):
    key = _dev(_surface(600_000, 2))
    return key, _run(bs, key, 1, seed=1, scale=0.75)


@pytest.mark.parametrize("cluster", [2, 5, 8, 11, 16])
def test_cluster_sizes_match_one_cta(bs, sheet600k, cluster):
    """A 600k-point sheet (19 super-groups, which none of these sizes divides) on every
    cluster size, truncated and full, equals the one-CTA ordering."""
    key, base = sheet600k
    assert _same(_run(bs, key, cluster, seed=1, scale=0.75), base)
    cut = _run(bs, key, cluster, seed=1, scale=0.75, max_count=70_000)
    assert _same(cut, [b[:70_000] for b in base])


def test_cluster_parts_beside_ordinary_ones_in_one_batch(bs):
    """A batch of two cluster parts and 300 small ones (the clusters on the library's side
    stream, the rest on the caller's): every part equals its own single-part ordering."""
    g = np.random.default_rng(5)
    keys = [_dev(_surface(300_000, 11)), _dev(_surface(280_000, 12))]
    for i in range(300):
        keys.append(_dev(_surface(int(g.integers(500, 20_000)), 100 + i)))
    seeds = list(range(len(keys)))
    try:
        bs.set_tuning("order_cluster", 0)
        got = bs.order_batched(keys, seeds=seeds, part_ids=seeds, scales=[1.25] * len(keys))
        torch.cuda.synchronize()
    finally:
        bs.set_tuning("order_cluster", 1)
    got = [[t.cpu().numpy() for t in o] for o in got]
    for i in [0, 1, 2, 50, 299, 301]:
        want = _run(bs, keys[i], 1, seed=i, part_id=i, scale=1.25)
        assert _same(got[i], want), i


def test_cluster_server_request(bs):
    """A request of 300k points through bs_server (completion flag set by the leader CTA)
    equals bs_order."""
    key = _surface(300_000, 21)
    want = _run(bs, _dev(key), 1, seed=4, part_id=2, scale=1.0)
    bs.set_tuning("order_cluster", 0)
    with bs.Server(budget_bytes=4 << 30) as srv:
        t = srv.submit(key, scale=1.0, seed=4, part_id=2)
        r = None
        t0 = time.time()
        while r is None and time.time() - t0 < 120:
            r = srv.poll(t)
            time.sleep(0.001)
    bs.set_tuning("order_cluster", 1)
    assert r is not None
    assert np.array_equal(r[0], want[0].view(np.uint32)) and np.array_equal(r[1], want[1])
    assert np.array_equal(r[2].view(np.uint32), want[2].view(np.uint32))
