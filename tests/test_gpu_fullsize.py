"""Full-size runs of the batching and serving workloads, checked against the oracle.

The batching workload (4096 tori, lognormal sizes, ~123M surfels) is sampled with one
bs_sample_visible_batched call and ordered with one bs_order_batched launch -- the launch
configuration bench.py times.  The O(N^2) oracle cannot redo all of it, so a seeded subset
of parts is recomputed completely (sampling and ordering, bit for bit), and the largest
parts are checked through properties that hold at any size (a permutation, non-increasing
radii, the r-net separation of sampled prefixes).  The serving workload pushes 20,000
requests through bs_server and checks a seeded subset the same way.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1904_08225_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs
    specs = W.batch_parts(4096, seed=0)
    meshes = [sp.mesh() for sp in specs]
    trip = [(torch.from_numpy(m.xyz).cuda(), torch.from_numpy(m.tri.view(np.int32)).cuda(),
             torch.from_numpy(m.rgb).cuda()) for m in meshes]
    caps = [6 * sp.res * sp.res for sp in specs]
    sv = bs.sample_visible_batched(trip, [sp.res for sp in specs], W.AXIS_DIRS, caps=caps)
    keys = [s["key"] for s in sv]
    orders = bs.order_batched(keys, seeds=[0] * len(keys), part_ids=list(range(len(keys))),
                              scales=[s["scale"] for s in sv])
    torch.cuda.synchronize()
    return bs, specs, meshes, sv, orders


def _subset(specs, n, max_n, seed):
    g = np.random.default_rng(seed)
    idx = [int(i) for i in g.permutation(len(specs)) if specs[i].n_target <= max_n]
    return idx[:n]


def test_batch_workload_size(batch):
    bs, specs, meshes, sv, orders = batch
    ns = np.array([s["n"] for s in sv])
    assert len(ns) == 4096 and ns.min() >= 1
    assert 80e6 <= ns.sum() <= 160e6  # ~123M for seed 0


def test_batch_subset_bit_exact(batch):
    """A seeded subset of parts: sampled surfels and full orderings equal the oracle's."""
    bs, specs, meshes, sv, orders = batch
    for i in _subset(specs, 24, 20_000, seed=1):
        ref, mn, s = oracle.sample_mesh(meshes[i], W.AXIS_DIRS, specs[i].res)
        assert np.array_equal(sv[i]["key"].cpu().numpy().view(np.uint64), ref["key"]), i
        assert np.array_equal(sv[i]["nrm"].cpu().numpy(), ref["nrm"]), i
        assert np.array_equal(sv[i]["src"].cpu().numpy().view(np.uint32), ref["src"]), i
        st = oracle.start_index(len(ref["key"]), seed=0, part_id=i)
        rp, rr = oracle.greedy(ref["key"], st, nthreads=oracle.num_threads())
        perm, rad2, radius = orders[i]
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), rp), i
        assert np.array_equal(rad2.cpu().numpy(), rr), i
        assert np.array_equal(radius.cpu().numpy().view(np.uint32), oracle.radius(rr, s).view(np.uint32)), i


def test_batch_largest_parts_equal_the_oracle(batch):
    """The three largest parts of the batch (421k-475k surfels), ordered inside the full
    4096-part launch: their whole perm / rad2 / radius equal the oracle's complete
    O(N^2) orderings, stored as digests by tests/golden/make_order_golden.py."""
    import golden_order as G
    bs, specs, meshes, sv, orders = batch
    ns = np.array([s["n"] for s in sv])
    recs = G.read("batch4096_largest_order.txt")
    assert sorted(r["id"] for r in recs) == sorted(int(i) for i in np.argsort(-ns)[:3])
    for r in recs:
        i = r["id"]
        perm, rad2, radius = (t.cpu().numpy() for t in orders[i])
        G.check(r, sv[i]["key"].cpu().numpy().view(np.uint64), perm, rad2, radius)


def test_batch_largest_parts_properties(batch):
    """The largest parts: a permutation with non-increasing radii whose first 500 entries
    equal the oracle's truncated ordering, and sampled prefixes that are r-separated."""
    bs, specs, meshes, sv, orders = batch
    ns = np.array([s["n"] for s in sv])
    for i in np.argsort(-ns)[:3]:
        i = int(i)
        key = sv[i]["key"].cpu().numpy().view(np.uint64)
        perm = orders[i][0].cpu().numpy().view(np.uint32)
        rad2 = orders[i][1].cpu().numpy()
        n = len(key)
        assert np.array_equal(np.sort(perm), np.arange(n, dtype=np.uint32))
        assert (np.diff(rad2[1:]) <= 0).all()
        st = oracle.start_index(n, seed=0, part_id=i)
        rp, rr = oracle.greedy(key, st, max_count=500, nthreads=oracle.num_threads())
        assert np.array_equal(perm[:500], rp) and np.array_equal(rad2[:500], rr)
        pts = oracle.unpack(key)
        g = np.random.default_rng(i)
        for k in [2, 100, n // 2, n - 1]:
            pre = pts[perm[:k]]
            d = ((pre[:-1] - pre[-1]) ** 2).sum(1)
            assert d.min() == rad2[k - 1]
            for t in g.integers(1, k, 50) if k > 2 else [1]:
                d2 = ((pts[perm[:t]] - pts[perm[t]]) ** 2).sum(1)
                assert d2.min() == rad2[t]


def test_serving_20k_requests(batch):
    """20,000 ordering requests (surfel arrays of the batch parts with 1k-1M surfels, each
    with its own seed) through bs_server under Poisson arrivals; a seeded subset equals
    the oracle, every result is a permutation with non-increasing radii."""
    bs, specs, meshes, sv, orders = batch
    ns = np.array([s["n"] for s in sv])
    pool = np.where((ns >= 1000) & (ns <= 60_000))[0]
    g = np.random.default_rng(4)
    nreq = 20_000
    pick = g.choice(pool, size=nreq)
    keys = {int(i): sv[int(i)]["key"].cpu().numpy().view(np.uint64) for i in np.unique(pick)}
    arr = np.cumsum(g.exponential(1.0 / 5000.0, nreq))
    check = set(int(r) for r in g.choice(nreq, size=12, replace=False))
    res = {}
    with bs.Server(budget_bytes=16 << 30) as srv:
        tickets = []
        t0 = time.perf_counter()
        for r in range(nreq):
            now = time.perf_counter() - t0
            if arr[r] > now:
                time.sleep(arr[r] - now)
            tickets.append(srv.submit(keys[int(pick[r])], scale=1.0, seed=r, part_id=int(pick[r])))
        pending = list(range(nreq))
        while pending:
            rest = []
            for r in pending:
                out = srv.poll(tickets[r])
                if out is None:
                    rest.append(r)
                    continue
                n = len(keys[int(pick[r])])
                assert len(out[0]) == n and (np.diff(out[1][1:]) <= 0).all()
                if r in check:
                    res[r] = out
            pending = rest
            if pending:
                time.sleep(0.002)
    for r in sorted(check):
        k = keys[int(pick[r])]
        rp, rr = oracle.greedy(k, oracle.start_index(len(k), seed=r, part_id=int(pick[r])),
                               nthreads=oracle.num_threads())
        assert np.array_equal(res[r][0], rp) and np.array_equal(res[r][1], rr), r
