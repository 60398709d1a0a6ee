"""Error paths of the library, made on the host (no GPU fault, trap or hang is caused):
a device-scratch allocation made to fail (bs_set_tuning("fail_next_allocs", k)), a server
request cancelled while queued, on the device or finished, and a server request that
outlives the server's timeout.  Each case checks that the failing call or request gets its
status, that nothing else in flight is disturbed (results still equal bs_order's), and
that memory and admission budget come back.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs as _bs
    _bs.load()
    yield _bs
    _bs.set_tuning("fail_next_allocs", 0)
    _bs.set_tuning("server_timeout_ms", 0)


def _keys(n, seed):
    g = np.random.default_rng(seed)
    pts = np.unique(g.integers(0, 1 << 20, size=(n + n // 8 + 8, 3)), axis=0)[:n].astype(np.uint64)
    return (pts[:, 0] << np.uint64(42)) | (pts[:, 1] << np.uint64(21)) | pts[:, 2]


def _want(bs, key, seed, part_id, scale=1.0):
    out = bs.order(torch.from_numpy(key.view(np.int64)).cuda(), seed=seed, part_id=part_id, scale=scale)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def _wait(srv, t, limit=120.0):
    t0 = time.time()
    while time.time() - t0 < limit:
        try:
            r = srv.poll(t)
        except Exception as e:  # noqa: BLE001 -- the caller checks the status
            return e
        if r is not None:
            return r
        time.sleep(0.001)
    raise AssertionError("request did not finish")


def _same(r, w):
    return (np.array_equal(r[0], w[0].view(np.uint32)) and np.array_equal(r[1], w[1])
            and np.array_equal(r[2].view(np.uint32), w[2].view(np.uint32)))


def test_allocation_failure_returns_enomem_then_recovers(bs):
    key = torch.from_numpy(_keys(20_000, 1).view(np.int64)).cuda()
    want = bs.order(key, seed=3)
    torch.cuda.synchronize()
    bs.set_tuning("fail_next_allocs", 1)
    with pytest.raises(bs.BsError) as e:
        bs.order(key, seed=3)
    assert e.value.status == bs.BS_ENOMEM
    got = bs.order(key, seed=3)  # the injection is used up: the next call runs
    torch.cuda.synchronize()
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])


def test_server_allocation_failure_spares_requests_in_flight(bs):
    big, small = _keys(600_000, 2), _keys(30_000, 3)
    wb, ws = _want(bs, big, 1, 1), _want(bs, small, 2, 2)
    with bs.Server(budget_bytes=8 << 30) as srv:
        tb = srv.submit(big, seed=1, part_id=1)
        time.sleep(0.3)  # the big request's launch has its memory and is running
        bs.set_tuning("fail_next_allocs", 1)
        tf = srv.submit(small, seed=2, part_id=2)
        rf = _wait(srv, tf)
        assert isinstance(rf, bs.BsError) and rf.status == bs.BS_ENOMEM
        rb = _wait(srv, tb)
        assert not isinstance(rb, Exception) and _same(rb, wb)
        # the failed launch gave back its budget: requests filling the budget still run
        ts = [srv.submit(small, seed=2, part_id=2) for _ in range(8)]
        for t in ts:
            r = _wait(srv, t)
            assert not isinstance(r, Exception) and _same(r, ws)


def test_server_cancel_queued_running_and_finished(bs):
    big, small = _keys(600_000, 4), _keys(20_000, 5)
    ws = _want(bs, small, 7, 7)
    one = int(600_000 * 40 * 1.5)  # holds one big request (about 24.6 MB of device state), not two
    with bs.Server(budget_bytes=one) as srv:
        t_run = srv.submit(big, seed=1, part_id=1)
        t_q = srv.submit(big, seed=2, part_id=2)  # waits: the budget holds one big request
        time.sleep(0.05)
        srv.cancel(t_q)
        e = _wait(srv, t_q)
        assert isinstance(e, bs.BsError) and e.status == bs.BS_ECANCELED
        srv.cancel(t_run)  # on the device: dropped when its launch ends
        e = _wait(srv, t_run)
        assert isinstance(e, bs.BsError) and e.status == bs.BS_ECANCELED
        # both budgets came back: a request needing the whole budget is admitted and runs
        t_after = srv.submit(big, seed=3, part_id=3)
        r = _wait(srv, t_after)
        assert not isinstance(r, Exception) and len(r[0]) == 600_000
        # a finished, uncollected result is dropped by a cancel
        t_done = srv.submit(small, seed=7, part_id=7)
        while srv._lib.bs_server_poll(srv._h, t_done, None, None, None) != bs.BS_OK:
            time.sleep(0.001)
        srv.cancel(t_done)
        e = _wait(srv, t_done)
        assert isinstance(e, bs.BsError) and e.status == bs.BS_ECANCELED
        t_ok = srv.submit(small, seed=7, part_id=7)
        assert _same(_wait(srv, t_ok), ws)
        with pytest.raises(bs.BsError) as e:
            srv.cancel(10**9)
        assert e.value.status == bs.BS_EINVAL


def test_server_request_timeout(bs):
    big = _keys(600_000, 6)
    bs.set_tuning("server_timeout_ms", 1)
    try:
        srv = bs.Server(budget_bytes=8 << 30)
    finally:
        bs.set_tuning("server_timeout_ms", 0)
    with srv:
        t = srv.submit(big, seed=1, part_id=1)
        e = _wait(srv, t)
        assert isinstance(e, bs.BsError) and e.status == bs.BS_ETIMEOUT
    # a server created afterwards has no timeout and orders the same request
    with bs.Server(budget_bytes=8 << 30) as srv2:
        t = srv2.submit(big, seed=1, part_id=1)
        r = _wait(srv2, t)
        assert not isinstance(r, Exception) and _same(r, _want(bs, big, 1, 1))
