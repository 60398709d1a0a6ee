"""bs_order_noalloc: the ordering entry point for callers that may not allocate device memory.

A caller running inside someone else's GPU memory budget (a plugin or render thread
of a host application, a real-time loop) cannot let the library call cudaMalloc.
bs_order_noalloc takes its scratch from a fixed array the library reserves on each
GPU; these tests call it through the C ABI and require the same bit-exact output as
bs_order, on consecutive calls that reuse that array.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs
    return bs


def _part(n, seed):
    g = np.random.default_rng(seed)
    pts = np.unique(g.integers(0, 1 << 21, size=(n + n // 8 + 4, 3)), axis=0)[:n].astype(np.uint64)
    key = (pts[:, 0] << np.uint64(42)) | (pts[:, 1] << np.uint64(21)) | pts[:, 2]
    return torch.from_numpy(key.view(np.int64)).cuda()


def _noalloc_call(bs, key, seed, part_id, max_count, scale, want_rad2=True, want_radius=True):
    """bs_order_noalloc straight through ctypes into caller-allocated outputs (rad2 and
    radius may be left out: the library then keeps rad2 in its fixed scratch)."""
    lib = bs.load()
    n = key.shape[0]
    m = n if max_count == 0 or max_count > n else max_count
    perm = torch.empty(m, dtype=torch.int32, device=key.device)
    rad2 = torch.empty(m, dtype=torch.int64, device=key.device) if want_rad2 else None
    radius = torch.empty(m, dtype=torch.float32, device=key.device) if want_radius else None
    s = bs.Surfels(key.data_ptr(), None, None, None, n, n, (C.c_float * 3)(), float(scale))
    o = bs.OrderOpts(seed, part_id, -1, max_count)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: C.c_void_p(t.data_ptr() if t is not None else None)  # noqa: E731
    st = lib.bs_order_noalloc(C.byref(s), C.byref(o), ptr(perm), ptr(rad2), ptr(radius), stream)
    assert st == bs.BS_OK, bs.last_error()
    return perm, rad2, radius


def _same(a, b):
    if a.dtype == torch.float32:
        a, b = a.view(torch.int32), b.view(torch.int32)
    return torch.equal(a, b)


def test_noalloc_matches_bs_order_on_consecutive_calls(lib):
    """Two calls in a row (a large part, then a smaller one that reuses the same scratch)
    give exactly what bs_order gives for each."""
    cases = [(_part(60000, 1), 3, 7, 0, 2.5), (_part(5000, 2), 9, 1, 0, 0.75), (_part(60000, 1), 3, 7, 1000, 2.5)]
    for key, seed, part_id, max_count, scale in cases:
        got = _noalloc_call(lib, key, seed, part_id, max_count, scale)
        want = lib.order(key, seed=seed, part_id=part_id, max_count=max_count, scale=scale)
        torch.cuda.synchronize()
        for a, b in zip(got, want):
            assert _same(a, b)


def test_noalloc_without_rad2_or_radius(lib):
    """rad2 left to the library's scratch: perm (and radius, when asked for) still equal
    bs_order's; with neither rad2 nor radius only perm is written."""
    key = _part(30000, 4)
    want = lib.order(key, seed=5, part_id=2, scale=1.5)
    perm, _, radius = _noalloc_call(lib, key, 5, 2, 0, 1.5, want_rad2=False)
    torch.cuda.synchronize()
    assert _same(perm, want[0]) and _same(radius, want[2])
    perm, _, _ = _noalloc_call(lib, key, 5, 2, 0, 1.5, want_rad2=False, want_radius=False)
    torch.cuda.synchronize()
    assert _same(perm, want[0])


def test_noalloc_at_its_size_limit(lib):
    """A part of exactly BS_NOALLOC_MAX_POINTS points fills the whole fixed scratch."""
    key = _part(65536, 5)
    assert key.shape[0] == 65536
    got = _noalloc_call(lib, key, 1, 0, 0, 1.0)
    want = lib.order(key, seed=1, part_id=0, scale=1.0)
    torch.cuda.synchronize()
    assert all(_same(a, b) for a, b in zip(got, want))


def test_noalloc_one_pick_loop(lib):
    """The one-pick-per-step kernel (order_algo 1) through the fixed scratch, radii by the
    separate radius kernel; the setting is restored afterwards."""
    key = _part(20000, 6)
    want = lib.order(key, seed=2, part_id=3, scale=0.5)
    try:
        lib.set_tuning("order_algo", 1)
        got = _noalloc_call(lib, key, 2, 3, 0, 0.5)
        torch.cuda.synchronize()
    finally:
        lib.set_tuning("order_algo", 2)
    assert all(_same(a, b) for a, b in zip(got, want))


def test_noalloc_rejects_parts_above_its_limit(lib):
    key = _part(65537, 3)
    with pytest.raises(lib.BsError) as e:
        lib.order_noalloc(key)
    assert e.value.status == lib.BS_EOVERFLOW
    assert "65536" in str(e.value)
