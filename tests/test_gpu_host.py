"""Host buffers at the C boundary: meshes given in host memory (pageable numpy or
page-locked) are uploaded by the library, and bs_sample_order_batched goes from host meshes
to host results in one call (Sec. 3.1 sampling, Sec. 3.2 ordering, Sec. 4.1 radii).  Every
result must equal the device-buffer calls bit for bit; the device-buffer path is itself
checked against the oracle in test_gpu_parity."""
import numpy as np
import pytest

from paper_1904_08225_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08225_gb300 import bs as _bs
    _bs.load()
    return _bs


def _packed(meshes):
    vofs = np.cumsum([0] + [m.nverts for m in meshes])
    tofs = np.cumsum([0] + [m.ntris for m in meshes])
    xyz = np.ascontiguousarray(np.concatenate([m.xyz for m in meshes]), np.float32)
    tri = np.ascontiguousarray(np.concatenate([m.tri for m in meshes]).view(np.int32))
    rgb = np.ascontiguousarray(np.concatenate([m.rgb for m in meshes]), np.uint8)
    return vofs, tofs, xyz, tri, rgb


def _eq(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
    b = b.cpu().numpy() if hasattr(b, "cpu") else np.asarray(b)
    return a.tobytes() == b.tobytes()


def test_host_mesh_sampling_equals_device(bs):
    m = W.cad_part(seed=3, nboxes=120, ncyl=30)
    dirs = np.concatenate([W.AXIS_DIRS, W.DIAG_DIRS])
    dev = bs.sample_visible(torch.from_numpy(m.xyz).cuda(), torch.from_numpy(m.tri.view(np.int32)).cuda(),
                            torch.from_numpy(m.rgb).cuda(), dirs, 200)
    for pin in (False, True):
        xyz, tri, rgb = (torch.from_numpy(m.xyz), torch.from_numpy(m.tri.view(np.int32)), torch.from_numpy(m.rgb))
        if pin:
            xyz, tri, rgb = xyz.pin_memory(), tri.pin_memory(), rgb.pin_memory()
        host = bs.sample_visible(xyz, tri, rgb, dirs, 200)
        torch.cuda.synchronize()
        assert host["n"] == dev["n"] and host["scale"] == dev["scale"]
        for k in ("key", "nrm", "rgb", "src"):
            assert _eq(host[k][:host["n"]], dev[k][:dev["n"]]), (pin, k)


def test_host_meshes_batched_and_render(bs):
    specs = W.batch_parts(40, seed=5)
    meshes = [sp.mesh() for sp in specs]
    vofs, tofs, xyz, tri, rgb = _packed(meshes)
    res = [sp.res for sp in specs]
    n_v, n_t = np.diff(vofs), np.diff(tofs)
    caps = [6 * r * r for r in res]
    dev = bs.sample_visible_packed(torch.from_numpy(xyz).cuda(), torch.from_numpy(tri).cuda(),
                                   torch.from_numpy(rgb).cuda(), vofs[:-1], n_v, tofs[:-1], n_t, res, W.AXIS_DIRS,
                                   caps=caps)
    for pin in (False, True):
        hx, ht, hr = torch.from_numpy(xyz), torch.from_numpy(tri), torch.from_numpy(rgb)
        if pin:
            hx, ht, hr = hx.pin_memory(), ht.pin_memory(), hr.pin_memory()
        host = bs.sample_visible_packed(hx, ht, hr, vofs[:-1], n_v, tofs[:-1], n_t, res, W.AXIS_DIRS, caps=caps)
        torch.cuda.synchronize()
        assert np.array_equal(host["n"], dev["n"])
        for i in range(len(res)):  # the rows each part wrote (the rest of its capacity is untouched)
            a, k_ = int(dev["ofs"][i]), int(dev["n"][i])
            for k in ("key", "nrm", "rgb", "src"):
                assert _eq(host[k][a:a + k_], dev[k][a:a + k_]), (pin, i, k)
    m = meshes[3]
    img_d = bs.render_mesh(torch.from_numpy(m.xyz).cuda(), torch.from_numpy(m.tri.view(np.int32)).cuda(), (0, 0, 1), 96)
    img_h = bs.render_mesh(torch.from_numpy(m.xyz), torch.from_numpy(m.tri.view(np.int32)), (0, 0, 1), 96)
    torch.cuda.synchronize()
    assert _eq(img_d, img_h)


@pytest.mark.parametrize("slack,max_count", [(0, 0), (7, 0), (0, 500)])
def test_sample_order_batched_host_to_host(bs, slack, max_count):
    """Host meshes to host results in one call equal sampling + ordering on device buffers;
    slack > 0 leaves gaps between the parts' rows (no single copy for back-to-back arrays)."""
    specs = W.batch_parts(60, seed=9)
    meshes = [sp.mesh() for sp in specs]
    vofs, tofs, xyz, tri, rgb = _packed(meshes)
    res = [sp.res for sp in specs]
    n_v, n_t = np.diff(vofs), np.diff(tofs)
    dev = bs.sample_visible_packed(torch.from_numpy(xyz).cuda(), torch.from_numpy(tri).cuda(),
                                   torch.from_numpy(rgb).cuda(), vofs[:-1], n_v, tofs[:-1], n_t, res, W.AXIS_DIRS,
                                   caps=[6 * r * r for r in res])
    n = dev["n"]
    caps = n + slack
    got = bs.sample_order_batched(xyz, tri, rgb, vofs[:-1], n_v, tofs[:-1], n_t, res, W.AXIS_DIRS, caps, seeds=4,
                                  max_counts=max_count)
    assert np.array_equal(got["n"], n)
    keys = [dev["key"][int(dev["ofs"][i]):int(dev["ofs"][i]) + int(n[i])] for i in range(len(n))]
    want = bs.order_batched(keys, seeds=[4] * len(n), part_ids=list(range(len(n))), scales=list(dev["scale"]),
                            max_counts=[max_count] * len(n))
    torch.cuda.synchronize()
    ofs = got["ofs"]
    for i in range(len(n)):
        a, m_ = int(ofs[i]), len(want[i][0])
        d0 = int(dev["ofs"][i])
        assert got["key"][a:a + n[i]].tobytes() == dev["key"][d0:d0 + n[i]].cpu().numpy().tobytes(), i
        assert got["nrm"][a:a + n[i]].tobytes() == dev["nrm"][d0:d0 + n[i]].cpu().numpy().tobytes(), i
        assert got["perm"][a:a + m_].tobytes() == want[i][0].cpu().numpy().tobytes(), i
        assert got["rad2"][a:a + m_].tobytes() == want[i][1].cpu().numpy().tobytes(), i
        assert got["radius"][a:a + m_].tobytes() == want[i][2].cpu().numpy().tobytes(), i


def test_sample_order_batched_device_and_overflow(bs):
    specs = W.batch_parts(12, seed=13)
    meshes = [sp.mesh() for sp in specs]
    vofs, tofs, xyz, tri, rgb = _packed(meshes)
    res = [sp.res for sp in specs]
    n_v, n_t = np.diff(vofs), np.diff(tofs)
    host = bs.sample_order_batched(xyz, tri, rgb, vofs[:-1], n_v, tofs[:-1], n_t, res, W.AXIS_DIRS,
                                   [6 * r * r for r in res], seeds=2)
    devg = bs.sample_order_batched(torch.from_numpy(xyz).cuda(), torch.from_numpy(tri).cuda(),
                                   torch.from_numpy(rgb).cuda(), vofs[:-1], n_v, tofs[:-1], n_t, res, W.AXIS_DIRS,
                                   [6 * r * r for r in res], seeds=2)
    torch.cuda.synchronize()
    assert np.array_equal(host["n"], devg["n"])
    for i in range(len(res)):
        a, k = int(host["ofs"][i]), int(host["n"][i])
        for name in ("key", "perm", "rad2", "radius"):
            assert host[name][a:a + k].tobytes() == devg[name][a:a + k].cpu().numpy().tobytes(), (i, name)
    small = [int(v) - 1 for v in host["n"]]
    with pytest.raises(bs.BsError) as e:
        bs.sample_order_batched(xyz, tri, rgb, vofs[:-1], n_v, tofs[:-1], n_t, res, W.AXIS_DIRS, small, seeds=2)
    assert e.value.status == bs.BS_EOVERFLOW
