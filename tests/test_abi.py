"""CPU checks of the C-ABI boundary: libbs.so builds, loads and exports what include/bs.h declares."""
import ctypes as C
import os
import re

import pytest

from paper_1904_08225_gb300 import bs, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bs.h")).read()
    decl = r"^(?:bs_status|bs_server\s*\*|void|double|const char\s*\*)\s*(bs_[a-z_]+)\s*\("
    return sorted(set(re.findall(decl, src, flags=re.M)))


def test_header_and_binding_agree():
    assert _declared() == sorted(bs.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(build.build())
    for name in _declared():
        assert hasattr(lib, name), name


def test_error_message_and_tuning_validation():
    lib = bs.load()
    assert lib.bs_set_tuning(b"order_threads", 100) == bs.BS_EINVAL
    assert "order_threads" in bs.last_error()
    assert lib.bs_set_tuning(b"nope", 1) == bs.BS_EINVAL
    assert lib.bs_set_tuning(b"order_threads", 0) == bs.BS_OK
    assert lib.bs_set_tuning(b"order_quarters", 3) == bs.BS_EINVAL
    assert lib.bs_set_tuning(b"order_quarters", 0) == bs.BS_OK
    assert lib.bs_set_tuning(b"order_full_parts", -1) == bs.BS_EINVAL
    assert lib.bs_set_tuning(b"order_full_parts", 0) == bs.BS_OK


def test_bad_arguments_rejected_without_gpu():
    """Argument checks happen on the host before any device call."""
    lib = bs.load()
    s = bs.Surfels(None, None, None, None, 0, 0, (C.c_float * 3)(), 1.0)
    o = bs.OrderOpts(0, 0, -1, 0)
    assert lib.bs_order(C.byref(s), C.byref(o), None, None, None, None) == bs.BS_EINVAL
    s.n = 1 << 40
    assert lib.bs_order(C.byref(s), C.byref(o), None, None, None, None) == bs.BS_EOVERFLOW
    mesh = bs.Mesh(None, 0, None, 0, None)
    d = (bs.Dir * 1)(bs.Dir(0, 0, 1))
    out = bs.Surfels(None, None, None, None, 0, 0, (C.c_float * 3)(), 0.0)
    assert lib.bs_sample_visible(C.byref(mesh), d, 1, 64, C.byref(out), None) == bs.BS_EINVAL
    mesh.nverts = 3
    mesh.xyz = 16          # a placeholder device address: never dereferenced, the checks come first
    mesh.on_device = 1
    assert lib.bs_sample_visible(C.byref(mesh), d, 1, 0, C.byref(out), None) == bs.BS_EINVAL
    host = bs.Mesh(16, 3, None, 0, None, 0)  # host arrays: scalar checks come before any upload
    assert lib.bs_sample_visible(C.byref(host), d, 1, 0, C.byref(out), None) == bs.BS_EINVAL
    assert lib.bs_sample_visible(C.byref(host), d, 0, 64, C.byref(out), None) == bs.BS_EINVAL
    ress = (C.c_int * 1)(5000)
    res_ = (bs.PartResult * 1)()
    assert lib.bs_sample_order_batched(C.byref(host), ress, 1, d, 1, C.byref(o), res_, 0, None) == bs.BS_EINVAL
    assert lib.bs_sample_visible(C.byref(mesh), d, 0, 64, C.byref(out), None) == bs.BS_EINVAL
    bad = (bs.Dir * 1)(bs.Dir(0, 0, 0))
    assert lib.bs_sample_visible(C.byref(mesh), bad, 1, 64, C.byref(out), None) == bs.BS_EINVAL
    bad = (bs.Dir * 1)(bs.Dir(2, 0, 0))
    assert lib.bs_sample_visible(C.byref(mesh), bad, 1, 64, C.byref(out), None) == bs.BS_EINVAL
    st = C.c_int(0)
    assert lib.bs_server_create(0, 0, C.byref(st)) is None and st.value == bs.BS_EINVAL


def test_numpy_struct_layout_matches_ctypes():
    """The packed bindings fill struct arrays through numpy views; their layout must be the
    ctypes (and so the C header's) layout."""
    import numpy as np
    from paper_1904_08225_gb300 import bs
    a, arr = bs._struct_array(bs.Mesh, 3)
    a["xyz"] = [16, 32, 48]
    a["ntris"] = [1, 2, 3]
    a["face_rgb"] = 2**40 + 8
    assert arr[1].xyz == 32 and arr[2].ntris == 3 and arr[0].face_rgb == 2**40 + 8
    s, sarr = bs._struct_array(bs.Surfels, 2)
    s["n"] = [5, 6]
    s["bbox_min"][1] = [1.5, 2.5, 3.5]
    s["scale"] = 0.25
    assert sarr[1].n == 6 and list(sarr[1].bbox_min) == [1.5, 2.5, 3.5] and sarr[0].scale == 0.25
    sarr[0].n = 99  # and back: the C side writes n through the same memory
    assert s["n"][0] == 99
    o, oarr = bs._struct_array(bs.OrderOpts, 2)
    o["seed"] = np.uint64(2**63 + 1)
    o["start"] = -1
    o["sample_step"] = 500
    assert oarr[1].seed == 2**63 + 1 and oarr[1].start == -1 and oarr[0].sample_step == 500
