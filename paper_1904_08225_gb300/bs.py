"""ctypes binding of libbs (include/bs.h): argument marshalling only.

Every step of sampling and ordering runs in the CUDA kernels of libbs.so; this
module allocates output tensors with PyTorch (device memory and streams are the
only things taken from it), passes raw pointers and sizes across the C ABI and
turns status codes into exceptions.  There is no CPU fallback: if the library or
a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

BS_OK, BS_EINVAL, BS_ENOMEM, BS_EOVERFLOW, BS_ETIMEOUT, BS_EBUSY, BS_ECUDA, BS_ENOTREADY, BS_ECANCELED = range(9)
STATUS_NAMES = ["BS_OK", "BS_EINVAL", "BS_ENOMEM", "BS_EOVERFLOW", "BS_ETIMEOUT", "BS_EBUSY", "BS_ECUDA",
                "BS_ENOTREADY", "BS_ECANCELED"]
INT64_MAX = (1 << 63) - 1

# symbols include/bs.h declares; the library must export every one
EXPORTS = ["bs_sample_visible", "bs_sample_visible_batched", "bs_order", "bs_order_noalloc", "bs_order_batched", "bs_server_create", "bs_server_submit",
           "bs_server_poll", "bs_server_times", "bs_server_cancel", "bs_server_destroy", "bs_set_tuning", "bs_last_launch_ms",
           "bs_prefix_median_nn", "bs_prefix_for_radius", "bs_prefix_estimate", "bs_scene_generate", "bs_sample_splats",
           "bs_prefix_for_radius_batched", "bs_render_mesh", "bs_render_splats", "bs_parent_frames",
           "bs_sample_order_batched",
           "bs_last_error"]


class BsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class Mesh(C.Structure):
    """bs_mesh: device pointers with on_device=1; host pointers (uploaded by the library) with 0."""
    _fields_ = [("xyz", C.c_void_p), ("nverts", C.c_uint32), ("tri", C.c_void_p), ("ntris", C.c_uint32),
                ("face_rgb", C.c_void_p), ("on_device", C.c_int32)]


class PartResult(C.Structure):
    """bs_part_result: one part's outputs of bs_sample_order_batched."""
    _fields_ = [("key", C.c_void_p), ("nrm", C.c_void_p), ("rgb", C.c_void_p), ("src", C.c_void_p),
                ("perm", C.c_void_p), ("rad2", C.c_void_p), ("radius", C.c_void_p), ("cap", C.c_uint64),
                ("n", C.c_uint64), ("bbox_min", C.c_float * 3), ("scale", C.c_double)]


class Dir(C.Structure):
    _fields_ = [("x", C.c_int8), ("y", C.c_int8), ("z", C.c_int8)]


class Surfels(C.Structure):
    _fields_ = [("key", C.c_void_p), ("nrm", C.c_void_p), ("rgb", C.c_void_p), ("src", C.c_void_p),
                ("n", C.c_uint64), ("cap", C.c_uint64), ("bbox_min", C.c_float * 3), ("scale", C.c_double)]


class SplatSet(C.Structure):
    _fields_ = [("key", C.c_void_p), ("nrm", C.c_void_p), ("rgb", C.c_void_p), ("perm", C.c_void_p),
                ("n", C.c_uint64), ("bbox_min", C.c_float * 3), ("scale", C.c_double), ("r2", C.c_int64),
                ("node", C.c_uint32)]


class SplatNode(C.Structure):
    _fields_ = [("frame_min", C.c_float * 3), ("scale", C.c_double), ("res", C.c_int32)]


class OrderOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("part_id", C.c_uint32), ("start", C.c_int64), ("max_count", C.c_uint64),
                ("variant", C.c_int32), ("sample_size", C.c_uint32), ("sample_step", C.c_uint32)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True) -> C.CDLL:
    """Load libbs.so (compiling it first when sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_stale else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libbs.so not found at {path}: build it with paper_1904_08225_gb300.build")
            lib = C.CDLL(path)
            P = C.c_void_p
            lib.bs_sample_visible.argtypes = [C.POINTER(Mesh), C.POINTER(Dir), C.c_int, C.c_int, C.POINTER(Surfels), P]
            lib.bs_sample_visible_batched.argtypes = [C.POINTER(Mesh), C.POINTER(C.c_int), C.c_int, C.POINTER(Dir),
                                                      C.c_int, C.POINTER(Surfels), P]
            lib.bs_prefix_for_radius_batched.argtypes = [P, P, P, C.c_int, P, P, P]
            lib.bs_sample_order_batched.argtypes = [P, P, C.c_int, P, C.c_int, P, P, C.c_int, P]
            lib.bs_parent_frames.argtypes = [P, P, P, C.c_int, P, P, P, P]
            lib.bs_render_mesh.argtypes = [C.POINTER(Mesh), C.POINTER(Dir), C.c_int, P, P]
            lib.bs_render_splats.argtypes = [C.POINTER(SplatSet), C.c_int, C.POINTER(SplatNode), C.POINTER(Dir), P, P]
            lib.bs_sample_splats.argtypes = [C.POINTER(SplatSet), C.c_int, C.POINTER(SplatNode), C.c_int,
                                             C.POINTER(Dir), C.c_int, C.POINTER(Surfels), P]
            lib.bs_order.argtypes = [C.POINTER(Surfels), C.POINTER(OrderOpts), P, P, P, P]
            lib.bs_order_noalloc.argtypes = [C.POINTER(Surfels), C.POINTER(OrderOpts), P, P, P, P]
            lib.bs_order_batched.argtypes = [C.POINTER(Surfels), C.c_int, C.POINTER(OrderOpts), P, P, P, P]
            lib.bs_server_create.argtypes = [C.c_uint64, C.c_int, C.POINTER(C.c_int)]
            lib.bs_server_create.restype = P
            lib.bs_server_submit.argtypes = [P, P, C.c_uint64, C.c_double, C.POINTER(OrderOpts), C.POINTER(C.c_uint64)]
            lib.bs_server_poll.argtypes = [P, C.c_uint64, P, P, P]
            lib.bs_server_times.argtypes = [P, C.c_uint64, P]
            lib.bs_server_destroy.argtypes = [P]
            lib.bs_server_cancel.argtypes = [P, C.c_uint64]
            lib.bs_set_tuning.argtypes = [C.c_char_p, C.c_int]
            lib.bs_last_launch_ms.argtypes = [C.c_char_p, C.POINTER(C.c_double)]
            lib.bs_prefix_median_nn.argtypes = [C.POINTER(Surfels), P, C.c_uint64, C.POINTER(C.c_int64), P]
            lib.bs_prefix_for_radius.argtypes = [P, C.c_uint64, C.c_int64, C.POINTER(C.c_uint64), P]
            lib.bs_prefix_estimate.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
            lib.bs_scene_generate.argtypes = [C.c_uint64, P, P, P, C.c_int, C.c_int, C.c_int, P, P, P, C.c_float,
                                              C.c_float, C.c_int, P, P, P, P]
            lib.bs_last_error.restype = C.c_char_p
            for fn in EXPORTS[:-1]:
                if fn not in ("bs_server_create", "bs_server_destroy", "bs_prefix_estimate"):
                    getattr(lib, fn).restype = C.c_int
            lib.bs_prefix_estimate.restype = C.c_double
            _lib = lib
    return _lib


def last_error() -> str:
    return load().bs_last_error().decode()


def _check(st: int, where: str):
    if st != BS_OK:
        raise BsError(st, where, last_error())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libbs needs a CUDA GPU; none is available")
    return torch


def _out_device(t):
    """Where the library writes its outputs: the tensor's own device, or the current CUDA
    device for a host (CPU) tensor -- the kernels write only device memory."""
    torch = _torch()
    return t.device if t.is_cuda else torch.device("cuda", torch.cuda.current_device())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def set_tuning(name: str, value: int):
    _check(load().bs_set_tuning(name.encode(), int(value)), "bs_set_tuning")


def last_launch_ms(kernel: str) -> float:
    """Device ms of the latest timed launch of an internal kernel (needs set_tuning("kernel_timing", 1))."""
    ms = C.c_double(0.0)
    _check(load().bs_last_launch_ms(kernel.encode(), C.byref(ms)), "bs_last_launch_ms")
    return ms.value


def scene_generate(seed: int, parts, nboxes: int = 200, ncyl: int = 50, stream=None, device=None,
                   local_indices: bool = False, out=None):
    """bs_scene_generate: CUDA tensors (xyz, tri as int32 view, rgb) of the concatenated parts.

    parts: list of (part_id, line, slot).  Tables and placement steps come from workloads.
    out: optional (xyz, tri, rgb) contiguous tensors of the right sizes to write into."""
    torch = _torch()
    from . import workloads as W
    lib = load()
    n = len(parts)
    pid = np.array([p[0] for p in parts], np.uint64)
    ln = np.array([p[1] for p in parts], np.int32)
    sl = np.array([p[2] for p in parts], np.int32)
    V = n * (W.BOX_VERTS * nboxes + W.CYL_VERTS * ncyl)
    T = n * (W.BOX_TRIS * nboxes + W.CYL_TRIS * ncyl)
    dev = device or torch.device("cuda")
    if out is None:
        xyz = torch.empty((V, 3), dtype=torch.float32, device=dev)
        tri = torch.empty((T, 3), dtype=torch.int32, device=dev)
        rgb = torch.empty((T, 3), dtype=torch.uint8, device=dev)
    else:
        xyz, tri, rgb = out
        if (xyz.numel() != 3 * V or tri.numel() != 3 * T or rgb.numel() != 3 * T or not xyz.is_contiguous()
                or not tri.is_contiguous() or not rgb.is_contiguous()):
            raise ValueError("scene_generate: out tensors of the wrong size or not contiguous")
    st = lib.bs_scene_generate(int(seed) & (2**64 - 1), pid.ctypes.data_as(C.c_void_p), ln.ctypes.data_as(C.c_void_p),
                               sl.ctypes.data_as(C.c_void_p), n, nboxes, ncyl,
                               W.SIZE_TABLE.ctypes.data_as(C.c_void_p), W.COS32.ctypes.data_as(C.c_void_p),
                               W.SIN32.ctypes.data_as(C.c_void_p), float(W.SCENE_DX), float(W.SCENE_DY),
                               int(local_indices), C.c_void_p(xyz.data_ptr()), C.c_void_p(tri.data_ptr()), C.c_void_p(rgb.data_ptr()),
                               _stream(stream))
    _check(st, "bs_scene_generate")
    return xyz, tri, rgb


def prefix_median_nn(key, perm, pm: int, stream=None) -> int:
    """Sec. 4.1 r_m^2 (lower-median squared NN distance inside the first pm surfels)."""
    lib = load()
    s = Surfels(key.data_ptr(), None, None, None, key.shape[0], key.shape[0], (C.c_float * 3)(), 1.0)
    out = C.c_int64(0)
    _check(lib.bs_prefix_median_nn(C.byref(s), C.c_void_p(perm.data_ptr()), int(pm), C.byref(out), _stream(stream)),
           "bs_prefix_median_nn")
    return out.value


def prefix_for_radius(rad2, r2: int, stream=None) -> int:
    """Sec. 4.1: shortest prefix of an exact ordering reaching every point within sqrt(r2)."""
    lib = load()
    out = C.c_uint64(0)
    _check(lib.bs_prefix_for_radius(C.c_void_p(rad2.data_ptr()), rad2.shape[0], int(r2), C.byref(out),
                                    _stream(stream)), "bs_prefix_for_radius")
    return out.value


def prefix_for_radius_batched(rad2s, ms, r2s, stream=None):
    """bs_prefix_for_radius_batched: (p, r2_at) int arrays for many orderings.

    rad2s: list of CUDA int64 tensors (or raw device addresses); ms, r2s: ints per part."""
    lib = load()
    P = len(ms)
    ptrs = np.ascontiguousarray([t if isinstance(t, (int, np.integer)) else t.data_ptr() for t in rad2s],
                                dtype=np.uintp)
    m = np.ascontiguousarray(ms, dtype=np.uint64)
    r2 = np.ascontiguousarray(r2s, dtype=np.int64)
    p = np.zeros(P, np.uint64)
    at = np.zeros(P, np.int64)
    if P:
        _check(lib.bs_prefix_for_radius_batched(C.c_void_p(ptrs.ctypes.data), C.c_void_p(m.ctypes.data),
                                                C.c_void_p(r2.ctypes.data), P, C.c_void_p(p.ctypes.data),
                                                C.c_void_p(at.ctypes.data), _stream(stream)),
               "bs_prefix_for_radius_batched")
    return p, at


def parent_frames(child_mins, child_scales, children_of, parent_res):
    """bs_parent_frames: frames of parent nodes and their children's prefix targets (Sec. 3.4).

    child_mins (C,3) float32 and child_scales (C,) of every child; children_of: per parent
    the list of its child indices (each child listed once, parents in order); parent_res:
    per parent.  Returns (frame_min float32 (P,3), frame_scale float64 (P,), child_r2
    int64 per listed child in listing order)."""
    lib = load()
    order = [c for cs in children_of for c in cs]
    mins = np.ascontiguousarray(np.asarray(child_mins, np.float32).reshape(-1, 3)[order])
    scales = np.ascontiguousarray(np.asarray(child_scales, np.float64).reshape(-1)[order])
    ofs = np.ascontiguousarray(np.concatenate([[0], np.cumsum([len(cs) for cs in children_of])]), dtype=np.uint64)
    res = np.ascontiguousarray(parent_res, dtype=np.int32)
    P = len(children_of)
    fmin = np.zeros((P, 3), np.float32)
    fs = np.zeros(P, np.float64)
    r2 = np.zeros(len(order), np.int64)
    _check(lib.bs_parent_frames(C.c_void_p(mins.ctypes.data), C.c_void_p(scales.ctypes.data),
                                C.c_void_p(ofs.ctypes.data), P, C.c_void_p(res.ctypes.data),
                                C.c_void_p(fmin.ctypes.data), C.c_void_p(fs.ctypes.data), C.c_void_p(r2.ctypes.data)),
           "bs_parent_frames")
    return fmin, fs, r2


def sample_order_batched(xyz, tri, rgb, vofs, nverts, tofs, ntris, res, dirs, caps, seeds=0, part_ids=None,
                         max_counts=0, stream=None, out=None):
    """bs_sample_order_batched over parts packed in shared buffers, host to host or device to
    device: xyz float32 (V,3), tri uint32/int32 (T,3) with part-local indices, rgb uint8
    (T,3) or None -- numpy arrays (host meshes, uploaded by the library) or CUDA tensors.
    Part i: vertices vofs[i]:+nverts[i], triangles tofs[i]:+ntris[i], at most caps[i]
    surfels.  out: optional dict of preallocated flat outputs (key, nrm, rgb, src, perm,
    rad2, radius; host numpy arrays or CUDA tensors, sum(caps) rows, part i at
    ofs[i] = sum(caps[:i])); host outputs are allocated when out is None and the meshes
    are numpy arrays.  Returns dict(out arrays..., ofs, n, bbox_min, scale)."""
    lib = load()
    vofs, nverts = np.asarray(vofs, np.int64), np.asarray(nverts, np.int64)
    tofs, ntris = np.asarray(tofs, np.int64), np.asarray(ntris, np.int64)
    P = len(vofs)

    def is_dev(a):
        return hasattr(a, "is_cuda") and a.is_cuda

    def addr(a):  # torch tensors (host or device) or numpy arrays (host)
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

    on_dev = is_dev(xyz)
    if any(is_dev(a) != on_dev for a in (tri, rgb) if a is not None):
        raise ValueError("xyz, tri and rgb must all be host arrays or all device tensors")
    d = np.asarray(dirs, dtype=np.int8).reshape(-1, 3)
    darr = (Dir * len(d))(*[Dir(int(a), int(b), int(c)) for a, b, c in d])
    capv = np.asarray(caps, np.int64)
    ofs = np.concatenate([[0], np.cumsum(capv)]).astype(np.int64)
    tot = int(ofs[-1])
    if out is None:
        if on_dev:
            torch = _torch()
            dev = _out_device(xyz)
            out = dict(key=torch.empty(tot, dtype=torch.int64, device=dev),
                       nrm=torch.empty((tot, 3), dtype=torch.int16, device=dev),
                       rgb=torch.empty((tot, 3), dtype=torch.uint8, device=dev),
                       src=torch.empty(tot, dtype=torch.int32, device=dev),
                       perm=torch.empty(tot, dtype=torch.int32, device=dev),
                       rad2=torch.empty(tot, dtype=torch.int64, device=dev),
                       radius=torch.empty(tot, dtype=torch.float32, device=dev))
        else:
            out = dict(key=np.empty(tot, np.uint64), nrm=np.empty((tot, 3), np.int16), rgb=np.empty((tot, 3), np.uint8),
                       src=np.empty(tot, np.uint32), perm=np.empty(tot, np.uint32), rad2=np.empty(tot, np.int64),
                       radius=np.empty(tot, np.float32))
    out_dev = is_dev(out["perm"])
    if any(is_dev(a) != out_dev for a in out.values() if a is not None):
        raise ValueError("the outputs must all be host arrays or all device tensors")
    mnp, marr = _struct_array(Mesh, P)
    mnp["xyz"] = addr(xyz) + 12 * vofs
    mnp["nverts"] = nverts
    mnp["tri"] = addr(tri) + 12 * tofs
    mnp["ntris"] = ntris
    mnp["face_rgb"] = 0 if rgb is None else addr(rgb) + 3 * tofs
    mnp["on_device"] = 1 if on_dev else 0
    onp, oarr = _struct_array(PartResult, P)
    width = dict(key=8, nrm=6, rgb=3, src=4, perm=4, rad2=8, radius=4)
    for name, w in width.items():
        a = out.get(name)
        onp[name] = 0 if a is None else addr(a) + w * ofs[:-1]
    onp["cap"] = capv
    opts = (OrderOpts * P)()
    pid = range(P) if part_ids is None else part_ids
    sd = np.broadcast_to(np.asarray(seeds, np.int64), (P,))
    mc = np.broadcast_to(np.asarray(max_counts, np.int64), (P,))
    for i, p_ in enumerate(pid):
        opts[i] = _opts(int(sd[i]), int(p_), -1, int(mc[i]))
    rarr = (C.c_int * P)(*np.broadcast_to(np.asarray(res, np.int64), (P,)).tolist())
    st = lib.bs_sample_order_batched(marr, rarr, P, darr, len(d), opts, oarr, 1 if out_dev else 0, _stream(stream))
    _check(st, "bs_sample_order_batched")
    return dict(out, ofs=ofs, n=onp["n"].astype(np.int64), bbox_min=onp["bbox_min"].copy(),
                scale=onp["scale"].copy())


def prefix_estimate(pm: int, rm2: int, r2: int) -> float:
    """The paper's p(r) = pm (r_m / r)^2."""
    return load().bs_prefix_estimate(int(pm), int(rm2), int(r2))


def sample_visible(xyz, tri, rgb, dirs, res: int, stream=None, cap: int | None = None):
    """Visible-surface surfels of a mesh (Sec. 3.1) via bs_sample_visible.

    xyz float32 (V,3), tri int32/uint32 (T,3), rgb uint8 (T,3) or None: CUDA tensors.
    dirs: (D,3) integer directions.  Returns dict(key u64-as-int64 (N,), nrm int16 (N,3),
    rgb uint8 (N,3), src int32-view of u32 (N,), bbox_min (3,), scale float).
    """
    torch = _torch()
    lib = load()
    d = np.asarray(dirs, dtype=np.int8).reshape(-1, 3)
    darr = (Dir * len(d))(*[Dir(int(a), int(b), int(c)) for a, b, c in d])
    dev = _out_device(xyz)
    xyz = xyz.contiguous()
    tri = tri.contiguous()
    rgb = rgb.contiguous() if rgb is not None else None
    mesh = Mesh(xyz.data_ptr(), xyz.shape[0], tri.data_ptr() if tri.numel() else None, tri.shape[0],
                rgb.data_ptr() if rgb is not None else None, 1 if xyz.is_cuda else 0)
    if cap is None:
        cap = len(d) * res * res
    key = torch.empty(cap, dtype=torch.int64, device=dev)
    nrm = torch.empty((cap, 3), dtype=torch.int16, device=dev)
    col = torch.empty((cap, 3), dtype=torch.uint8, device=dev)
    src = torch.empty(cap, dtype=torch.int32, device=dev)
    out = Surfels(key.data_ptr(), nrm.data_ptr(), col.data_ptr(), src.data_ptr(), 0, cap, (C.c_float * 3)(), 0.0)
    st = lib.bs_sample_visible(C.byref(mesh), darr, len(d), int(res), C.byref(out), _stream(stream))
    _check(st, "bs_sample_visible")
    n = int(out.n)
    return dict(key=key[:n], nrm=nrm[:n], rgb=col[:n], src=src[:n], n=n,
                bbox_min=np.array(list(out.bbox_min), np.float32), scale=float(out.scale))


def sample_visible_batched(meshes, res, dirs, stream=None, caps=None):
    """bs_sample_visible_batched over a list of (xyz, tri, rgb-or-None) CUDA tensor triples.

    res: per-part resolutions.  Returns a list of dicts like sample_visible()."""
    torch = _torch()
    lib = load()
    P = len(meshes)
    d = np.asarray(dirs, dtype=np.int8).reshape(-1, 3)
    darr = (Dir * len(d))(*[Dir(int(a), int(b), int(c)) for a, b, c in d])
    marr = (Mesh * P)()
    rarr = (C.c_int * P)(*[int(r) for r in res])
    outs = (Surfels * P)()
    keep = []
    capl = [int(caps[i]) if caps is not None else len(d) * int(res[i]) ** 2 for i in range(P)]
    ofs = np.concatenate([[0], np.cumsum(capl)]).astype(np.int64)
    dev = _out_device(meshes[0][0]) if P else None
    tot = int(ofs[-1])
    # one allocation per field; part i owns rows ofs[i]:ofs[i+1]
    key = torch.empty(tot, dtype=torch.int64, device=dev)
    nrm = torch.empty((tot, 3), dtype=torch.int16, device=dev)
    col = torch.empty((tot, 3), dtype=torch.uint8, device=dev)
    src = torch.empty(tot, dtype=torch.int32, device=dev)
    for i, (xyz, tri, rgb) in enumerate(meshes):
        xyz, tri = xyz.contiguous(), tri.contiguous()
        rgb = rgb.contiguous() if rgb is not None else None
        keep.append((xyz, tri, rgb))
        marr[i] = Mesh(xyz.data_ptr(), xyz.shape[0], tri.data_ptr() if tri.numel() else None, tri.shape[0],
                       rgb.data_ptr() if rgb is not None else None, 1 if xyz.is_cuda else 0)
        o = int(ofs[i])
        outs[i] = Surfels(key.data_ptr() + 8 * o, nrm.data_ptr() + 6 * o, col.data_ptr() + 3 * o,
                          src.data_ptr() + 4 * o, 0, capl[i], (C.c_float * 3)(), 0.0)
    st = lib.bs_sample_visible_batched(marr, rarr, P, darr, len(d), outs, _stream(stream))
    _check(st, "bs_sample_visible_batched")
    res_list = []
    for i in range(P):
        o = int(ofs[i])
        n = int(outs[i].n)
        res_list.append(dict(key=key[o:o + n], nrm=nrm[o:o + n], rgb=col[o:o + n], src=src[o:o + n], n=n,
                             bbox_min=np.array(list(outs[i].bbox_min), np.float32), scale=float(outs[i].scale)))
    return res_list


def sample_splats(sets, nodes, dirs, caps=None, stream=None):
    """bs_sample_splats: parent nodes sampled from child surfels drawn as oriented discs.

    sets: list of dicts with key (CUDA int64 (n,)), nrm (CUDA int16 (n,3)), rgb (CUDA uint8
    (n,3) or None), perm (CUDA int32 view of u32 or None; splat i = surfel perm[i]), n,
    bbox_min (3 floats), scale, r2 (squared disc radius in the set's units) and node.
    nodes: list of (frame_min (3 floats), scale, res).  dirs: axis directions.
    Returns one dict per node like sample_visible()."""
    torch = _torch()
    lib = load()
    d = np.asarray(dirs, dtype=np.int8).reshape(-1, 3)
    darr = (Dir * len(d))(*[Dir(int(a), int(b), int(c)) for a, b, c in d])
    S = len(sets)
    sarr = (SplatSet * max(S, 1))()
    for i, st in enumerate(sets):
        sarr[i] = SplatSet(st["key"].data_ptr(), st["nrm"].data_ptr(),
                           st["rgb"].data_ptr() if st.get("rgb") is not None else None,
                           st["perm"].data_ptr() if st.get("perm") is not None else None,
                           int(st["n"]), (C.c_float * 3)(*[float(x) for x in st["bbox_min"]]), float(st["scale"]),
                           int(st["r2"]), int(st["node"]))
    K = len(nodes)
    narr = (SplatNode * K)(*[SplatNode((C.c_float * 3)(*[float(x) for x in fm]), float(sc), int(r))
                             for fm, sc, r in nodes])
    capl = [int(caps[i]) if caps is not None else len(d) * int(nodes[i][2]) ** 2 for i in range(K)]
    ofs = np.concatenate([[0], np.cumsum(capl)]).astype(np.int64)
    dev = sets[0]["key"].device if sets else torch.device("cuda")
    tot = int(ofs[-1])
    key = torch.empty(tot, dtype=torch.int64, device=dev)
    nrm = torch.empty((tot, 3), dtype=torch.int16, device=dev)
    col = torch.empty((tot, 3), dtype=torch.uint8, device=dev)
    src = torch.empty(tot, dtype=torch.int32, device=dev)
    onp, oarr = _struct_array(Surfels, K)
    onp["key"] = key.data_ptr() + 8 * ofs[:-1]
    onp["nrm"] = nrm.data_ptr() + 6 * ofs[:-1]
    onp["rgb"] = col.data_ptr() + 3 * ofs[:-1]
    onp["src"] = src.data_ptr() + 4 * ofs[:-1]
    onp["cap"] = capl
    st_ = lib.bs_sample_splats(sarr, S, narr, K, darr, len(d), oarr, _stream(stream))
    _check(st_, "bs_sample_splats")
    out = []
    for i in range(K):
        o, n = int(ofs[i]), int(onp["n"][i])
        out.append(dict(key=key[o:o + n], nrm=nrm[o:o + n], rgb=col[o:o + n], src=src[o:o + n], n=n,
                        bbox_min=onp["bbox_min"][i].copy(), scale=float(onp["scale"][i])))
    return out


def render_mesh(xyz, tri, d, res: int, stream=None):
    """bs_render_mesh: (res, res) CUDA int64 image (uint64 bits) of depth << 32 | triangle."""
    torch = _torch()
    lib = load()
    xyz, tri = xyz.contiguous(), tri.contiguous()
    m = Mesh(xyz.data_ptr(), xyz.shape[0], tri.data_ptr() if tri.numel() else None, tri.shape[0], None,
             1 if xyz.is_cuda else 0)
    img = torch.empty((res, res), dtype=torch.int64, device=_out_device(xyz))
    dd = Dir(*[int(x) for x in d])
    _check(lib.bs_render_mesh(C.byref(m), C.byref(dd), int(res), C.c_void_p(img.data_ptr()), _stream(stream)),
           "bs_render_mesh")
    return img


def render_splats(sets, node, d, stream=None):
    """bs_render_splats: (res, res) CUDA int64 image (uint64 bits) of depth << 32 | splat.

    sets as for sample_splats (node fields ignored); node = (frame_min, scale, res)."""
    torch = _torch()
    lib = load()
    S = len(sets)
    sarr = (SplatSet * max(S, 1))()
    for i, st in enumerate(sets):
        sarr[i] = SplatSet(st["key"].data_ptr(), st["nrm"].data_ptr(),
                           st["rgb"].data_ptr() if st.get("rgb") is not None else None,
                           st["perm"].data_ptr() if st.get("perm") is not None else None,
                           int(st["n"]), (C.c_float * 3)(*[float(x) for x in st["bbox_min"]]), float(st["scale"]),
                           int(st["r2"]), 0)
    fm, sc, res = node
    nd = SplatNode((C.c_float * 3)(*[float(x) for x in fm]), float(sc), int(res))
    img = torch.empty((res, res), dtype=torch.int64, device=sets[0]["key"].device if sets else torch.device("cuda"))
    dd = Dir(*[int(x) for x in d])
    _check(lib.bs_render_splats(sarr, S, C.byref(nd), C.byref(dd), C.c_void_p(img.data_ptr()), _stream(stream)),
           "bs_render_splats")
    return img


def _np_dtype(ct) -> np.dtype:
    """numpy structured dtype with the layout of a ctypes Structure (pointers as uintp)."""
    names, formats, offsets = [], [], []
    for name, t in ct._fields_:
        names.append(name)
        offsets.append(getattr(ct, name).offset)
        if t is C.c_void_p:
            formats.append(np.uintp)
        elif issubclass(t, C.Array):
            formats.append((np.dtype(t._type_), t._length_))
        else:
            formats.append(np.dtype(t))
    return np.dtype(dict(names=names, formats=formats, offsets=offsets, itemsize=C.sizeof(ct)))


def _struct_array(ct, n: int):
    """(numpy structured array, ctypes array over the same memory) of n zeroed structs."""
    a = np.zeros(n, _np_dtype(ct))
    return a, (ct * n).from_buffer(a)


def sample_visible_packed(xyz, tri, rgb, vofs, nverts, tofs, ntris, res, dirs, caps=None, stream=None):
    """bs_sample_visible_batched over parts that share packed buffers (no per-part tensors).

    Part i: vertices xyz[vofs[i]:vofs[i]+nverts[i]], triangles tri[tofs[i]:tofs[i]+ntris[i]]
    with indices local to its vertices, face colours rgb[tofs[i]:...] (or rgb None).
    Returns dict(key, nrm, rgb, src: flat CUDA tensors; ofs int64 (P+1): part i's rows start
    at ofs[i]; n int64 (P,); bbox_min float32 (P,3); scale float64 (P,))."""
    torch = _torch()
    lib = load()
    vofs, nverts = np.asarray(vofs, np.int64), np.asarray(nverts, np.int64)
    tofs, ntris = np.asarray(tofs, np.int64), np.asarray(ntris, np.int64)
    P = len(vofs)
    d = np.asarray(dirs, dtype=np.int8).reshape(-1, 3)
    darr = (Dir * len(d))(*[Dir(int(a), int(b), int(c)) for a, b, c in d])
    resv = np.broadcast_to(np.asarray(res, np.int64), (P,))
    capv = (len(d) * resv * resv) if caps is None else np.broadcast_to(np.asarray(caps, np.int64), (P,))
    ofs = np.concatenate([[0], np.cumsum(capv)]).astype(np.int64)
    dev = _out_device(xyz)
    tot = int(ofs[-1])
    key = torch.empty(tot, dtype=torch.int64, device=dev)
    nrm = torch.empty((tot, 3), dtype=torch.int16, device=dev)
    col = torch.empty((tot, 3), dtype=torch.uint8, device=dev)
    src = torch.empty(tot, dtype=torch.int32, device=dev)
    mnp, marr = _struct_array(Mesh, P)
    mnp["xyz"] = xyz.data_ptr() + 12 * vofs
    mnp["nverts"] = nverts
    mnp["tri"] = tri.data_ptr() + 12 * tofs
    mnp["ntris"] = ntris
    mnp["face_rgb"] = 0 if rgb is None else rgb.data_ptr() + 3 * tofs
    mnp["on_device"] = 1 if xyz.is_cuda else 0
    onp, oarr = _struct_array(Surfels, P)
    onp["key"] = key.data_ptr() + 8 * ofs[:-1]
    onp["nrm"] = nrm.data_ptr() + 6 * ofs[:-1]
    onp["rgb"] = col.data_ptr() + 3 * ofs[:-1]
    onp["src"] = src.data_ptr() + 4 * ofs[:-1]
    onp["cap"] = capv
    rarr = (C.c_int * P)(*resv.tolist())
    st = lib.bs_sample_visible_batched(marr, rarr, P, darr, len(d), oarr, _stream(stream))
    _check(st, "bs_sample_visible_batched")
    return dict(key=key, nrm=nrm, rgb=col, src=src, ofs=ofs, n=onp["n"].astype(np.int64),
                bbox_min=onp["bbox_min"].copy(), scale=onp["scale"].copy())


def order_packed(key, kofs, n, max_counts=None, seeds=0, part_ids=None, scales=1.0, starts=-1, stream=None,
                 want_radius: bool = True, variant: int = 0, sample_size: int = 200, sample_step: int = 500):
    """bs_order_batched over parts stored in one flat key tensor: part i is key[kofs[i]:kofs[i]+n[i]].

    Returns (perm, rad2, radius-or-None flat tensors, mofs int64 (P+1)): part i's outputs are
    entries mofs[i]:mofs[i+1]."""
    torch = _torch()
    lib = load()
    kofs, n = np.asarray(kofs, np.int64)[:len(n)], np.asarray(n, np.int64)
    P = len(n)
    mc = np.zeros(P, np.int64) if max_counts is None else np.broadcast_to(np.asarray(max_counts, np.int64), (P,))
    m = np.where((mc == 0) | (mc > n), n, mc)
    mofs = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    dev = key.device
    perm = torch.empty(int(mofs[-1]), dtype=torch.int32, device=dev)
    rad2 = torch.empty(int(mofs[-1]), dtype=torch.int64, device=dev)
    radius = torch.empty(int(mofs[-1]), dtype=torch.float32, device=dev) if want_radius else None
    snp, sarr = _struct_array(Surfels, P)
    snp["key"] = key.data_ptr() + 8 * kofs
    snp["n"] = n
    snp["cap"] = n
    snp["scale"] = np.broadcast_to(np.asarray(scales, np.float64), (P,))
    onp, oarr = _struct_array(OrderOpts, P)
    onp["seed"] = np.broadcast_to(np.asarray(seeds, np.uint64), (P,))
    onp["part_id"] = np.arange(P) if part_ids is None else np.asarray(part_ids, np.uint32)
    onp["start"] = np.broadcast_to(np.asarray(starts, np.int64), (P,))
    onp["max_count"] = mc
    onp["variant"] = variant
    onp["sample_size"] = sample_size if variant == 1 else 0
    onp["sample_step"] = sample_step if variant == 1 else 0
    pp = np.ascontiguousarray(perm.data_ptr() + 4 * mofs[:-1], dtype=np.uintp)
    rp = np.ascontiguousarray(rad2.data_ptr() + 8 * mofs[:-1], dtype=np.uintp)
    fp = np.ascontiguousarray((radius.data_ptr() + 4 * mofs[:-1]) if want_radius else np.zeros(P), dtype=np.uintp)
    st = lib.bs_order_batched(sarr, P, oarr, C.c_void_p(pp.ctypes.data), C.c_void_p(rp.ctypes.data),
                              C.c_void_p(fp.ctypes.data), _stream(stream))
    _check(st, "bs_order_batched")
    return perm, rad2, radius, mofs


def _opts(seed=0, part_id=0, start=-1, max_count=0, variant=0, sample_size=200, sample_step=500) -> OrderOpts:
    return OrderOpts(int(seed) & (2**64 - 1), int(part_id), int(start), int(max_count), int(variant),
                     int(sample_size) if variant == 1 else 0, int(sample_step) if variant == 1 else 0)


def order(key, start: int = -1, seed: int = 0, part_id: int = 0, max_count: int = 0, scale: float = 1.0,
          stream=None, want_radius: bool = True, out=None, variant: int = 0, sample_size: int = 200,
          sample_step: int = 500):
    """Exact greedy permutation of one part (bs_order).  key: CUDA int64 tensor (N,).

    Returns (perm int32 view of u32 (m,), rad2 int64 (m,), radius float32 (m,) or None).
    """
    torch = _torch()
    lib = load()
    n = key.shape[0]
    m = n if max_count == 0 or max_count > n else max_count
    if out is None:
        perm = torch.empty(m, dtype=torch.int32, device=key.device)
        rad2 = torch.empty(m, dtype=torch.int64, device=key.device)
        radius = torch.empty(m, dtype=torch.float32, device=key.device) if want_radius else None
    else:
        perm, rad2, radius = out
    s = Surfels(key.data_ptr(), None, None, None, n, n, (C.c_float * 3)(), float(scale))
    o = _opts(seed, part_id, start, max_count, variant, sample_size, sample_step)
    st = lib.bs_order(C.byref(s), C.byref(o), _ptr(perm), _ptr(rad2), _ptr(radius), _stream(stream))
    _check(st, "bs_order")
    return perm, rad2, radius


def order_noalloc(key, start: int = -1, seed: int = 0, part_id: int = 0, max_count: int = 0, scale: float = 1.0,
                  stream=None, want_radius: bool = True, out=None):
    """bs_order_noalloc: same result as order(), with the library's fixed scratch instead of
    allocations (parts of at most 65536 points; calls that overlap on the GPU race)."""
    torch = _torch()
    lib = load()
    n = key.shape[0]
    m = n if max_count == 0 or max_count > n else max_count
    if out is None:
        perm = torch.empty(m, dtype=torch.int32, device=key.device)
        rad2 = torch.empty(m, dtype=torch.int64, device=key.device)
        radius = torch.empty(m, dtype=torch.float32, device=key.device) if want_radius else None
    else:
        perm, rad2, radius = out
    s = Surfels(key.data_ptr(), None, None, None, n, n, (C.c_float * 3)(), float(scale))
    o = _opts(seed, part_id, start, max_count)
    st = lib.bs_order_noalloc(C.byref(s), C.byref(o), _ptr(perm), _ptr(rad2), _ptr(radius), _stream(stream))
    _check(st, "bs_order_noalloc")
    return perm, rad2, radius


def order_batched(keys, starts=None, seeds=None, part_ids=None, max_counts=None, scales=None, stream=None,
                  want_radius: bool = True, outs=None, variants=None, sample_size: int = 200, sample_step: int = 500):
    """bs_order_batched over a list of CUDA int64 key tensors; returns a list of (perm, rad2, radius)."""
    torch = _torch()
    lib = load()
    P = len(keys)
    starts = starts if starts is not None else [-1] * P
    seeds = seeds if seeds is not None else [0] * P
    part_ids = part_ids if part_ids is not None else list(range(P))
    max_counts = max_counts if max_counts is not None else [0] * P
    scales = scales if scales is not None else [1.0] * P
    parts = (Surfels * P)()
    opts = (OrderOpts * P)()
    pp = (C.c_void_p * P)()
    rp = (C.c_void_p * P)()
    fp = (C.c_void_p * P)()
    result = []
    ms = [k.shape[0] if mc == 0 or mc > k.shape[0] else mc for k, mc in zip(keys, max_counts)]
    if outs is None and P:
        # one allocation per output field; part i owns entries mo[i]:mo[i+1]
        mo = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
        dev = keys[0].device
        perm_all = torch.empty(int(mo[-1]), dtype=torch.int32, device=dev)
        rad2_all = torch.empty(int(mo[-1]), dtype=torch.int64, device=dev)
        radius_all = torch.empty(int(mo[-1]), dtype=torch.float32, device=dev) if want_radius else None
    for i, k in enumerate(keys):
        n = k.shape[0]
        m = ms[i]
        if outs is None:
            a, b = int(mo[i]), int(mo[i + 1])
            perm, rad2 = perm_all[a:b], rad2_all[a:b]
            radius = radius_all[a:b] if want_radius else None
        else:
            perm, rad2, radius = outs[i]
        parts[i] = Surfels(k.data_ptr(), None, None, None, n, n, (C.c_float * 3)(), float(scales[i]))
        opts[i] = _opts(seeds[i], part_ids[i], starts[i], max_counts[i], variants[i] if variants else 0,
                        sample_size, sample_step)
        pp[i] = perm.data_ptr()
        rp[i] = rad2.data_ptr()
        fp[i] = radius.data_ptr() if radius is not None else None
        result.append((perm, rad2, radius))
    st = lib.bs_order_batched(parts, P, opts, C.cast(pp, C.c_void_p), C.cast(rp, C.c_void_p),
                              C.cast(fp, C.c_void_p), _stream(stream))
    _check(st, "bs_order_batched")
    return result


class Server:
    """Continuous-batching ordering server (bs_server_*); host arrays in and out."""

    def __init__(self, budget_bytes: int = 64 << 30, max_inflight: int = 0):
        _torch()
        self._lib = load()
        st = C.c_int(0)
        self._h = self._lib.bs_server_create(int(budget_bytes), int(max_inflight), C.byref(st))
        if not self._h:
            raise BsError(st.value, "bs_server_create", last_error())
        self._m = {}

    def submit(self, key: np.ndarray, scale: float = 1.0, start: int = -1, seed: int = 0, part_id: int = 0,
               max_count: int = 0, variant: int = 0, sample_size: int = 200, sample_step: int = 500) -> int:
        k = np.ascontiguousarray(key, dtype=np.uint64)
        t = C.c_uint64(0)
        o = _opts(seed, part_id, start, max_count, variant, sample_size, sample_step)
        st = self._lib.bs_server_submit(self._h, k.ctypes.data_as(C.c_void_p), k.shape[0], float(scale), C.byref(o),
                                        C.byref(t))
        _check(st, "bs_server_submit")
        n = k.shape[0]
        self._m[t.value] = n if max_count == 0 or max_count > n else max_count
        return t.value

    def poll(self, ticket: int):
        """(perm u32, rad2 i64, radius f32) numpy arrays, or None while not ready."""
        m = self._m[ticket]
        st = self._lib.bs_server_poll(self._h, ticket, None, None, None)
        if st == BS_ENOTREADY:
            return None
        _check(st, "bs_server_poll")
        perm = np.empty(m, np.uint32)
        rad2 = np.empty(m, np.int64)
        radius = np.empty(m, np.float32)
        st = self._lib.bs_server_poll(self._h, ticket, perm.ctypes.data_as(C.c_void_p),
                                      rad2.ctypes.data_as(C.c_void_p), radius.ctypes.data_as(C.c_void_p))
        if st == BS_ENOTREADY:
            return None
        _check(st, "bs_server_poll")
        return perm, rad2, radius

    def cancel(self, ticket: int) -> None:
        """bs_server_cancel: the request is dropped (polling it then raises BS_ECANCELED)."""
        _check(self._lib.bs_server_cancel(self._h, ticket), "bs_server_cancel")

    def times(self, ticket: int):
        t = (C.c_double * 3)()
        _check(self._lib.bs_server_times(self._h, ticket, t), "bs_server_times")
        return tuple(t)

    def close(self):
        if self._h:
            self._lib.bs_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
