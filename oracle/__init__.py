"""CPU oracle for surfel sampling and greedy-permutation ordering (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import this package; the product
path (``paper_1904_08225_gb300``) never does and shares no code with it.

The arithmetic lives in ``bs_oracle.c`` (plain C, compiled here with gcc and
``-ffp-contract=off``); this module only marshals numpy arrays.  Each function
cites the passage of Brandt et al., "Rendering of Complex Heterogenous Scenes
using Progressive Blue Surfels", that it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INT64_MAX = np.iinfo(np.int64).max
Q = (1 << 21) - 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            lib.or_philox4x32_10.argtypes = [P, P, P]
            lib.or_morton3.argtypes = [C.c_uint32] * 3
            lib.or_morton3.restype = C.c_uint64
            lib.or_quantise.argtypes = [P, C.c_uint64, P, P, P]
            lib.or_quantise.restype = C.c_int
            lib.or_frame.argtypes = [P, P]
            lib.or_raster_dir.argtypes = [P, C.c_uint64, P, C.c_uint64, P, C.c_int, P, P, P]
            lib.or_sample_visible.argtypes = [P, C.c_uint64, P, C.c_uint64, P, P, C.c_int, C.c_int,
                                              P, P, P, P, C.c_uint64]
            lib.or_sample_visible.restype = C.c_int64
            lib.or_start_index.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_int64, P]
            lib.or_start_index.restype = C.c_int
            lib.or_greedy.argtypes = [P, C.c_uint64, C.c_uint64, C.c_uint64, P, P, P, P, C.c_int]
            lib.or_greedy.restype = C.c_int
            lib.or_radius.argtypes = [P, C.c_uint64, C.c_double, P]
            lib.or_sampled.argtypes = [P, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                       C.c_uint32, P, P, P]
            lib.or_sampled.restype = C.c_int
            lib.or_prefix_median_nn.argtypes = [P, P, C.c_uint64]
            lib.or_prefix_median_nn.restype = C.c_int64
            lib.or_prefix_for_radius.argtypes = [P, C.c_uint64, C.c_int64]
            lib.or_prefix_for_radius.restype = C.c_uint64
            lib.or_num_threads.restype = C.c_int
            lib.or_sample_splats.argtypes = [C.c_uint64, P, P, P, C.c_int, P, P, P, P, P, C.c_double, P, C.c_int,
                                             C.c_int, P, P, P, P, C.c_uint64]
            lib.or_sample_splats.restype = C.c_int64
            lib.or_render_splats.argtypes = [C.c_uint64, P, P, C.c_int, P, P, P, P, P, C.c_double, P, C.c_int, P]
            lib.or_render_splats.restype = C.c_int
            lib.or_parent_frame.argtypes = [P, P, C.c_uint64, P, P]
            lib.or_parent_frame.restype = C.c_int
            lib.or_child_target_r2.argtypes = [C.c_double, C.c_double, C.c_int]
            lib.or_child_target_r2.restype = C.c_int64
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al., SC'11); the random start of Sec. 3.2."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    _load().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def morton3(x: int, y: int, z: int) -> int:
    return int(_load().or_morton3(x, y, z))


def quantise(xyz: np.ndarray):
    """Sec. 3.1 node-local positions as 21-bit integers: (q int32 (V,3), bbox_min, scale).

    Raises ValueError for a non-finite vertex or a zero extent.
    """
    x = np.ascontiguousarray(xyz, dtype=np.float32)
    q = np.zeros((x.shape[0], 3), np.int32)
    mn = np.zeros(3, np.float32)
    s = np.zeros(1, np.float64)
    if _load().or_quantise(_p(x), x.shape[0], _p(q), _p(mn), _p(s)) != 0:
        raise ValueError("mesh cannot be quantised (non-finite vertex or zero extent)")
    return q, mn, float(s[0])


def frame(d) -> tuple[np.ndarray, np.ndarray]:
    """Integer view frame (u, v) of direction d (Sec. 3.1 orthographic views)."""
    dd = np.ascontiguousarray(d, dtype=np.int8)
    f = np.zeros(9, np.int64)
    _load().or_frame(_p(dd), _p(f))
    return f[0:3].copy(), f[3:6].copy()


def raster_dir(q: np.ndarray, tri: np.ndarray, d, res: int, counts: bool = False):
    """Depth pass of one direction (Sec. 3.1): returns (depth u64 (res,res), fragments[, per-pixel count])."""
    qq = np.ascontiguousarray(q, dtype=np.int32)
    tt = np.ascontiguousarray(tri, dtype=np.uint32)
    dd = np.ascontiguousarray(d, dtype=np.int8)
    depth = np.zeros((res, res), np.uint64)
    nf = np.zeros(1, np.uint64)
    cnt = np.zeros((res, res), np.uint32) if counts else None
    _load().or_raster_dir(_p(qq), qq.shape[0], _p(tt), tt.shape[0], _p(dd), res, _p(depth), _p(nf),
                          _p(cnt) if counts else None)
    if counts:
        return depth, int(nf[0]), cnt
    return depth, int(nf[0])


def sample_visible(q: np.ndarray, tri: np.ndarray, rgb: np.ndarray | None, dirs, res: int):
    """Initial surfel set of Sec. 3.1: one surfel per covered pixel, duplicates merged.

    Returns dict(key u64 (N,), nrm i16 (N,3), rgb u8 (N,3), src u32 (N,)) in
    ascending Morton order of the quantised position.
    """
    lib = _load()
    qq = np.ascontiguousarray(q, dtype=np.int32)
    tt = np.ascontiguousarray(tri, dtype=np.uint32)
    dd = np.ascontiguousarray(dirs, dtype=np.int8).reshape(-1, 3)
    cc = None if rgb is None else np.ascontiguousarray(rgb, dtype=np.uint8)
    args = (_p(qq), qq.shape[0], _p(tt), tt.shape[0], None if cc is None else _p(cc), _p(dd), dd.shape[0], res)
    n = lib.or_sample_visible(*args, None, None, None, None, 0)
    if n < 0:
        raise ValueError(f"or_sample_visible failed ({n})")
    key = np.zeros(n, np.uint64)
    nrm = np.zeros((n, 3), np.int16)
    col = np.zeros((n, 3), np.uint8)
    src = np.zeros(n, np.uint32)
    n2 = lib.or_sample_visible(*args, _p(key), _p(nrm), _p(col), _p(src), n)
    assert n2 == n
    return dict(key=key, nrm=nrm, rgb=col, src=src)


def sample_mesh(mesh, dirs, res: int):
    """Quantise then sample a workloads.Mesh: returns (surfels dict, bbox_min, scale)."""
    q, mn, s = quantise(mesh.xyz)
    return sample_visible(q, mesh.tri, mesh.rgb, dirs, res), mn, s


def sample_splats(sets, frame_min, frame_scale: float, dirs, res: int):
    """Parent-node sampling from child surfels drawn as oriented discs (Sec. 3.4, Sec. 4.2).

    sets: list of dicts with key u64 (n,) in the set's own frame, nrm int16 (n,3),
    rgb uint8 (n,3) or None, bbox_min (3,) float32, scale (float) and r2 (int, squared disc
    radius in the set's units).  The parent frame is (frame_min float32 (3,), frame_scale).
    dirs: axis directions.  Returns dict(key, nrm, rgb, src) like sample_visible().
    """
    lib = _load()
    keys = [np.ascontiguousarray(st["key"], dtype=np.uint64) for st in sets]
    n = [len(k) for k in keys]
    ofs = np.concatenate([[0], np.cumsum(n)]).astype(np.uint64)
    skey = np.ascontiguousarray(np.concatenate(keys) if keys else np.zeros(0, np.uint64), dtype=np.uint64)
    snrm = np.ascontiguousarray(np.concatenate([np.asarray(st["nrm"], np.int16).reshape(-1, 3) for st in sets])
                                if sets else np.zeros((0, 3), np.int16), dtype=np.int16)
    have_rgb = any(st.get("rgb") is not None for st in sets)
    srgb = None
    if have_rgb:
        srgb = np.ascontiguousarray(np.concatenate([
            np.asarray(st["rgb"], np.uint8).reshape(-1, 3) if st.get("rgb") is not None
            else np.zeros((len(k), 3), np.uint8) for st, k in zip(sets, keys)]), dtype=np.uint8)
    bmin = np.ascontiguousarray(np.array([st["bbox_min"] for st in sets], np.float32).reshape(-1))
    scale = np.ascontiguousarray([float(st["scale"]) for st in sets], dtype=np.float64)
    r2 = np.ascontiguousarray([int(st["r2"]) for st in sets], dtype=np.int64)
    fmin = np.ascontiguousarray(frame_min, dtype=np.float32)
    dd = np.ascontiguousarray(dirs, dtype=np.int8).reshape(-1, 3)
    args = (len(skey), _p(skey), _p(snrm), None if srgb is None else _p(srgb), len(sets), _p(ofs), _p(bmin),
            _p(scale), _p(r2), _p(fmin), float(frame_scale), _p(dd), dd.shape[0], res)
    cnt = lib.or_sample_splats(*args, None, None, None, None, 0)
    if cnt < 0:
        raise ValueError(f"or_sample_splats failed ({cnt})")
    key = np.zeros(cnt, np.uint64)
    nrm = np.zeros((cnt, 3), np.int16)
    col = np.zeros((cnt, 3), np.uint8)
    src = np.zeros(cnt, np.uint32)
    c2 = lib.or_sample_splats(*args, _p(key), _p(nrm), _p(col), _p(src), cnt)
    assert c2 == cnt
    return dict(key=key, nrm=nrm, rgb=col, src=src)


def render_splats(sets, frame_min, frame_scale: float, d, res: int) -> np.ndarray:
    """Headless image of discs for one axis direction (the depth pass of sample_splats):
    (res, res) u64 of depth << 32 | global splat index, all ones where no disc lands."""
    lib = _load()
    keys = [np.ascontiguousarray(st["key"], dtype=np.uint64) for st in sets]
    ofs = np.concatenate([[0], np.cumsum([len(k) for k in keys])]).astype(np.uint64)
    skey = np.ascontiguousarray(np.concatenate(keys) if keys else np.zeros(0, np.uint64), dtype=np.uint64)
    snrm = np.ascontiguousarray(np.concatenate([np.asarray(st["nrm"], np.int16).reshape(-1, 3) for st in sets])
                                if sets else np.zeros((0, 3), np.int16), dtype=np.int16)
    bmin = np.ascontiguousarray(np.array([st["bbox_min"] for st in sets], np.float32).reshape(-1))
    scale = np.ascontiguousarray([float(st["scale"]) for st in sets], dtype=np.float64)
    r2 = np.ascontiguousarray([int(st["r2"]) for st in sets], dtype=np.int64)
    fmin = np.ascontiguousarray(frame_min, dtype=np.float32)
    dd = np.ascontiguousarray(d, dtype=np.int8).reshape(3)
    depth = np.zeros((res, res), np.uint64)
    if lib.or_render_splats(len(skey), _p(skey), _p(snrm), len(sets), _p(ofs), _p(bmin), _p(scale), _p(r2), _p(fmin),
                            float(frame_scale), _p(dd), res, _p(depth)) != 0:
        raise ValueError("or_render_splats: bad arguments")
    return depth


def parent_frame(mins, scales):
    """Frame of a parent node (Sec. 3.4): (min float32 (3,), scale) holding every child's
    quantisation cube [m_c, m_c + Q/s_c]; the largest extent maps onto 2^21 - 1."""
    mn = np.ascontiguousarray(np.asarray(mins, np.float32).reshape(-1, 3))
    sc = np.ascontiguousarray(np.asarray(scales, np.float64).reshape(-1))
    if mn.shape[0] != sc.shape[0]:
        raise ValueError("one bbox minimum per child scale")
    fmin = np.zeros(3, np.float32)
    fs = np.zeros(1, np.float64)
    if _load().or_parent_frame(_p(mn), _p(sc), mn.shape[0], _p(fmin), _p(fs)) != 0:
        raise ValueError("no children, or a non-positive scale")
    return fmin, float(fs[0])


def child_target_r2(child_scale: float, parent_scale: float, parent_res: int) -> int:
    """Squared length, in child units, of one pixel step of the parent's raster: the child
    prefix a parent draws is the shortest reaching every child surfel within it (Sec. 4.1)."""
    return int(_load().or_child_target_r2(float(child_scale), float(parent_scale), int(parent_res)))


def start_index(n: int, seed: int = 0, part_id: int = 0, start: int = -1) -> int:
    """Random starting surfel of Sec. 3.2 from Philox (or the given start)."""
    out = np.zeros(1, np.uint64)
    if _load().or_start_index(n, seed & (2**64 - 1), part_id, start, _p(out)) != 0:
        raise ValueError("bad start index")
    return int(out[0])


def greedy(key: np.ndarray, start: int, max_count: int = 0, nthreads: int | None = None,
           stats: bool = False):
    """Exact greedy permutation (Sec. 3.2 goal, Sec. 3.3 reference), O(N^2).

    Returns (perm u32 (m,), rad2 i64 (m,)) and, with stats=True, also
    (visits, improved) for the algorithmic-work count.
    """
    k = np.ascontiguousarray(key, dtype=np.uint64)
    n = k.shape[0]
    m = n if max_count == 0 or max_count > n else max_count
    perm = np.zeros(m, np.uint32)
    rad2 = np.zeros(m, np.int64)
    vis = np.zeros(1, np.uint64)
    imp = np.zeros(1, np.uint64)
    if nthreads is None:
        nthreads = 1 if n < 20000 else num_threads()
    if _load().or_greedy(_p(k), n, start, max_count, _p(perm), _p(rad2), _p(vis), _p(imp), nthreads) != 0:
        raise ValueError("bad greedy arguments")
    if stats:
        return perm, rad2, int(vis[0]), int(imp[0])
    return perm, rad2


def sampled(key: np.ndarray, start: int, max_count: int = 0, seed: int = 0, part_id: int = 0,
            sample_size: int = 200, step: int = 500, rounds: bool = False):
    """The paper's randomised progressive sampling (Sec. 3.2): (perm u32, rad2 i64[, round of each pick])."""
    k = np.ascontiguousarray(key, dtype=np.uint64)
    n = k.shape[0]
    m = n if max_count == 0 or max_count > n else max_count
    perm = np.zeros(m, np.uint32)
    rad2 = np.zeros(m, np.int64)
    rnd = np.zeros(m, np.uint32)
    if _load().or_sampled(_p(k), n, start, max_count, seed & (2**64 - 1), part_id, sample_size, step,
                          _p(perm), _p(rad2), _p(rnd)) != 0:
        raise ValueError("bad sampled arguments")
    return (perm, rad2, rnd) if rounds else (perm, rad2)


def prefix_median_nn(key: np.ndarray, perm: np.ndarray, pm: int) -> int:
    """Sec. 4.1 r_m^2: lower-median squared nearest-neighbour distance inside the first pm surfels."""
    k = np.ascontiguousarray(key, dtype=np.uint64)
    p = np.ascontiguousarray(perm, dtype=np.uint32)
    return int(_load().or_prefix_median_nn(_p(k), _p(p), pm))


def prefix_for_radius(rad2: np.ndarray, r2: int) -> int:
    """Sec. 4.1: shortest prefix whose reach sqrt(rad2[p]) is at most r (m if none)."""
    r = np.ascontiguousarray(rad2, dtype=np.int64)
    return int(_load().or_prefix_for_radius(_p(r), r.shape[0], r2))


def radius(rad2: np.ndarray, scale: float) -> np.ndarray:
    """Per-prefix splat radius sqrt(rad2)/S (r-net radius of Sec. 4.1) as float32."""
    r = np.ascontiguousarray(rad2, dtype=np.int64)
    out = np.zeros(r.shape[0], np.float32)
    _load().or_radius(_p(r), r.shape[0], scale, _p(out))
    return out


def num_threads() -> int:
    return int(_load().or_num_threads())


def unpack(key: np.ndarray) -> np.ndarray:
    """(N,3) int64 coordinates of packed keys (x<<42 | y<<21 | z)."""
    k = np.asarray(key, dtype=np.uint64)
    m = np.uint64(0x1FFFFF)
    return np.stack([(k >> np.uint64(42)) & m, (k >> np.uint64(21)) & m, k & m], -1).astype(np.int64)


def pack(p: np.ndarray) -> np.ndarray:
    p = np.asarray(p, dtype=np.uint64)
    return (p[..., 0] << np.uint64(42)) | (p[..., 1] << np.uint64(21)) | p[..., 2]
