"""Seeded synthetic scene parts: the inputs both the CUDA path and the CPU oracle consume.

This module only builds triangle meshes (float32 vertices, uint32 index triples,
per-face RGB8) and per-part parameters. It holds none of the method's arithmetic
(no quantisation, rasterisation, dedup or ordering), so the oracle and the GPU
path can both be fed from it without sharing any step of the method.

The paper's own inputs (the Stanford bunny, the UNC power plant and the CAD
production lines of Sec. 5) are not available; these generators stand in for
them with the shapes and size distributions of the workloads:

* ``torus``      -- a procedural torus (R=1.0, r=0.3, 128x64 quads = 16,384 tris).
* ``cad_part``   -- a CAD-like part: a seeded union of axis-aligned boxes and
                    32-segment cylinders in the unit cube (log-uniform sizes),
                    about 192k triangles with per-face RGB8 colours.
* ``batch_parts``-- thousands of randomly shaped and rotated tori whose surfel
                    counts follow a lognormal distribution (batched ordering).
* ``request_trace`` -- Poisson arrivals of ordering requests with lognormal sizes.

All randomness comes from numpy's counter-based Philox bit generator keyed by the
caller's seed, so every mesh is reproducible on any host.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Mesh", "torus", "cad_part", "cube", "quad_grid", "AXIS_DIRS", "DIAG_DIRS",
    "CORNER_DIRS", "batch_parts", "request_trace", "CUBE_ROTATIONS", "rng",
]

# View directions as integer vectors with components in {-1, 0, 1}.  The paper
# renders from the eight bounding-box corners (Sec. 3.1); the torus workload uses
# the six axis directions, the CAD part adds the two main diagonals.
AXIS_DIRS = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                     dtype=np.int8)
DIAG_DIRS = np.array([[1, 1, 1], [-1, -1, -1]], dtype=np.int8)
CORNER_DIRS = np.array(list(itertools.product([-1, 1], repeat=3)), dtype=np.int8)


@dataclass
class Mesh:
    """A triangle soup: ``xyz`` float32 (V,3), ``tri`` uint32 (T,3), ``rgb`` uint8 (T,3)."""
    xyz: np.ndarray
    tri: np.ndarray
    rgb: np.ndarray | None = None

    @property
    def nverts(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def ntris(self) -> int:
        return int(self.tri.shape[0])

    def __post_init__(self):
        self.xyz = np.ascontiguousarray(self.xyz, dtype=np.float32)
        self.tri = np.ascontiguousarray(self.tri, dtype=np.uint32)
        if self.rgb is not None:
            self.rgb = np.ascontiguousarray(self.rgb, dtype=np.uint8)


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Counter-based generator for (seed, stream): independent streams per part."""
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream) & (2**64 - 1)]))


def _grid_tris(nu: int, nv: int, wrap_u: bool, wrap_v: bool, base: int = 0) -> np.ndarray:
    """Two triangles per quad of an (nu x nv) vertex lattice (optionally periodic)."""
    iu = np.arange(nu if wrap_u else nu - 1)
    iv = np.arange(nv if wrap_v else nv - 1)
    I, J = np.meshgrid(iu, iv, indexing="ij")
    I1 = (I + 1) % nu
    J1 = (J + 1) % nv
    a = I * nv + J
    b = I1 * nv + J
    c = I1 * nv + J1
    d = I * nv + J1
    t = np.stack([np.stack([a, b, c], -1), np.stack([a, c, d], -1)], axis=-2).reshape(-1, 3)
    return (t + base).astype(np.uint32)


def torus(R: float = 1.0, r: float = 0.3, nu: int = 128, nv: int = 64,
          rot: np.ndarray | None = None, centre=(0.0, 0.0, 0.0), seed: int | None = None) -> Mesh:
    """Torus with ``nu`` major x ``nv`` minor quads (2*nu*nv triangles, nu*nv vertices)."""
    th = 2.0 * np.pi * np.arange(nu) / nu
    ph = 2.0 * np.pi * np.arange(nv) / nv
    T, P = np.meshgrid(th, ph, indexing="ij")
    x = (R + r * np.cos(P)) * np.cos(T)
    y = (R + r * np.cos(P)) * np.sin(T)
    z = r * np.sin(P)
    xyz = np.stack([x, y, z], -1).reshape(-1, 3)
    if rot is not None:
        xyz = xyz @ np.asarray(rot, dtype=np.float64).T
    xyz = xyz + np.asarray(centre, dtype=np.float64)
    tri = _grid_tris(nu, nv, True, True)
    rgb = None
    if seed is not None:
        rgb = rng(seed, 1).integers(0, 256, size=(tri.shape[0], 3), dtype=np.uint8)
    return Mesh(xyz.astype(np.float32), tri, rgb)


def quad_grid(n: int, corner0, edge_u, edge_v) -> tuple[np.ndarray, np.ndarray]:
    """An (n x n)-quad planar patch: returns (vertices float64 (n+1)^2 x 3, tris)."""
    s = np.arange(n + 1) / n
    S, Tt = np.meshgrid(s, s, indexing="ij")
    c0 = np.asarray(corner0, dtype=np.float64)
    eu = np.asarray(edge_u, dtype=np.float64)
    ev = np.asarray(edge_v, dtype=np.float64)
    v = c0 + S[..., None] * eu + Tt[..., None] * ev
    return v.reshape(-1, 3), _grid_tris(n + 1, n + 1, False, False)


def _box(lo, hi, n: int = 2):
    """Closed axis-aligned box, each face an (n x n)-quad grid (6*2*n*n triangles)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    d = hi - lo
    faces = [
        (lo, [0, d[1], 0], [0, 0, d[2]]),                       # x = lo
        (lo + [d[0], 0, 0], [0, 0, d[2]], [0, d[1], 0]),        # x = hi
        (lo, [0, 0, d[2]], [d[0], 0, 0]),                       # y = lo
        (lo + [0, d[1], 0], [d[0], 0, 0], [0, 0, d[2]]),        # y = hi
        (lo, [d[0], 0, 0], [0, d[1], 0]),                       # z = lo
        (lo + [0, 0, d[2]], [0, d[1], 0], [d[0], 0, 0]),        # z = hi
    ]
    vs, ts, base = [], [], 0
    for c0, eu, ev in faces:
        v, t = quad_grid(n, c0, eu, ev)
        vs.append(v)
        ts.append(t + base)
        base += v.shape[0]
    return np.concatenate(vs), np.concatenate(ts)


def cube(lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), n: int = 1) -> Mesh:
    v, t = _box(lo, hi, n)
    return Mesh(v.astype(np.float32), t)


def _cylinder(centre, axis: int, radius: float, length: float, nseg: int = 32, nrings: int = 3):
    """Closed cylinder: side of ``nseg`` x (nrings-1) quads, centre-fan caps.

    With nseg=32, nrings=3: 96 side + 2 centre vertices, 128 side + 64 cap triangles.
    """
    a = 2.0 * np.pi * np.arange(nseg) / nseg
    ca, sa = np.cos(a) * radius, np.sin(a) * radius
    ax = [(axis + 1) % 3, (axis + 2) % 3]
    zs = (np.arange(nrings) / (nrings - 1) - 0.5) * length
    verts = np.zeros((nrings * nseg + 2, 3))
    for k, z in enumerate(zs):
        verts[k * nseg:(k + 1) * nseg, ax[0]] = ca
        verts[k * nseg:(k + 1) * nseg, ax[1]] = sa
        verts[k * nseg:(k + 1) * nseg, axis] = z
    verts[nrings * nseg, axis] = zs[0]
    verts[nrings * nseg + 1, axis] = zs[-1]
    verts += np.asarray(centre, np.float64)
    side = _grid_tris(nrings, nseg, False, True)
    c0, c1 = nrings * nseg, nrings * nseg + 1
    j = np.arange(nseg)
    j1 = (j + 1) % nseg
    # caps wound like the side quads, so the surface is closed and consistently oriented
    cap0 = np.stack([np.full(nseg, c0), j, j1], -1)
    top = (nrings - 1) * nseg
    cap1 = np.stack([np.full(nseg, c1), top + j1, top + j], -1)
    return verts, np.concatenate([side, cap0, cap1]).astype(np.uint32)


def _loguniform(g: np.random.Generator, lo: float, hi: float, size):
    return np.exp(g.uniform(np.log(lo), np.log(hi), size=size))


def cad_part(seed: int = 0, nboxes: int = 2000, ncyl: int = 500, size_lo: float = 0.01,
             size_hi: float = 0.3, box_div: int = 2) -> Mesh:
    """CAD-like part: a seeded union of axis-aligned boxes and 32-segment cylinders.

    Centres are uniform in the unit cube, sizes log-uniform in [size_lo, size_hi]
    per box side and per cylinder radius / length.  Box faces are split 2x2 and
    cylinders get two side bands plus centre-fan caps, so the default part has
    2000*48 + 500*192 = 192,000 triangles.  Every box face and every cylinder band
    or cap gets its own RGB8 colour.
    """
    g = rng(seed, 2)
    vs, ts, cs = [], [], []
    base = 0
    bc = g.uniform(0.0, 1.0, size=(nboxes, 3))
    bs = _loguniform(g, size_lo, size_hi, (nboxes, 3))
    bcol = g.integers(0, 256, size=(nboxes, 6, 3), dtype=np.uint8)
    fpt = 2 * box_div * box_div  # triangles per box face
    for i in range(nboxes):
        v, t = _box(bc[i] - bs[i] / 2, bc[i] + bs[i] / 2, box_div)
        vs.append(v)
        ts.append(t + base)
        cs.append(np.repeat(bcol[i], fpt, axis=0))
        base += v.shape[0]
    cc = g.uniform(0.0, 1.0, size=(ncyl, 3))
    cax = g.integers(0, 3, size=ncyl)
    crad = _loguniform(g, size_lo, size_hi, ncyl)
    clen = _loguniform(g, size_lo, size_hi, ncyl)
    ccol = g.integers(0, 256, size=(ncyl, 3, 3), dtype=np.uint8)
    for i in range(ncyl):
        v, t = _cylinder(cc[i], int(cax[i]), float(crad[i]), float(clen[i]))
        vs.append(v)
        ts.append(t + base)
        nside = t.shape[0] - 64
        cs.append(np.concatenate([np.repeat(ccol[i, 0:1], nside, 0),
                                  np.repeat(ccol[i, 1:2], 32, 0),
                                  np.repeat(ccol[i, 2:3], 32, 0)]))
        base += v.shape[0]
    if not vs:
        return Mesh(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32), np.zeros((0, 3), np.uint8))
    return Mesh(np.concatenate(vs).astype(np.float32), np.concatenate(ts), np.concatenate(cs))


def _cube_rotations() -> np.ndarray:
    """The 24 proper rotations of the cube: signed permutation matrices, det = +1."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            m = np.zeros((3, 3), np.int64)
            for r, c in enumerate(perm):
                m[r, c] = signs[r]
            if round(np.linalg.det(m)) == 1:
                out.append(m)
    return np.array(out)


CUBE_ROTATIONS = _cube_rotations()


@dataclass
class PartSpec:
    """One part of a batch: a torus shape plus its raster resolution and seed."""
    R: float
    r: float
    nu: int
    nv: int
    rot: int
    res: int
    n_target: int
    seed: int

    def mesh(self) -> Mesh:
        return torus(self.R, self.r, self.nu, self.nv, CUBE_ROTATIONS[self.rot], seed=self.seed)


def batch_parts(nparts: int = 4096, seed: int = 0, n_median: float = 20_000.0, n_sigma: float = 1.0,
                n_lo: int = 1_000, n_hi: int = 500_000, t_median: float = 10_000.0,
                t_lo: int = 2_000, t_hi: int = 50_000, surfels_per_px2: float = 2.0,
                res_lo: int = 16, res_hi: int = 1024) -> list[PartSpec]:
    """Batched-ordering workload: tori with lognormal triangle and surfel counts.

    Per part: R ~ U[0.5, 1], r/R ~ U[0.1, 0.45], one of the 24 cube rotations,
    triangle count lognormal clamped to [t_lo, t_hi], and a target surfel count
    lognormal(median n_median, sigma n_sigma) clamped to [n_lo, n_hi].  Six axis
    views of a torus cover about ``surfels_per_px2`` * res^2 pixels, so the raster
    resolution is chosen as sqrt(target / surfels_per_px2), rounded to a multiple of
    8 and clamped to [res_lo, res_hi]; the actual count is whatever the sampler emits.
    """
    g = rng(seed, 3)
    out = []
    Rs = g.uniform(0.5, 1.0, nparts)
    rr = g.uniform(0.1, 0.45, nparts)
    rots = g.integers(0, 24, nparts)
    tcount = np.clip(np.exp(g.normal(np.log(t_median), 0.8, nparts)), t_lo, t_hi)
    ncount = np.clip(np.exp(g.normal(np.log(n_median), n_sigma, nparts)), n_lo, n_hi)
    for i in range(nparts):
        aspect = 1.0 / rr[i]
        nv = max(6, int(round(math.sqrt(tcount[i] / 2.0 / aspect))))
        nu = max(8, int(round(tcount[i] / 2.0 / nv)))
        res = int(round(math.sqrt(ncount[i] / surfels_per_px2) / 8.0)) * 8
        res = int(min(max(res, res_lo), res_hi))
        out.append(PartSpec(float(Rs[i]), float(Rs[i] * rr[i]), nu, nv, int(rots[i]), res,
                            int(ncount[i]), seed * 1_000_003 + i))
    return out


@dataclass
class Request:
    arrival_s: float
    part: Mesh
    res: int
    seed: int


def request_trace(nreq: int, rate_hz: float, seed: int = 0, n_median: float = 30_000.0,
                  n_lo: int = 1_000, n_hi: int = 1_000_000, boxes_per_kpx: float = 0.0):
    """Serving workload: Poisson arrival times plus lognormal request sizes.

    Returns (arrival times in seconds, per-request target surfel counts, seeds).
    Meshes are built lazily by the caller (``cad_part`` with a box count scaled
    to the target), so a long trace does not hold every mesh at once.
    """
    g = rng(seed, 4)
    gaps = g.exponential(1.0 / rate_hz, nreq)
    t = np.cumsum(gaps) - gaps[0]
    n = np.clip(np.exp(g.normal(np.log(n_median), 1.0, nreq)), n_lo, n_hi).astype(np.int64)
    seeds = g.integers(0, 2**31, nreq)
    return t, n, seeds


# ---------------------------------------------------------------------------
# Scene-scale workload: production lines of CAD-like parts, regenerated from a seed.
#
# The same parts are produced on the device by bs_scene_generate (libbs) and here on
# the host (for the oracle's checks); both follow this float32 recipe exactly:
#   * random words: w(part, prim, k) = Philox4x32-10(ctr = {part_lo, part_hi, prim, k},
#     key = {seed_lo, seed_hi}); uniform u(x) = float32(x >> 8) * 2^-24 (exact);
#   * sizes: SIZE_TABLE[x >> 22], 1024 log-uniform values in [0.01, 0.3] (host-made);
#   * box b: centre (u(w0[0]), u(w0[1]), u(w0[2])), sizes SIZE_TABLE[w1[a] >> 22],
#     h = s * 0.5, lo = c - h, mid = lo + h, hi = c + h; 6 faces of 2x2 quads
#     (9 vertices, 8 triangles each), one RGB8 per face from w2, w3 bytes;
#   * cylinder: axis w0[0] % 3, centre (u(w0[1]), u(w0[2]), u(w0[3])), radius
#     SIZE_TABLE[w1[0] >> 22], length SIZE_TABLE[w1[1] >> 22], ring point j =
#     (COS32[j] * r + c, SIN32[j] * r + c) across the axis, levels c - L*0.5, c, c + L*0.5;
#     3 rings of 32 + 2 cap centres, 128 side + 64 cap triangles, colours from w2;
#   * placement: part p of line l at slot i adds (i * SCENE_DX, l * SCENE_DY, 0).
# All additions and multiplications are single float32 operations in this order.
# ---------------------------------------------------------------------------
SIZE_TABLE = np.exp(np.log(0.01) + (np.arange(1024) + 0.5) / 1024 * (np.log(0.3) - np.log(0.01))).astype(np.float32)
COS32 = np.cos(2.0 * np.pi * np.arange(32) / 32).astype(np.float32)
SIN32 = np.sin(2.0 * np.pi * np.arange(32) / 32).astype(np.float32)
SCENE_DX = np.float32(1.25)
SCENE_DY = np.float32(1.75)
BOX_VERTS, BOX_TRIS, CYL_VERTS, CYL_TRIS = 54, 48, 98, 192


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 (Salmon et al., SC'11) on numpy uint32 arrays (broadcast)."""
    M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
    W0, W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
    x = [np.asarray(c, dtype=np.uint32).copy() for c in (c0, c1, c2, c3)]
    x = np.broadcast_arrays(*x)
    x = [a.copy() for a in x]
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = M0 * x[0].astype(np.uint64)
            p1 = M1 * x[2].astype(np.uint64)
            y0 = (p1 >> np.uint64(32)).astype(np.uint32) ^ x[1] ^ k0
            y1 = p1.astype(np.uint32)
            y2 = (p0 >> np.uint64(32)).astype(np.uint32) ^ x[3] ^ k1
            y3 = p0.astype(np.uint32)
            x = [y0, y1, y2, y3]
            k0 = np.uint32(k0 + W0)
            k1 = np.uint32(k1 + W1)
    return x


def _u(x):
    return (x >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)


def scene_part(seed: int, part: int, line: int, slot: int, nboxes: int = 200, ncyl: int = 50) -> Mesh:
    """One scene part (float32 recipe above), placed at its line and slot."""
    f = np.float32
    s_lo, s_hi = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    p_lo, p_hi = part & 0xFFFFFFFF, (part >> 32) & 0xFFFFFFFF
    off = np.array([f(slot) * SCENE_DX, f(line) * SCENE_DY, f(0.0)], np.float32)
    vs, ts, cs = [], [], []
    base = 0
    prim = np.arange(nboxes, dtype=np.uint32)
    w0 = philox4x32_10(p_lo, p_hi, prim, 0, s_lo, s_hi)
    w1 = philox4x32_10(p_lo, p_hi, prim, 1, s_lo, s_hi)
    w2 = philox4x32_10(p_lo, p_hi, prim, 2, s_lo, s_hi)
    w3 = philox4x32_10(p_lo, p_hi, prim, 3, s_lo, s_hi)
    c = np.stack([_u(w0[0]), _u(w0[1]), _u(w0[2])], -1)
    sz = np.stack([SIZE_TABLE[w1[a] >> np.uint32(22)] for a in range(3)], -1)
    h = sz * f(0.5)
    lo = c - h
    mid = lo + h
    hi = c + h
    grid = np.stack([lo, mid, hi], 1)  # (nb, 3 levels, 3 axes)
    colbytes = np.stack([w2[0], w2[1], w2[2], w2[3], w3[0], w3[1]], -1)  # 6 words -> 6 faces
    # faces: (axis fixed, level, axes varying u, v) in the order of workloads._box
    faces = [(0, 0, 1, 2), (0, 2, 2, 1), (1, 0, 2, 0), (1, 2, 0, 2), (2, 0, 0, 1), (2, 2, 1, 0)]
    tri9 = _grid_tris(3, 3, False, False)
    for b in range(nboxes):
        for fi, (ax, lev, ua, va) in enumerate(faces):
            v = np.zeros((3, 3, 3), np.float32)
            for i in range(3):
                for j in range(3):
                    v[i, j, ax] = grid[b, lev, ax]
                    v[i, j, ua] = grid[b, i, ua]
                    v[i, j, va] = grid[b, j, va]
            vs.append(v.reshape(-1, 3) + off)
            ts.append(tri9 + base)
            base += 9
            cw = int(colbytes[b, fi])
            cs.append(np.tile(np.array([cw & 255, (cw >> 8) & 255, (cw >> 16) & 255], np.uint8), (8, 1)))
    prim = np.arange(nboxes, nboxes + ncyl, dtype=np.uint32)
    w0 = philox4x32_10(p_lo, p_hi, prim, 0, s_lo, s_hi)
    w1 = philox4x32_10(p_lo, p_hi, prim, 1, s_lo, s_hi)
    w2 = philox4x32_10(p_lo, p_hi, prim, 2, s_lo, s_hi)
    for q in range(ncyl):
        axis = int(w0[0][q] % 3)
        cc = np.array([_u(w0[1][q]), _u(w0[2][q]), _u(w0[3][q])], np.float32)
        r = SIZE_TABLE[w1[0][q] >> 22]
        L = SIZE_TABLE[w1[1][q] >> 22]
        a1, a2 = (axis + 1) % 3, (axis + 2) % 3
        hl = L * f(0.5)
        levels = [cc[axis] - hl, cc[axis], cc[axis] + hl]
        v = np.zeros((98, 3), np.float32)
        for k, z in enumerate(levels):
            v[k * 32:(k + 1) * 32, a1] = COS32 * r + cc[a1]
            v[k * 32:(k + 1) * 32, a2] = SIN32 * r + cc[a2]
            v[k * 32:(k + 1) * 32, axis] = z
        v[96, a1], v[96, a2], v[96, axis] = cc[a1], cc[a2], levels[0]
        v[97, a1], v[97, a2], v[97, axis] = cc[a1], cc[a2], levels[2]
        side = _grid_tris(3, 32, False, True)
        j = np.arange(32)
        j1 = (j + 1) % 32
        cap0 = np.stack([np.full(32, 96), j, j1], -1)
        cap1 = np.stack([np.full(32, 97), 64 + j1, 64 + j], -1)
        vs.append(v + off)
        ts.append(np.concatenate([side, cap0, cap1]).astype(np.uint32) + base)
        base += 98
        cw = [int(w2[t][q]) for t in range(3)]
        cs.append(np.concatenate([np.tile(np.array([cw[0] & 255, (cw[0] >> 8) & 255, (cw[0] >> 16) & 255], np.uint8), (128, 1)),
                                  np.tile(np.array([cw[1] & 255, (cw[1] >> 8) & 255, (cw[1] >> 16) & 255], np.uint8), (32, 1)),
                                  np.tile(np.array([cw[2] & 255, (cw[2] >> 8) & 255, (cw[2] >> 16) & 255], np.uint8), (32, 1))]))
    return Mesh(np.concatenate(vs).astype(np.float32), np.concatenate(ts), np.concatenate(cs))


@dataclass
class SceneNode:
    """A node of the scene hierarchy: a range of consecutive parts of one line."""
    line: int
    first: int      # first slot in the line
    count: int      # number of parts
    level: int      # 0 = one part, 1 = a group of parts, 2 = a whole line

    def parts(self, per_line: int):
        return [(self.line * per_line + s, self.line, s) for s in range(self.first, self.first + self.count)]


def scene_nodes(lines: int = 20, per_line: int = 2500, group: int = 50) -> list[SceneNode]:
    """Hierarchy of the scene: every part (level 0), groups of `group` consecutive parts
    (level 1) and whole lines (level 2).  Every node holds more than 10k triangles, the
    paper's threshold for giving a subtree its own approximation (Sec. 3.4)."""
    nodes = []
    for l in range(lines):
        for s in range(per_line):
            nodes.append(SceneNode(l, s, 1, 0))
        for s in range(0, per_line, group):
            nodes.append(SceneNode(l, s, min(group, per_line - s), 1))
        nodes.append(SceneNode(l, 0, per_line, 2))
    return nodes


def scene_node_mesh(seed: int, node: SceneNode, per_line: int, nboxes: int = 200, ncyl: int = 50) -> Mesh:
    """Host mesh of a node: its parts concatenated in slot order."""
    ms = [scene_part(seed, p, l, s, nboxes, ncyl) for p, l, s in node.parts(per_line)]
    vofs = np.cumsum([0] + [m.nverts for m in ms])
    return Mesh(np.concatenate([m.xyz for m in ms]), np.concatenate([m.tri + np.uint32(o) for m, o in zip(ms, vofs)]),
                np.concatenate([m.rgb for m in ms]))
