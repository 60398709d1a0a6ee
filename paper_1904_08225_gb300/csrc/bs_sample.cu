// bs_sample.cu -- visible-surface sampling (Sec. 3.1): quantise each mesh, rasterise it
// orthographically from several integer directions with an integer rasteriser,
// emit one surfel per covered pixel, merge identical positions and sort each part's
// surfels into ascending Morton order.  Any number of parts go through one set of
// launches; a single part is the one-part case.
//
// Pipeline (all on the caller's stream):
//   k_bbox -> k_scale -> k_quantise              node-local 21-bit integer positions (8192-vertex chunks)
//   k_setup   (dir x triangle, all parts)        snapped screen coords, winding, area
//   k_raster  (warp per dir x triangle)          64-bit atomicMin(depth << 32 | tri)
//   k_cover_count -> scan -> k_resolve           covered pixels in (part, emission) order
//   radix sort (Morton code), then (part)        stable LSD, 8-bit digits
//   k_unique_count -> scan -> k_segments -> k_unique_write
//                                                keep the first row of each (part, position)
//
// Arithmetic: integers throughout, except the quantiser (IEEE double subtract and
// multiply, written with explicit round-to-nearest intrinsics so nothing is fused)
// and the unit normal (IEEE double multiply/add/sqrt/divide, same intrinsics).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <vector>

#include "bs_internal.cuh"

namespace bs {

// ---------------------------------------------------------------------------
// View frames: camera on the +d side looking along -d.  k = first axis with the
// smallest |d_k|; u = d x e_k, v = d x u; depth w = -(d . q).  The projection of
// the quantisation cube onto u (resp. v) is mapped onto res pixels; vertices are
// snapped to 1/256 pixel with round-half-up; pixel p has its centre at 256p+128.
// ---------------------------------------------------------------------------
struct View {
    int32_t u[3], v[3], d[3];
    int64_t ulo, vlo, U1, V1, wbias;
    uint64_t mU, mV;  // floor((2^64 - 1) / (2 U1)) and likewise for V1: exact division in project
};

struct Views {
    View v[BS_MAX_DIRS];
    int ndirs;
};

static void make_frame(const bs_dir &dir, View &V) {
    const int64_t d[3] = {dir.x, dir.y, dir.z};
    int k = 0;
    for (int a = 1; a < 3; ++a)
        if ((d[a] < 0 ? -d[a] : d[a]) < (d[k] < 0 ? -d[k] : d[k])) k = a;
    int64_t e[3] = {0, 0, 0};
    e[k] = 1;
    const int64_t u[3] = {d[1] * e[2] - d[2] * e[1], d[2] * e[0] - d[0] * e[2], d[0] * e[1] - d[1] * e[0]};
    const int64_t v[3] = {d[1] * u[2] - d[2] * u[1], d[2] * u[0] - d[0] * u[2], d[0] * u[1] - d[1] * u[0]};
    int64_t ulo = 0, uspan = 0, vlo = 0, vspan = 0, wb = 0;
    for (int a = 0; a < 3; ++a) {
        V.u[a] = (int32_t)u[a];
        V.v[a] = (int32_t)v[a];
        V.d[a] = (int32_t)d[a];
        if (u[a] < 0) ulo += u[a] * QMAX;
        uspan += (u[a] < 0 ? -u[a] : u[a]) * QMAX;
        if (v[a] < 0) vlo += v[a] * QMAX;
        vspan += (v[a] < 0 ? -v[a] : v[a]) * QMAX;
        if (d[a] > 0) wb += d[a] * QMAX;
    }
    V.ulo = ulo;
    V.vlo = vlo;
    V.U1 = uspan + 1;
    V.V1 = vspan + 1;
    V.wbias = wb;
    V.mU = ~0ull / (uint64_t)(2 * V.U1);
    V.mV = ~0ull / (uint64_t)(2 * V.V1);
}

// ---------------------------------------------------------------------------
// Part table and per-part state
// ---------------------------------------------------------------------------
struct SPart {
    const float *xyz;
    const uint32_t *tri;
    const uint8_t *rgb;
    uint64_t *okey;
    int16_t *onrm;
    uint8_t *orgb;
    uint32_t *osrc;
    uint64_t cap;
    uint64_t vofs;  // first vertex of this part in the packed q array
    uint64_t tofs;  // first triangle of this part in the packed triangle numbering
    uint64_t pofs;  // first pixel (all directions) of this part in the packed depth buffer
    uint32_t nverts, ntris;
    int32_t res;
    uint32_t pad;
};

struct SState {
    uint32_t mn_ord[3], mx_ord[3];  // order-preserving encodings of the float bounds
    uint32_t nonfinite, invalid, badtri, pad0;
    float mn[3];
    float pad1;
    double scale;
    uint64_t first_out, end_out;  // [first_out, end_out): this part's surfels in the packed output numbering
};

// index of the part whose range [ofs[p], ofs[p+1]) holds x (ofs ascending, ofs[0] = 0)
__device__ __forceinline__ int find_part(const uint64_t *__restrict__ ofs, int nparts, uint64_t x) {
    int lo = 0, hi = nparts - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ofs[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Quantisation: bbox over float32 vertices, isotropic scale S = (2^21-1)/E.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Vertices are processed in chunks of VCHUNK per block, so one large part uses the whole
// GPU; chunk c of the call belongs to part find_part(cofs, nparts, c).
constexpr uint32_t VCHUNK = 8192;

__global__ void k_bbox_init(SState *__restrict__ st, int nparts) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nparts) return;
    SState &S = st[p];
    for (int a = 0; a < 3; ++a) { S.mn_ord[a] = 0xffffffffu; S.mx_ord[a] = 0u; }
    S.nonfinite = 0;
    S.badtri = 0;
    S.first_out = 0;
    S.end_out = 0;
}

// per chunk: min / max of the order-preserving encodings, count of non-finite coordinates
__global__ void __launch_bounds__(256) k_bbox(const SPart *__restrict__ parts, const uint64_t *__restrict__ cofs,
                                              int nparts, SState *__restrict__ st) {
    const int p = find_part(cofs, nparts, blockIdx.x);
    const SPart P = parts[p];
    const uint64_t v0 = (blockIdx.x - cofs[p]) * (uint64_t)VCHUNK;
    const uint64_t v1 = min((uint64_t)P.nverts, v0 + VCHUNK);
    uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u}, bad = 0;
    for (uint64_t e = 3 * v0 + threadIdx.x; e < 3 * v1; e += blockDim.x) {
        const float f = P.xyz[e];
        const int a = (int)(e % 3);
        if (!isfinite(f)) {
            ++bad;
        } else {
            const uint32_t o = f2ord(f);
            // branch-free per-axis update keeps the loads independent
            mn[0] = a == 0 ? min(mn[0], o) : mn[0];
            mn[1] = a == 1 ? min(mn[1], o) : mn[1];
            mn[2] = a == 2 ? min(mn[2], o) : mn[2];
            mx[0] = a == 0 ? max(mx[0], o) : mx[0];
            mx[1] = a == 1 ? max(mx[1], o) : mx[1];
            mx[2] = a == 2 ? max(mx[2], o) : mx[2];
        }
    }
    __shared__ uint32_t red[8][7];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(0xffffffffu, mn[a]);
        mx[a] = __reduce_max_sync(0xffffffffu, mx[a]);
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) { red[warp][a] = mn[a]; red[warp][3 + a] = mx[a]; }
        red[warp][6] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        uint32_t v = red[0][threadIdx.x];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            const uint32_t x = red[w][threadIdx.x];
            v = threadIdx.x < 3 ? min(v, x) : (threadIdx.x < 6 ? max(v, x) : v + x);
        }
        SState &S = st[p];
        if (threadIdx.x < 3) atomicMin(&S.mn_ord[threadIdx.x], v);
        else if (threadIdx.x < 6) atomicMax(&S.mx_ord[threadIdx.x - 3], v);
        else if (v) atomicAdd(&S.nonfinite, v);
    }
}

// per part: cube extent E = max side (double), scale S = (2^21 - 1) / E
__global__ void k_scale(const SPart *__restrict__ parts, SState *__restrict__ st, int nparts) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nparts) return;
    SState &S = st[p];
    double E = 0.0;
    for (int a = 0; a < 3; ++a) {
        const float lo = ord2f(S.mn_ord[a]);
        const float hi = ord2f(S.mx_ord[a]);
        const double e = __dsub_rn((double)hi, (double)lo);
        if (e > E) E = e;
        S.mn[a] = __fadd_rn(lo, 0.0f);  // report -0.0 as +0.0
    }
    S.invalid = (S.nonfinite != 0u || parts[p].nverts == 0 || !(E > 0.0)) ? 1u : 0u;
    S.scale = S.invalid ? 0.0 : __ddiv_rn(2097151.0, E);
}

__global__ void __launch_bounds__(256) k_quantise(const SPart *__restrict__ parts, const uint64_t *__restrict__ cofs,
                                                  int nparts, const SState *__restrict__ st, int32_t *__restrict__ q) {
    const int p = find_part(cofs, nparts, blockIdx.x);
    const SPart P = parts[p];
    const SState &S = st[p];
    if (S.invalid) return;
    const double sc = S.scale;
    const uint64_t v0 = (blockIdx.x - cofs[p]) * (uint64_t)VCHUNK;
    const uint64_t v1 = min((uint64_t)P.nverts, v0 + VCHUNK);
    for (uint64_t i = 3 * v0 + threadIdx.x; i < 3 * v1; i += blockDim.x) {
        const int a = (int)(i % 3);
        const double t = __dmul_rn(__dsub_rn((double)P.xyz[i], (double)S.mn[a]), sc);
        int64_t v = (int64_t)floor(t);
        v = v < 0 ? 0 : (v > QMAX ? QMAX : v);
        q[3ull * P.vofs + i] = (int32_t)v;
    }
}

// ---------------------------------------------------------------------------
// Triangle setup per (direction, triangle): snapped integer screen coordinates,
// biased depth, winding normalised so that area2 > 0 (vertex order kept in ord).
// ---------------------------------------------------------------------------
struct TriSetup {
    int32_t x[3], y[3];
    uint32_t w[3];
    uint32_t ord;   // bits 0-1: input vertex of slot 0, 2-3 slot 1, 4-5 slot 2; bits 8-23: part;
                    // 0xffffffff = skip
    int64_t area2;
    uint64_t rcp;   // floor((2^64 - 1) / area2): exact division by area2, see div_area
};

__device__ __forceinline__ int setup_part(const TriSetup &s) { return (int)((s.ord >> 8) & 0xffffu); }

// floor(num / d) for d >= 1 from m = floor((2^64 - 1) / d) (division by an invariant
// integer, Granlund and Montgomery, PLDI 1994): the high word of num * m is at most two
// below the quotient, so two conditional corrections make it exact.
__device__ __forceinline__ uint64_t div_area(uint64_t num, uint64_t d, uint64_t m) {
    uint64_t q = __umul64hi(num, m);
    uint64_t r = num - q * d;
    if (r >= d) { ++q; r -= d; }
    if (r >= d) { ++q; }
    return q;
}

__device__ __forceinline__ void project(const View &V, int res, const int32_t *q, int32_t &X, int32_t &Y,
                                        uint32_t &W) {
    const int64_t x = q[0], y = q[1], z = q[2];
    const int64_t uq = V.u[0] * x + V.u[1] * y + V.u[2] * z;
    const int64_t vq = V.v[0] * x + V.v[1] * y + V.v[2] * z;
    const int64_t dq = V.d[0] * x + V.d[1] * y + V.d[2] * z;
    // the numerators are non-negative (ulo and vlo are the smallest projections of the
    // quantised cube), so the quotients are floors: div_area with the view's reciprocals
    X = (int32_t)div_area((uint64_t)((uq - V.ulo) * res * 512 + V.U1), (uint64_t)(2 * V.U1), V.mU);
    Y = (int32_t)div_area((uint64_t)((vq - V.vlo) * res * 512 + V.V1), (uint64_t)(2 * V.V1), V.mV);
    W = (uint32_t)(-dq + V.wbias);
}

// The triangle normal n: integer cross product of its quantised edges, input vertex order.
__device__ __forceinline__ void tri_normal(const int32_t *a, const int32_t *b, const int32_t *c, int64_t n[3]) {
    int64_t e1[3], e2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e1[k] = (int64_t)b[k] - a[k];
        e2[k] = (int64_t)c[k] - a[k];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
}

// n as snorm16 components round(32767 n_a / |n|), round half to even, in double
// precision (0 for a degenerate triangle).  Turning n toward a camera negates every
// component exactly (the rounding is symmetric), so this is computed once per triangle.
__device__ __noinline__ uint64_t snorm_pack(const int64_t n[3]) {
    const double f0 = (double)n[0], f1 = (double)n[1], f2 = (double)n[2];
    double ss = __dadd_rn(__dmul_rn(f0, f0), __dmul_rn(f1, f1));
    ss = __dadd_rn(ss, __dmul_rn(f2, f2));
    uint64_t np = 0;
    if (ss != 0.0) {
        const double len = __dsqrt_rn(ss);
        const double c[3] = {f0, f1, f2};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int v = __double2int_rn(__ddiv_rn(__dmul_rn(32767.0, c[a]), len));
            np |= (uint64_t)(uint16_t)(int16_t)v << (16 * a);
        }
    }
    return np;
}

// packed snorm16 components negated
__device__ __forceinline__ uint64_t snorm_negate(uint64_t np) {
    uint64_t r = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) r |= (uint64_t)(uint16_t)(int16_t)(-(int)(int16_t)(uint16_t)(np >> (16 * a))) << (16 * a);
    return r;
}

// grid: (triangles of all parts, directions); setup[dir * T + global triangle].  Bit 24
// of a kept setup's ord: the triangle's normal points away from this view's camera (the
// surfel takes the negated normal); the first direction writes each triangle's snorm16
// normal to tnrm.
__global__ void k_setup(const SPart *__restrict__ parts, const uint64_t *__restrict__ tofs, int nparts,
                        uint64_t T, const int32_t *__restrict__ q, SState *__restrict__ st, const Views views,
                        TriSetup *__restrict__ out, uint64_t *__restrict__ tnrm) {
    const int dir = blockIdx.y;
    const View &V = views.v[dir];
    for (uint64_t tg = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; tg < T; tg += (uint64_t)gridDim.x * blockDim.x) {
        const int p = find_part(tofs, nparts, tg);
        const SPart &P = parts[p];
        const uint32_t t = (uint32_t)(tg - P.tofs);
        TriSetup s;
        const uint32_t v0 = P.tri[3ull * t], v1 = P.tri[3ull * t + 1], v2 = P.tri[3ull * t + 2];
        if (st[p].invalid || v0 >= P.nverts || v1 >= P.nverts || v2 >= P.nverts) {
            s.ord = 0xffffffffu;
            s.area2 = 0;
            s.rcp = 0;
            out[(uint64_t)dir * T + tg] = s;
            if (!st[p].invalid && dir == 0) atomicAdd(&st[p].badtri, 1u);
            continue;
        }
        const int32_t *qp = q + 3ull * P.vofs;
        int32_t X[3], Y[3];
        uint32_t W[3];
        project(V, P.res, qp + 3ull * v0, X[0], Y[0], W[0]);
        project(V, P.res, qp + 3ull * v1, X[1], Y[1], W[1]);
        project(V, P.res, qp + 3ull * v2, X[2], Y[2], W[2]);
        int64_t a2 = (int64_t)(X[1] - X[0]) * (Y[2] - Y[0]) - (int64_t)(Y[1] - Y[0]) * (X[2] - X[0]);
        int o1 = 1, o2 = 2;
        if (a2 < 0) { o1 = 2; o2 = 1; a2 = -a2; }
        s.x[0] = X[0]; s.y[0] = Y[0]; s.w[0] = W[0];
        s.x[1] = X[o1]; s.y[1] = Y[o1]; s.w[1] = W[o1];
        s.x[2] = X[o2]; s.y[2] = Y[o2]; s.w[2] = W[o2];
        int64_t n[3];
        tri_normal(qp + 3ull * v0, qp + 3ull * v1, qp + 3ull * v2, n);
        const bool flip = n[0] * V.d[0] + n[1] * V.d[1] + n[2] * V.d[2] < 0;
        if (dir == 0) tnrm[tg] = snorm_pack(n);
        s.ord = a2 == 0 ? 0xffffffffu
                        : (uint32_t)(0 | (o1 << 2) | (o2 << 4) | ((uint32_t)p << 8) | ((uint32_t)flip << 24));
        s.area2 = a2;
        s.rcp = a2 == 0 ? 0ull : ~0ull / (uint64_t)a2;
        out[(uint64_t)dir * T + tg] = s;
    }
}

// Coverage of pixel centre (sx, sy): an edge a->b owns centres exactly on it when
// its direction points down (dy < 0) or, horizontal, right (dx > 0) -- the same as
// sampling at p + eps*(1, eta), so shared edges and vertices are covered once.
__device__ __forceinline__ bool edge_in(int32_t ax, int32_t ay, int32_t bx, int32_t by, int32_t sx, int32_t sy,
                                        int64_t &lam) {
    lam = (int64_t)(bx - ax) * (sy - ay) - (int64_t)(by - ay) * (sx - ax);
    const int32_t dx = bx - ax, dy = by - ay;
    return lam > 0 || (lam == 0 && (dy < 0 || (dy == 0 && dx > 0)));
}

__device__ __forceinline__ bool cover(const TriSetup &s, int32_t px, int32_t py, int64_t lam[3]) {
    const int32_t sx = 256 * px + 128, sy = 256 * py + 128;
    const bool a = edge_in(s.x[1], s.y[1], s.x[2], s.y[2], sx, sy, lam[0]);
    const bool b = edge_in(s.x[2], s.y[2], s.x[0], s.y[0], sx, sy, lam[1]);
    const bool c = edge_in(s.x[0], s.y[0], s.x[1], s.y[1], sx, sy, lam[2]);
    return a && b && c;
}

__device__ __forceinline__ void pixel_span(int32_t lo, int32_t hi, int res, int32_t &p0, int32_t &p1) {
    p0 = lo <= 128 ? 0 : (lo - 128 + 255) / 256;
    p1 = hi < 128 ? -1 : (hi - 128) / 256;
    if (p1 > res - 1) p1 = res - 1;
}

// Depth pass of one (direction, triangle) over pixels [px0, px1] x [py0, py1], by `lanes`
// threads starting at pixel offset `first`.
__device__ __forceinline__ void raster_pixels(const TriSetup &s, int32_t px0, int32_t px1, int32_t py0, int32_t py1,
                                              uint32_t first, uint32_t lanes, int res, uint32_t t,
                                              unsigned long long *__restrict__ dbuf) {
    const uint32_t wdt = (uint32_t)(px1 - px0 + 1);
    const uint32_t npx = wdt * (uint32_t)(py1 - py0 + 1);
    for (uint32_t pp = first; pp < npx; pp += lanes) {
        const int32_t py = py0 + (int32_t)(pp / wdt), px = px0 + (int32_t)(pp % wdt);
        int64_t lam[3];
        if (!cover(s, px, py, lam)) continue;
        const uint64_t num = (uint64_t)lam[0] * s.w[0] + (uint64_t)lam[1] * s.w[1] + (uint64_t)lam[2] * s.w[2];
        const uint64_t z = div_area(num, (uint64_t)s.area2, s.rcp);
        atomicMin(dbuf + (uint64_t)py * res + px, (unsigned long long)((z << 32) | t));
    }
}

// A thread per (direction, triangle): triangles whose screen bbox holds at most
// RASTER_SMALL pixels are rasterised by their own thread; larger ones by the whole warp,
// one after another.
constexpr uint32_t RASTER_SMALL = 16;

__global__ void __launch_bounds__(256) k_raster(const SPart *__restrict__ parts, uint64_t T,
                                                const TriSetup *__restrict__ setup,
                                                unsigned long long *__restrict__ depth) {
    const int dir = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < T; base += stride) {
        const uint64_t tg = base + lane;
        TriSetup s;
        bool valid = false;
        int32_t px0 = 0, px1 = -1, py0 = 0, py1 = -1;
        int res = 0;
        uint32_t t = 0;
        unsigned long long *dbuf = nullptr;
        if (tg < T) {
            s = setup[(uint64_t)dir * T + tg];
            if (s.ord != 0xffffffffu) {
                const SPart &P = parts[setup_part(s)];
                res = P.res;
                t = (uint32_t)(tg - P.tofs);
                dbuf = depth + P.pofs + (uint64_t)dir * res * res;
                const int32_t xmin = min(s.x[0], min(s.x[1], s.x[2])), xmax = max(s.x[0], max(s.x[1], s.x[2]));
                const int32_t ymin = min(s.y[0], min(s.y[1], s.y[2])), ymax = max(s.y[0], max(s.y[1], s.y[2]));
                pixel_span(xmin, xmax, res, px0, px1);
                pixel_span(ymin, ymax, res, py0, py1);
                valid = px1 >= px0 && py1 >= py0;
            }
        }
        const uint32_t npx = valid ? (uint32_t)(px1 - px0 + 1) * (uint32_t)(py1 - py0 + 1) : 0u;
        if (valid && npx <= RASTER_SMALL) raster_pixels(s, px0, px1, py0, py1, 0u, 1u, res, t, dbuf);
        uint32_t big = __ballot_sync(0xffffffffu, npx > RASTER_SMALL);
        while (big) {
            const int j = __ffs(big) - 1;
            big &= big - 1;
            // the whole warp on lane j's triangle (its record reloaded: one broadcast load)
            const TriSetup sj = setup[(uint64_t)dir * T + base + j];
            const int32_t bx0 = __shfl_sync(0xffffffffu, px0, j), bx1 = __shfl_sync(0xffffffffu, px1, j);
            const int32_t by0 = __shfl_sync(0xffffffffu, py0, j), by1 = __shfl_sync(0xffffffffu, py1, j);
            const int rj = __shfl_sync(0xffffffffu, res, j);
            const uint32_t tj = __shfl_sync(0xffffffffu, t, j);
            unsigned long long *dj = (unsigned long long *)__shfl_sync(0xffffffffu, (unsigned long long)dbuf, j);
            raster_pixels(sj, bx0, bx1, by0, by1, (uint32_t)lane, 32u, rj, tj, dj);
        }
    }
}

// ---------------------------------------------------------------------------
// Order-preserving compaction helpers: a tile is 8 warps x 16 rounds x 32 lanes;
// warp w owns the contiguous items [base + 512w, base + 512w + 512).
// ---------------------------------------------------------------------------
constexpr int TILE_WARPS = 8;
constexpr int TILE_ROUNDS = 16;
constexpr int TILE = TILE_WARPS * TILE_ROUNDS * 32;  // 4096

__global__ void k_cover_count(const unsigned long long *__restrict__ depth, uint64_t npix,
                              uint32_t *__restrict__ blockcnt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    uint32_t c = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        c += (i < npix && depth[i] != ~0ull) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ uint32_t wc[TILE_WARPS];
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < TILE_WARPS; ++w) s += wc[w];
        blockcnt[blockIdx.x] = s;
    }
}

// Exclusive scan of a[0..n) in place by one block; total written to *total.
__global__ void __launch_bounds__(1024) k_scan_excl(uint32_t *a, uint32_t n, uint32_t *total) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < n; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < n ? a[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            ws[lane] = s;  // inclusive warp totals
        }
        __syncthreads();
        const uint32_t before = carry + (warp ? ws[warp - 1] : 0u) + x - v;
        if (i < n) a[i] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// Multi-block exclusive scan: chunk sums, scan of the sums, chunk-local scans.
constexpr uint32_t SCAN_CHUNK = 4096;

__global__ void __launch_bounds__(1024) k_chunk_sum(const uint32_t *__restrict__ a, uint64_t n,
                                                    uint32_t *__restrict__ sums) {
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_CHUNK;
    uint32_t s = 0;
    for (uint32_t r = threadIdx.x; r < SCAN_CHUNK; r += 1024)
        if (base + r < n) s += a[base + r];
    s = __reduce_add_sync(0xffffffffu, s);
    __shared__ uint32_t ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = ws[threadIdx.x];
        v = __reduce_add_sync(0xffffffffu, v);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(1024) k_chunk_scan(uint32_t *__restrict__ a, uint64_t n,
                                                     const uint32_t *__restrict__ sums) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = sums[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base0 = (uint64_t)blockIdx.x * SCAN_CHUNK;
    for (uint32_t r0 = 0; r0 < SCAN_CHUNK; r0 += 1024) {
        const uint64_t i = base0 + r0 + threadIdx.x;
        const uint32_t v = i < n ? a[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            ws[lane] = s;
        }
        __syncthreads();
        const uint32_t before = carry + (warp ? ws[warp - 1] : 0u) + x - v;
        if (i < n) a[i] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
}

// Exclusive scan of a[0..n) in place (total to *total); tmp holds n / SCAN_CHUNK + 1 words.
static void scan_excl(uint32_t *a, uint64_t n, uint32_t *total, uint32_t *tmp, cudaStream_t stream) {
    if (n <= 65536) {
        k_scan_excl<<<1, 1024, 0, stream>>>(a, (uint32_t)n, total);
        return;
    }
    const uint32_t nch = (uint32_t)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    k_chunk_sum<<<nch, 1024, 0, stream>>>(a, n, tmp);
    k_scan_excl<<<1, 1024, 0, stream>>>(tmp, nch, total);
    k_chunk_scan<<<nch, 1024, 0, stream>>>(a, n, tmp);
}

static size_t scan_tmp_words(uint64_t n) { return (size_t)(n / SCAN_CHUNK + 2); }

struct Rows {
    uint64_t *morton;
    uint64_t *key;
    uint64_t *nrm;  // 3 x int16 packed little-endian in the low 48 bits
    uint32_t *rgb;  // 3 bytes packed
    uint32_t *e;
    uint32_t *part;
    uint32_t *idx;
};

// Resolve one covered pixel of direction dir: integer barycentric interpolation of
// the quantised vertices (floor), normal of the triangle turned toward the camera
// (snorm16, round half to even), face colour.
__device__ void resolve_pixel(const TriSetup &s, const int32_t *__restrict__ q, const uint32_t *__restrict__ tri,
                              const uint8_t *__restrict__ rgb, uint32_t t, uint64_t tn, int32_t px, int32_t py,
                              uint64_t &key, uint64_t &nrm_packed, uint32_t &rgb_packed) {
    int64_t lam[3];
    cover(s, px, py, lam);
    const uint32_t vi[3] = {tri[3ull * t + 0], tri[3ull * t + 1], tri[3ull * t + 2]};
    const uint32_t slot[3] = {vi[s.ord & 3u], vi[(s.ord >> 2) & 3u], vi[(s.ord >> 4) & 3u]};
    uint64_t pos[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const uint64_t num = (uint64_t)lam[0] * (uint64_t)q[3ull * slot[0] + a] +
                             (uint64_t)lam[1] * (uint64_t)q[3ull * slot[1] + a] +
                             (uint64_t)lam[2] * (uint64_t)q[3ull * slot[2] + a];
        pos[a] = div_area(num, (uint64_t)s.area2, s.rcp);
    }
    key = pack_pos(pos[0], pos[1], pos[2]);
    nrm_packed = ((s.ord >> 24) & 1u) ? snorm_negate(tn) : tn;
    rgb_packed = rgb ? ((uint32_t)rgb[3ull * t] | ((uint32_t)rgb[3ull * t + 1] << 8) | ((uint32_t)rgb[3ull * t + 2] << 16))
                     : 0u;
}

__global__ void __launch_bounds__(256) k_resolve(const unsigned long long *__restrict__ depth, uint64_t npix,
                                                 const SPart *__restrict__ parts, const uint64_t *__restrict__ pofs,
                                                 int nparts, uint64_t T, const int32_t *__restrict__ q,
                                                 const TriSetup *__restrict__ setup, const uint64_t *__restrict__ tnrm,
                                                 const uint32_t *__restrict__ blockofs, Rows rows) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    __shared__ uint32_t wc[TILE_WARPS];
    uint32_t c = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        c += (i < npix && depth[i] != ~0ull) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    uint32_t out = blockofs[blockIdx.x];
    for (int w = 0; w < warp; ++w) out += wc[w];
    // the part of the lane's pixels, searched again only when they leave its range
    int p = -1;
    uint64_t p_lo = 1, p_hi = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        const unsigned long long dv = i < npix ? depth[i] : ~0ull;
        const bool hit = dv != ~0ull;
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const uint32_t o = out + __popc(m & ((1u << lane) - 1u));
            if (i < p_lo || i >= p_hi) {
                p = find_part(pofs, nparts, i);
                p_lo = pofs[p];
                p_hi = p + 1 < nparts ? pofs[p + 1] : npix;
            }
            const SPart &P = parts[p];
            // a part's pixels number below BS_MAX_DIRS * BS_MAX_RES^2 < 2^32
            const uint32_t res = (uint32_t)P.res, res2 = res * res;
            const uint32_t local = (uint32_t)(i - P.pofs);
            const uint32_t dir = local / res2;
            const uint32_t pix = local - dir * res2;
            const uint32_t pyu = pix / res;
            const int32_t py = (int32_t)pyu, px = (int32_t)(pix - pyu * res);
            const uint32_t t = (uint32_t)(dv & 0xffffffffull);
            const TriSetup s = setup[(uint64_t)dir * T + P.tofs + t];
            uint64_t key, np;
            uint32_t cp;
            resolve_pixel(s, q + 3ull * P.vofs, P.tri, P.rgb, t, tnrm[P.tofs + t], px, py, key, np, cp);
            rows.morton[o] = morton_of(key);
            rows.key[o] = key;
            rows.nrm[o] = np;
            rows.rgb[o] = cp;
            rows.e[o] = (uint32_t)local;
            rows.part[o] = (uint32_t)p;
            rows.idx[o] = o;
        }
        out += __popc(m);
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (u64 key, u32 value), 8-bit digits.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rs_hist(const uint64_t *__restrict__ keys, uint32_t n, int shift,
                                                 uint32_t *__restrict__ counts, uint32_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * TILE;
    for (int r = 0; r < TILE / 256; ++r) {
        const uint64_t i = base + (uint64_t)r * 256 + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// One digit pass: each block ranks its TILE rows by digit (stable: input order within a
// digit), stages them in shared memory in digit order and writes every digit's run to its
// place, so that consecutive threads store to consecutive addresses.
constexpr size_t RS_SMEM = (size_t)TILE * 12 + (size_t)TILE_WARPS * 257 * 4 + 2 * 257 * 4 + 32 * 4;
__global__ void __launch_bounds__(256) k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                    uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                    uint32_t n, int shift, const uint32_t *__restrict__ offsets,
                                                    uint32_t ntiles) {
    extern __shared__ __align__(16) unsigned char rs_sm[];
    uint64_t *sk = (uint64_t *)rs_sm;                         // the tile's keys in digit order
    uint32_t *sv = (uint32_t *)(sk + TILE);                   // and values
    uint32_t(*cnt)[257] = (uint32_t(*)[257])(sv + TILE);      // per warp and digit
    uint32_t *dstart = &cnt[TILE_WARPS][0];                   // a digit's first staged row
    uint32_t *soff = dstart + 257;                            // its output offset less dstart
    uint32_t *wsum = soff + 257;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < TILE_WARPS * 257; d += 256) (&cnt[0][0])[d] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    uint64_t k[TILE_ROUNDS];
    uint32_t v[TILE_ROUNDS], rank[TILE_ROUNDS];
#pragma unroll
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        const bool ok = i < n;
        k[r] = ok ? kin[i] : 0ull;
        v[r] = ok ? vin[i] : 0u;
        const uint32_t d = ok ? (uint32_t)((k[r] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = __popc(peers & ((1u << lane) - 1u));
        rank[r] = cnt[warp][d] + before;
        __syncwarp();
        if (before == 0) cnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // digit d: the warps' exclusive prefix, then the digits' exclusive prefix in the tile
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < TILE_WARPS; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t pre = 0;
        for (int w = 0; w < warp; ++w) pre += wsum[w];
        const uint32_t st = pre + x - run;
        dstart[d] = st;
        soff[d] = offsets[(uint64_t)d * ntiles + blockIdx.x] - st;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)((k[r] >> shift) & 255u);
            const uint32_t pos = dstart[d] + cnt[warp][d] + rank[r];
            sk[pos] = k[r];
            sv[pos] = v[r];
        }
    }
    __syncthreads();
    const uint64_t b0 = (uint64_t)blockIdx.x * TILE;
    const uint32_t nvalid = (uint32_t)min((uint64_t)TILE, (uint64_t)n - b0);
    for (uint32_t j = threadIdx.x; j < nvalid; j += 256) {
        const uint64_t key = sk[j];
        const uint32_t dst = soff[(uint32_t)((key >> shift) & 255u)] + j;
        kout[dst] = key;
        vout[dst] = sv[j];
    }
}

// Sorts (keys, vals) by the low `bits` bits of keys (bits a multiple of 16, so the
// number of passes is even and the result ends in (keys, vals)).
static void radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *ktmp, uint32_t *vtmp, uint32_t n, int bits,
                       uint32_t *counts, uint32_t *scan_tmp, cudaStream_t stream) {
    if (n == 0) return;
    const uint32_t ntiles = (n + TILE - 1) / TILE;
    uint64_t *ka = keys, *kb = ktmp;
    uint32_t *va = vals, *vb = vtmp;
    cudaFuncSetAttribute(k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RS_SMEM);
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<ntiles, 256, 0, stream>>>(ka, n, shift, counts, ntiles);
        scan_excl(counts, 256ull * ntiles, nullptr, scan_tmp, stream);
        k_rs_scatter<<<ntiles, 256, RS_SMEM, stream>>>(ka, va, kb, vb, n, shift, counts, ntiles);
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
}

// part id of each sorted row as a sort key
__global__ void k_part_keys(const uint32_t *__restrict__ idx, const uint32_t *__restrict__ part, uint32_t n,
                            uint64_t *__restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = part[idx[i]];
}

// ---------------------------------------------------------------------------
// Merge: keep the first row of each (part, Morton code).  Rows are stable-sorted by
// (part, Morton) and were emitted in increasing e, so the first has the smallest e.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool keep_row(const uint32_t *__restrict__ idx, const Rows &rows, uint64_t i) {
    if (i == 0) return true;
    const uint32_t a = idx[i], b = idx[i - 1];
    return rows.morton[a] != rows.morton[b] || rows.part[a] != rows.part[b];
}

__global__ void k_unique_count(const uint32_t *__restrict__ idx, Rows rows, uint32_t n,
                               uint32_t *__restrict__ blockcnt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    uint32_t c = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        c += (i < n && keep_row(idx, rows, i)) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ uint32_t wc[TILE_WARPS];
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < TILE_WARPS; ++w) s += wc[w];
        blockcnt[blockIdx.x] = s;
    }
}

// mode 0: record each part's [first_out, end_out); mode 1: write the kept rows of
// parts that fit their capacity
template <int MODE>
__global__ void k_unique_pass(const uint32_t *__restrict__ idx, Rows rows, uint32_t n,
                              const uint32_t *__restrict__ blockofs, const SPart *__restrict__ parts,
                              SState *__restrict__ st) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    __shared__ uint32_t wc[TILE_WARPS];
    uint32_t c = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        c += (i < n && keep_row(idx, rows, i)) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    uint32_t out = blockofs[blockIdx.x];
    for (int w = 0; w < warp; ++w) out += wc[w];
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        const bool keep = i < n && keep_row(idx, rows, i);
        const uint32_t msk = __ballot_sync(0xffffffffu, keep);
        const uint32_t o = out + __popc(msk & ((1u << lane) - 1u));
        if (i < n) {
            const uint32_t row = idx[i];
            const uint32_t p = rows.part[row];
            if (MODE == 0) {
                if (i == 0 || rows.part[idx[i - 1]] != p) st[p].first_out = o;
                if (i == n - 1 || rows.part[idx[i + 1]] != p) st[p].end_out = (uint64_t)o + (keep ? 1u : 0u);
            } else if (keep) {
                const SPart &P = parts[p];
                const uint64_t cnt = st[p].end_out - st[p].first_out;
                if (cnt <= P.cap) {
                    const uint64_t w = (uint64_t)o - st[p].first_out;
                    P.okey[w] = rows.key[row];
                    if (P.onrm) {
                        const uint64_t np = rows.nrm[row];
                        P.onrm[3 * w + 0] = (int16_t)(uint16_t)(np & 0xffffu);
                        P.onrm[3 * w + 1] = (int16_t)(uint16_t)((np >> 16) & 0xffffu);
                        P.onrm[3 * w + 2] = (int16_t)(uint16_t)((np >> 32) & 0xffffu);
                    }
                    if (P.orgb) {
                        const uint32_t cp = rows.rgb[row];
                        P.orgb[3 * w + 0] = (uint8_t)(cp & 0xffu);
                        P.orgb[3 * w + 1] = (uint8_t)((cp >> 8) & 0xffu);
                        P.orgb[3 * w + 2] = (uint8_t)((cp >> 16) & 0xffu);
                    }
                    if (P.osrc) P.osrc[w] = rows.e[row];
                }
            }
        }
        out += __popc(msk);
    }
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Scratch {
    char *base = nullptr;
    size_t off = 0;
    char *take(size_t bytes) {
        char *p = base + off;
        off = align_up(off + bytes);
        return p;
    }
};

static bs_status alloc_async(char **p, size_t bytes, cudaStream_t stream, const char *what) {
    cudaError_t e = pool_malloc_async((void **)p, bytes ? bytes : 256, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("bs_sample_visible: %s scratch allocation of %zu bytes failed: %s", what, bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA;
    }
    return BS_OK;
}

// ---------------------------------------------------------------------------
// Phase 2, shared by triangle and splat sampling: `resolve` writes one row per covered
// pixel (packed pixel order, so increasing e within a part); the rows are stable-sorted
// by Morton code and then part, the first row of each (part, position) is kept and
// every part's outputs are written.  *B receives the scratch block (freed by the caller).
// ---------------------------------------------------------------------------
template <class Resolve>
static bs_status merge_rows(uint32_t nrows, int nparts, const SPart *d_parts, SState *d_st, uint32_t *tot, int sms,
                            cudaStream_t stream, char **B, Resolve resolve) {
    if (nrows == 0) return BS_OK;
    const uint32_t rtiles = (nrows + TILE - 1) / TILE;
    Scratch Bs;
    {
        Scratch probe;
        for (int i = 0; i < 3; ++i) probe.take((size_t)nrows * 8);          // morton, key, nrm
        for (int i = 0; i < 4; ++i) probe.take((size_t)nrows * 4);          // rgb, e, part, idx
        probe.take((size_t)nrows * 8);                                      // sort key temp
        probe.take((size_t)nrows * 4);                                      // sort value temp
        probe.take((size_t)nrows * 8);                                      // part keys
        probe.take(256ull * rtiles * 4);                                    // digit counts
        probe.take(scan_tmp_words(256ull * rtiles) * 4);
        probe.take(((size_t)rtiles + 1) * 4);
        const bs_status rc = alloc_async(B, probe.off, stream, "merge");
        if (rc != BS_OK) return rc;
        Bs.base = *B;
    }
    Rows rows;
    rows.morton = (uint64_t *)Bs.take((size_t)nrows * 8);
    rows.key = (uint64_t *)Bs.take((size_t)nrows * 8);
    rows.nrm = (uint64_t *)Bs.take((size_t)nrows * 8);
    rows.rgb = (uint32_t *)Bs.take((size_t)nrows * 4);
    rows.e = (uint32_t *)Bs.take((size_t)nrows * 4);
    rows.part = (uint32_t *)Bs.take((size_t)nrows * 4);
    rows.idx = (uint32_t *)Bs.take((size_t)nrows * 4);
    uint64_t *ktmp = (uint64_t *)Bs.take((size_t)nrows * 8);
    uint32_t *vtmp = (uint32_t *)Bs.take((size_t)nrows * 4);
    uint64_t *pkey = (uint64_t *)Bs.take((size_t)nrows * 8);
    uint32_t *cnt = (uint32_t *)Bs.take(256ull * rtiles * 4);
    uint32_t *cnt_tmp = (uint32_t *)Bs.take(scan_tmp_words(256ull * rtiles) * 4);
    uint32_t *ubc = (uint32_t *)Bs.take(((size_t)rtiles + 1) * 4);
    resolve(rows);
    // stable: by Morton code, then by part (rows of one part stay in Morton order)
    uint32_t *sorted_idx = rows.idx;
    // sort a copy of the Morton codes so rows.morton stays indexable by row
    cudaMemcpyAsync(pkey, rows.morton, (size_t)nrows * 8, cudaMemcpyDeviceToDevice, stream);
    radix_sort(pkey, sorted_idx, ktmp, vtmp, nrows, 64, cnt, cnt_tmp, stream);
    if (nparts > 1) {
        k_part_keys<<<(unsigned)std::min<uint64_t>((nrows + 255) / 256, (uint64_t)sms * 32), 256, 0, stream>>>(
            sorted_idx, rows.part, nrows, pkey);
        radix_sort(pkey, sorted_idx, ktmp, vtmp, nrows, 16, cnt, cnt_tmp, stream);
    }
    k_unique_count<<<rtiles, 256, 0, stream>>>(sorted_idx, rows, nrows, ubc);
    scan_excl(ubc, rtiles, tot + 1, cnt_tmp, stream);
    k_unique_pass<0><<<rtiles, 256, 0, stream>>>(sorted_idx, rows, nrows, ubc, d_parts, d_st);
    k_unique_pass<1><<<rtiles, 256, 0, stream>>>(sorted_idx, rows, nrows, ubc, d_parts, d_st);
    return BS_OK;
}

// Host epilogue, shared: read the part states back, report counts and frames, and the
// first error (invalid part, bad triangle, capacity).
static bs_status finish_parts(int nparts, SState *d_st, std::vector<SState> &hs, bs_surfels *out,
                              cudaStream_t stream, const char *who) {
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hs.data(), d_st, (size_t)nparts * sizeof(SState), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        set_error("%s: merge phase failed: %s", who, cudaGetErrorString(cudaGetLastError()));
        return BS_ECUDA;
    }
    for (int p = 0; p < nparts; ++p) {
        const SState &S = hs[(size_t)p];
        out[p].n = S.end_out - S.first_out;
        for (int a = 0; a < 3; ++a) out[p].bbox_min[a] = S.mn[a];
        out[p].scale = S.scale;
    }
    for (int p = 0; p < nparts; ++p) {
        const SState &S = hs[(size_t)p];
        if (S.invalid) {
            out[p].n = 0;
            set_error(S.nonfinite ? "%s: part %d: non-finite vertex coordinate" : "%s: part %d: mesh has zero extent",
                      who, p);
            return BS_EINVAL;
        }
        if (S.badtri) {
            out[p].n = 0;
            set_error("%s: part %d: %u triangles reference a vertex index >= nverts", who, p, S.badtri);
            return BS_EINVAL;
        }
    }
    for (int p = 0; p < nparts; ++p)
        if (out[p].n > out[p].cap) {
            set_error("%s: part %d: %llu surfels exceed capacity %llu", who, p, (unsigned long long)out[p].n,
                      (unsigned long long)out[p].cap);
            return BS_EOVERFLOW;
        }
    return BS_OK;
}

bs_status sample_visible_parts(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs, int ndirs,
                               bs_surfels *out, cudaStream_t stream, unsigned long long *image) {
    if (nparts < 1 || nparts > 65535) { set_error("bs_sample_visible: nparts=%d outside [1, 65535]", nparts); return BS_EINVAL; }
    if (!meshes || !res || !dirs || !out) { set_error("bs_sample_visible: NULL argument"); return BS_EINVAL; }
    if (ndirs < 1 || ndirs > BS_MAX_DIRS) { set_error("bs_sample_visible: ndirs=%d outside [1,%d]", ndirs, BS_MAX_DIRS); return BS_EINVAL; }
    Views views;
    views.ndirs = ndirs;
    for (int i = 0; i < ndirs; ++i) {
        const bs_dir &d = dirs[i];
        const bool okc = d.x >= -1 && d.x <= 1 && d.y >= -1 && d.y <= 1 && d.z >= -1 && d.z <= 1;
        if (!okc || (d.x == 0 && d.y == 0 && d.z == 0)) {
            set_error("bs_sample_visible: direction %d is not a nonzero vector in {-1,0,1}^3", i);
            return BS_EINVAL;
        }
        make_frame(d, views.v[i]);
    }
    std::vector<SPart> hp((size_t)nparts);
    std::vector<uint64_t> tofs((size_t)nparts), pofs((size_t)nparts), cofs((size_t)nparts);
    uint64_t V = 0, T = 0, NP = 0, NC = 0;
    for (int p = 0; p < nparts; ++p) {
        const bs_mesh &m = meshes[p];
        if (res[p] < 1 || res[p] > BS_MAX_RES) { set_error("bs_sample_visible: part %d: res=%d outside [1,%d]", p, res[p], BS_MAX_RES); return BS_EINVAL; }
        if (m.nverts == 0 || !m.xyz) { set_error("bs_sample_visible: part %d: empty mesh", p); return BS_EINVAL; }
        if (m.ntris > 0 && !m.tri) { set_error("bs_sample_visible: part %d: NULL triangle array", p); return BS_EINVAL; }
        if (out[p].cap > 0 && !out[p].key) { set_error("bs_sample_visible: part %d: NULL key output", p); return BS_EINVAL; }
        SPart &P = hp[(size_t)p];
        P.xyz = m.xyz; P.tri = m.tri; P.rgb = m.face_rgb;
        P.okey = out[p].key; P.onrm = out[p].nrm; P.orgb = out[p].rgb; P.osrc = out[p].src;
        P.cap = out[p].cap;
        P.nverts = m.nverts; P.ntris = m.ntris; P.res = res[p]; P.pad = 0;
        P.vofs = V; P.tofs = T; P.pofs = NP;
        tofs[(size_t)p] = T;
        pofs[(size_t)p] = NP;
        cofs[(size_t)p] = NC;
        NC += (m.nverts + VCHUNK - 1) / VCHUNK;
        V += m.nverts;
        T += m.ntris;
        NP += (uint64_t)ndirs * res[p] * res[p];
    }
    if (NP >= (1ull << 32)) { set_error("bs_sample_visible: %llu pixels in one call (limit 2^32)", (unsigned long long)NP); return BS_EINVAL; }
    const uint32_t ptiles = (uint32_t)((NP + TILE - 1) / TILE);
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    // ---- phase 1: quantise, set up, raster, count covered pixels ----
    Scratch A;
    size_t a_bytes = 0;
    {
        Scratch probe;
        probe.take((size_t)nparts * sizeof(SPart));
        probe.take((size_t)nparts * sizeof(SState));
        probe.take((size_t)nparts * 8);
        probe.take((size_t)nparts * 8);
        probe.take((size_t)nparts * 8);
        probe.take(3 * V * sizeof(int32_t));
        probe.take((size_t)ndirs * T * sizeof(TriSetup));
        probe.take((size_t)T * 8);
        if (!image) probe.take(NP * sizeof(unsigned long long));
        probe.take(((size_t)ptiles + 1) * 4);
        probe.take(scan_tmp_words(ptiles) * 4);
        probe.take(16);
        a_bytes = probe.off;
    }
    bs_status rc = alloc_async(&A.base, a_bytes, stream, "raster");
    if (rc != BS_OK) return rc;
    SPart *d_parts = (SPart *)A.take((size_t)nparts * sizeof(SPart));
    SState *d_st = (SState *)A.take((size_t)nparts * sizeof(SState));
    uint64_t *d_tofs = (uint64_t *)A.take((size_t)nparts * 8);
    uint64_t *d_pofs = (uint64_t *)A.take((size_t)nparts * 8);
    uint64_t *d_cofs = (uint64_t *)A.take((size_t)nparts * 8);
    int32_t *q = (int32_t *)A.take(3 * V * sizeof(int32_t));
    TriSetup *setup = (TriSetup *)A.take((size_t)ndirs * T * sizeof(TriSetup));
    uint64_t *tnrm = (uint64_t *)A.take((size_t)T * 8);
    // the depth buffer: the caller's image when only the depth pass is wanted
    unsigned long long *depth = image ? image : (unsigned long long *)A.take(NP * sizeof(unsigned long long));
    uint32_t *bc = (uint32_t *)A.take(((size_t)ptiles + 1) * 4);
    uint32_t *stmp = (uint32_t *)A.take(scan_tmp_words(ptiles) * 4);
    uint32_t *tot = (uint32_t *)A.take(16);
    char *B = nullptr;
    std::vector<SState> hs((size_t)nparts);
    uint32_t nrows = 0;
    do {
        if (cudaMemcpyAsync(d_parts, hp.data(), (size_t)nparts * sizeof(SPart), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_tofs, tofs.data(), (size_t)nparts * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_pofs, pofs.data(), (size_t)nparts * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_cofs, cofs.data(), (size_t)nparts * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemsetAsync(depth, 0xff, NP * sizeof(unsigned long long), stream) != cudaSuccess ||
            cudaMemsetAsync(tot, 0, 16, stream) != cudaSuccess) {
            set_error("bs_sample_visible: upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = BS_ECUDA;
            break;
        }
        k_bbox_init<<<(nparts + 255) / 256, 256, 0, stream>>>(d_st, nparts);
        k_bbox<<<(unsigned)NC, 256, 0, stream>>>(d_parts, d_cofs, nparts, d_st);
        k_scale<<<(nparts + 255) / 256, 256, 0, stream>>>(d_parts, d_st, nparts);
        k_quantise<<<(unsigned)NC, 256, 0, stream>>>(d_parts, d_cofs, nparts, d_st, q);
        if (T > 0) {
            dim3 gs((unsigned)std::min<uint64_t>((T + 255) / 256, (uint64_t)sms * 32), ndirs);
            k_setup<<<gs, 256, 0, stream>>>(d_parts, d_tofs, nparts, T, q, d_st, views, setup, tnrm);
            dim3 gr((unsigned)std::min<uint64_t>((T + 255) / 256, (uint64_t)sms * 16), ndirs);
            k_raster<<<gr, 256, 0, stream>>>(d_parts, T, setup, depth);
        }
        if (image) {  // depth pass only: report the part's state, no surfels
            rc = finish_parts(nparts, d_st, hs, out, stream, "bs_render_mesh");
            break;
        }
        k_cover_count<<<ptiles, 256, 0, stream>>>(depth, NP, bc);
        scan_excl(bc, ptiles, tot, stmp, stream);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&nrows, tot, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            set_error("bs_sample_visible: raster phase failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = BS_ECUDA;
            break;
        }
        // ---- phase 2: resolve, sort, merge, write ----
        rc = merge_rows(nrows, nparts, d_parts, d_st, tot, sms, stream, &B, [&](const Rows &rows) {
            k_resolve<<<ptiles, 256, 0, stream>>>(depth, NP, d_parts, d_pofs, nparts, T, q, setup, tnrm, bc, rows);
        });
        if (rc != BS_OK) break;
        rc = finish_parts(nparts, d_st, hs, out, stream, "bs_sample_visible");
    } while (0);
    if (B) cudaFreeAsync(B, stream);
    cudaFreeAsync(A.base, stream);
    return rc;
}

bs_status sample_visible(const bs_mesh *mesh, const bs_dir *dirs, int ndirs, int res, bs_surfels *out,
                         cudaStream_t stream) {
    if (!mesh || !dirs || !out) { set_error("bs_sample_visible: NULL argument"); return BS_EINVAL; }
    return sample_visible_parts(mesh, &res, 1, dirs, ndirs, out, stream, nullptr);
}


// ===========================================================================
// Splat sampling: a parent node's initial surfel set rendered from its children's
// surfels instead of their triangles (Sec. 3.4, bottom-up), each surfel drawn as the
// oriented disc of Sec. 4.2.  Axis views only.  Coverage, depth and the emitted hit
// point are exact integer arithmetic in units of 1/(2 res) of a pixel-centre step:
// pixel (px, py) has its ray at u = ulo + (2px + 1) U1 / (2 res) (likewise v); with
// DU = (2px + 1) U1 - 2 res (cu - ulo) and nw = n.d > 0 (normal turned to the camera),
// the ray meets the plane n.(p - c) = 0 within the disc iff
//   (DU^2 + DV^2) nw^2 + (nu DU + nv DV)^2 <= R2 (2 res)^2 nw^2,
// at depth dc + (nu DU + nv DV) / (nw 2 res), dc = -(d.c) + wbias.
// ===========================================================================
struct SSet {
    const uint64_t *key;
    const int16_t *nrm;
    const uint8_t *rgb;
    const uint32_t *perm;
    float bmin[3];
    uint32_t node;
    double scale;
    int64_t r2;
};

struct Splat {          // one splat in its node's frame
    int32_t c[3];
    int16_t n[3];
    uint16_t pad;
    uint32_t rgb;       // 3 bytes packed
    uint32_t node;
    int64_t R2;         // squared radius in node units
    int64_t Rb;         // ceil(sqrt(R2))
};

__device__ __forceinline__ int64_t floor_div64(int64_t a, int64_t b) {  // b > 0
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

// splat g of the call: its set, its surfel (through perm), moved to its node's frame
__global__ void k_splat_setup(const SSet *__restrict__ sets, const uint64_t *__restrict__ sofs, int nsets, uint64_t S,
                              const SState *__restrict__ st, Splat *__restrict__ out) {
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < S; g += (uint64_t)gridDim.x * blockDim.x) {
        const int si = find_part(sofs, nsets, g);
        const SSet &T = sets[si];
        const uint64_t i = g - sofs[si];
        const uint64_t idx = T.perm ? (uint64_t)T.perm[i] : i;
        const uint64_t key = T.key[idx];
        const SState &N = st[T.node];
        const uint32_t qc[3] = {pos_x(key), pos_y(key), pos_z(key)};
        Splat sp;
        for (int a = 0; a < 3; ++a) {
            double t = __ddiv_rn((double)qc[a], T.scale);
            t = __dadd_rn((double)T.bmin[a], t);
            t = __dsub_rn(t, (double)N.mn[a]);
            t = __dmul_rn(t, N.scale);
            const double f = floor(t);
            sp.c[a] = f < 0.0 ? 0 : (f > (double)QMAX ? (int32_t)QMAX : (int32_t)f);
            sp.n[a] = T.nrm[3 * idx + a];
        }
        const double rmax2 = 3.0 * (double)QMAX * (double)QMAX;
        double r = __ddiv_rn(__dsqrt_rn(__ll2double_rn(T.r2)), T.scale);
        r = __dmul_rn(r, N.scale);
        const double rr = __dmul_rn(r, r);
        sp.R2 = rr >= rmax2 ? (int64_t)rmax2 : (int64_t)ceil(rr);
        int64_t rb = (int64_t)__dsqrt_rn(__ll2double_rn(sp.R2));
        for (int it = 0; it < 4 && rb * rb < sp.R2; ++it) ++rb;
        sp.Rb = rb;
        sp.rgb = T.rgb ? ((uint32_t)T.rgb[3 * idx] | ((uint32_t)T.rgb[3 * idx + 1] << 8) |
                          ((uint32_t)T.rgb[3 * idx + 2] << 16))
                       : 0u;
        sp.node = T.node;
        sp.pad = 0;
        out[g] = sp;
    }
}

// A splat in one view: normal components (turned to the camera), scaled centre, pixel box.
struct SplatView {
    int64_t nu, nv, nw, cu2, cv2, dc, two_res;
    int32_t px0, px1, py0, py1;
    bool flip;
};

__device__ __forceinline__ bool splat_view(const View &V, const Splat &sp, int res, SplatView &w) {
    int64_t nu = 0, nv = 0, nw = 0, cu = 0, cv = 0, cd = 0;
    for (int a = 0; a < 3; ++a) {
        nu += (int64_t)V.u[a] * sp.n[a];
        nv += (int64_t)V.v[a] * sp.n[a];
        nw += (int64_t)V.d[a] * sp.n[a];
        cu += (int64_t)V.u[a] * sp.c[a];
        cv += (int64_t)V.v[a] * sp.c[a];
        cd += (int64_t)V.d[a] * sp.c[a];
    }
    w.flip = nw < 0;
    if (w.flip) { nu = -nu; nv = -nv; nw = -nw; }
    w.nu = nu; w.nv = nv; w.nw = nw;
    w.two_res = 2 * (int64_t)res;
    w.cu2 = (cu - V.ulo) * w.two_res;
    w.cv2 = (cv - V.vlo) * w.two_res;
    w.dc = -cd + V.wbias;
    if (nw == 0) return false;  // seen edge-on
    // a covered pixel has |DU|, |DV| <= 2 res Rb
    const int64_t span = w.two_res * sp.Rb;
    int64_t px0 = -floor_div64(-(w.cu2 - span - V.U1), 2 * V.U1), px1 = floor_div64(w.cu2 + span - V.U1, 2 * V.U1);
    int64_t py0 = -floor_div64(-(w.cv2 - span - V.V1), 2 * V.V1), py1 = floor_div64(w.cv2 + span - V.V1, 2 * V.V1);
    px0 = px0 < 0 ? 0 : px0;
    py0 = py0 < 0 ? 0 : py0;
    px1 = px1 > res - 1 ? res - 1 : px1;
    py1 = py1 > res - 1 ? res - 1 : py1;
    w.px0 = (int32_t)px0; w.px1 = (int32_t)px1; w.py0 = (int32_t)py0; w.py1 = (int32_t)py1;
    return px0 <= px1 && py0 <= py1;
}

__device__ __forceinline__ void splat_pixels(const View &V, const SplatView &w, int64_t R2, uint32_t g, int res,
                                             uint32_t first, uint32_t lanes, unsigned long long *__restrict__ dbuf) {
    const uint32_t wdt = (uint32_t)(w.px1 - w.px0 + 1);
    const uint32_t npx = wdt * (uint32_t)(w.py1 - w.py0 + 1);
    const __int128 nw2 = (__int128)w.nw * w.nw;
    const __int128 rhs = (__int128)R2 * ((__int128)w.two_res * w.two_res) * nw2;
    for (uint32_t pp = first; pp < npx; pp += lanes) {
        const int32_t py = w.py0 + (int32_t)(pp / wdt), px = w.px0 + (int32_t)(pp % wdt);
        const int64_t DU = (2 * (int64_t)px + 1) * V.U1 - w.cu2;
        const int64_t DV = (2 * (int64_t)py + 1) * V.V1 - w.cv2;
        const __int128 t = (__int128)w.nu * DU + (__int128)w.nv * DV;
        const __int128 lhs = ((__int128)DU * DU + (__int128)DV * DV) * nw2 + t * t;
        if (lhs > rhs) continue;
        int64_t z = floor_div64(w.dc * w.nw * w.two_res + w.nu * DU + w.nv * DV, w.nw * w.two_res);
        z = z < 0 ? 0 : (z > 0xFFFFFFFFll ? 0xFFFFFFFFll : z);
        atomicMin(dbuf + (uint64_t)py * res + px, (unsigned long long)(((uint64_t)z << 32) | g));
    }
}

// a thread per (direction, splat); discs whose pixel box holds more than RASTER_SMALL
// pixels are drawn by the whole warp
__global__ void __launch_bounds__(256) k_splat_raster(const SPart *__restrict__ parts, uint64_t S,
                                                      const Splat *__restrict__ splats, const Views views,
                                                      unsigned long long *__restrict__ depth) {
    const int dir = blockIdx.y;
    const View &V = views.v[dir];
    const int lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < S; base += stride) {
        const uint64_t g = base + lane;
        SplatView w;
        bool valid = false;
        int res = 0;
        int64_t R2 = 0;
        unsigned long long *dbuf = nullptr;
        if (g < S) {
            const Splat sp = splats[g];
            const SPart &P = parts[sp.node];
            res = P.res;
            R2 = sp.R2;
            dbuf = depth + P.pofs + (uint64_t)dir * res * res;
            valid = splat_view(V, sp, res, w);
        }
        const uint32_t npx = valid ? (uint32_t)(w.px1 - w.px0 + 1) * (uint32_t)(w.py1 - w.py0 + 1) : 0u;
        if (valid && npx <= RASTER_SMALL) splat_pixels(V, w, R2, (uint32_t)g, res, 0u, 1u, dbuf);
        uint32_t big = __ballot_sync(0xffffffffu, npx > RASTER_SMALL);
        while (big) {
            const int j = __ffs(big) - 1;
            big &= big - 1;
            // the whole warp on lane j's disc (its record reloaded: one broadcast load)
            const Splat sj = splats[base + j];
            const SPart &Pj = parts[sj.node];
            SplatView wj;
            splat_view(V, sj, Pj.res, wj);
            splat_pixels(V, wj, sj.R2, (uint32_t)(base + j), Pj.res, (uint32_t)lane, 32u,
                         depth + Pj.pofs + (uint64_t)dir * Pj.res * Pj.res);
        }
    }
}

__global__ void __launch_bounds__(256) k_splat_resolve(const unsigned long long *__restrict__ depth, uint64_t npix,
                                                       const SPart *__restrict__ parts, const uint64_t *__restrict__ pofs,
                                                       int nparts, const Splat *__restrict__ splats, const Views views,
                                                       const uint32_t *__restrict__ blockofs, Rows rows) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    __shared__ uint32_t wc[TILE_WARPS];
    uint32_t c = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        c += (i < npix && depth[i] != ~0ull) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    uint32_t out = blockofs[blockIdx.x];
    for (int w = 0; w < warp; ++w) out += wc[w];
    int p = -1;
    uint64_t p_lo = 1, p_hi = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        const unsigned long long dv = i < npix ? depth[i] : ~0ull;
        const bool hit = dv != ~0ull;
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const uint32_t o = out + __popc(m & ((1u << lane) - 1u));
            if (i < p_lo || i >= p_hi) {
                p = find_part(pofs, nparts, i);
                p_lo = pofs[p];
                p_hi = p + 1 < nparts ? pofs[p + 1] : npix;
            }
            const SPart &P = parts[p];
            const uint64_t res2 = (uint64_t)P.res * P.res;
            const uint64_t local = i - P.pofs;
            const int dir = (int)(local / res2);
            const uint64_t pix = local - (uint64_t)dir * res2;
            const int64_t py = (int64_t)(pix / P.res), px = (int64_t)(pix % P.res);
            const uint32_t g = (uint32_t)(dv & 0xffffffffull);
            const Splat sp = splats[g];
            const View &V = views.v[dir];
            SplatView w;
            splat_view(V, sp, P.res, w);
            const int64_t DU = (2 * px + 1) * V.U1 - w.cu2;
            const int64_t DV = (2 * py + 1) * V.V1 - w.cv2;
            const int64_t W = w.nu * DU + w.nv * DV;
            uint64_t pos[3];
            for (int a = 0; a < 3; ++a) {
                int64_t q = sp.c[a];
                if (V.u[a] != 0) q += floor_div64((int64_t)V.u[a] * DU, w.two_res);
                if (V.v[a] != 0) q += floor_div64((int64_t)V.v[a] * DV, w.two_res);
                if (V.d[a] != 0) q += floor_div64(-(int64_t)V.d[a] * W, w.nw * w.two_res);
                pos[a] = (uint64_t)(q < 0 ? 0 : (q > QMAX ? QMAX : q));
            }
            const uint64_t key = pack_pos(pos[0], pos[1], pos[2]);
            uint64_t np = 0;
            for (int a = 0; a < 3; ++a) {
                const int16_t v = w.flip ? (int16_t)-sp.n[a] : sp.n[a];
                np |= (uint64_t)(uint16_t)v << (16 * a);
            }
            rows.morton[o] = morton_of(key);
            rows.key[o] = key;
            rows.nrm[o] = np;
            rows.rgb[o] = sp.rgb;
            rows.e[o] = (uint32_t)local;
            rows.part[o] = (uint32_t)p;
            rows.idx[o] = o;
        }
        out += __popc(m);
    }
}

bs_status sample_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *nodes, int nnodes, const bs_dir *dirs,
                        int ndirs, bs_surfels *out, cudaStream_t stream) {
    const char *who = "bs_sample_splats";
    if (nnodes < 1 || nnodes > 65535) { set_error("%s: nnodes=%d outside [1, 65535]", who, nnodes); return BS_EINVAL; }
    if (nsets < 0 || (nsets > 0 && !sets) || !nodes || !dirs || !out) { set_error("%s: NULL or bad argument", who); return BS_EINVAL; }
    if (ndirs < 1 || ndirs > BS_MAX_DIRS) { set_error("%s: ndirs=%d outside [1,%d]", who, ndirs, BS_MAX_DIRS); return BS_EINVAL; }
    Views views;
    views.ndirs = ndirs;
    for (int i = 0; i < ndirs; ++i) {
        const bs_dir d = dirs[i];
        const int nz = (d.x != 0) + (d.y != 0) + (d.z != 0);
        const bool unit = (d.x >= -1 && d.x <= 1) && (d.y >= -1 && d.y <= 1) && (d.z >= -1 && d.z <= 1);
        if (nz != 1 || !unit) { set_error("%s: direction %d is not an axis direction", who, i); return BS_EINVAL; }
        make_frame(d, views.v[i]);
    }
    std::vector<SPart> hp((size_t)nnodes);
    std::vector<SState> hs((size_t)nnodes);
    std::vector<uint64_t> pofs((size_t)nnodes);
    uint64_t NP = 0;
    for (int p = 0; p < nnodes; ++p) {
        const bs_splat_node &N = nodes[p];
        if (N.res < 1 || N.res > BS_MAX_RES) { set_error("%s: node %d: res=%d outside [1,%d]", who, p, N.res, BS_MAX_RES); return BS_EINVAL; }
        if (!(N.scale > 0.0) || !std::isfinite(N.scale) || !std::isfinite(N.frame_min[0]) || !std::isfinite(N.frame_min[1]) ||
            !std::isfinite(N.frame_min[2])) {
            set_error("%s: node %d: bad frame", who, p);
            return BS_EINVAL;
        }
        if (out[p].cap > 0 && !out[p].key) { set_error("%s: node %d: NULL key output", who, p); return BS_EINVAL; }
        SPart &P = hp[(size_t)p];
        memset(&P, 0, sizeof(P));
        P.okey = out[p].key; P.onrm = out[p].nrm; P.orgb = out[p].rgb; P.osrc = out[p].src;
        P.cap = out[p].cap;
        P.res = N.res;
        P.pofs = NP;
        pofs[(size_t)p] = NP;
        NP += (uint64_t)ndirs * N.res * N.res;
        SState &T = hs[(size_t)p];
        memset(&T, 0, sizeof(T));
        for (int a = 0; a < 3; ++a) T.mn[a] = N.frame_min[a];
        T.scale = N.scale;
    }
    if (NP >= (1ull << 32)) { set_error("%s: %llu pixels in one call (limit 2^32)", who, (unsigned long long)NP); return BS_EINVAL; }
    std::vector<SSet> hsets((size_t)std::max(nsets, 1));
    std::vector<uint64_t> sofs((size_t)std::max(nsets, 1));
    uint64_t S = 0;
    for (int i = 0; i < nsets; ++i) {
        const bs_splat_set &T = sets[i];
        if (T.node >= (uint32_t)nnodes) { set_error("%s: set %d: node %u >= nnodes", who, i, T.node); return BS_EINVAL; }
        if (T.n > 0 && (!T.key || !T.nrm)) { set_error("%s: set %d: NULL key or normal array", who, i); return BS_EINVAL; }
        if (T.r2 < 0 || !(T.scale > 0.0) || !std::isfinite(T.scale)) { set_error("%s: set %d: bad radius or scale", who, i); return BS_EINVAL; }
        SSet &D = hsets[(size_t)i];
        D.key = T.key; D.nrm = T.nrm; D.rgb = T.rgb; D.perm = T.perm;
        for (int a = 0; a < 3; ++a) D.bmin[a] = T.bbox_min[a];
        D.node = T.node; D.scale = T.scale; D.r2 = T.r2;
        sofs[(size_t)i] = S;
        S += T.n;
        if (S >= 0xFFFFFFFFull) { set_error("%s: more than 2^32 - 1 splats", who); return BS_EINVAL; }
    }
    const uint32_t ptiles = (uint32_t)((NP + TILE - 1) / TILE);
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    Scratch A;
    size_t a_bytes = 0;
    {
        Scratch probe;
        probe.take((size_t)nnodes * sizeof(SPart));
        probe.take((size_t)nnodes * sizeof(SState));
        probe.take((size_t)nnodes * 8);
        probe.take(hsets.size() * sizeof(SSet));
        probe.take(sofs.size() * 8);
        probe.take((size_t)std::max<uint64_t>(S, 1) * sizeof(Splat));
        probe.take(NP * sizeof(unsigned long long));
        probe.take(((size_t)ptiles + 1) * 4);
        probe.take(scan_tmp_words(ptiles) * 4);
        probe.take(16);
        a_bytes = probe.off;
    }
    bs_status rc = alloc_async(&A.base, a_bytes, stream, "splat");
    if (rc != BS_OK) return rc;
    SPart *d_parts = (SPart *)A.take((size_t)nnodes * sizeof(SPart));
    SState *d_st = (SState *)A.take((size_t)nnodes * sizeof(SState));
    uint64_t *d_pofs = (uint64_t *)A.take((size_t)nnodes * 8);
    SSet *d_sets = (SSet *)A.take(hsets.size() * sizeof(SSet));
    uint64_t *d_sofs = (uint64_t *)A.take(sofs.size() * 8);
    Splat *d_splats = (Splat *)A.take((size_t)std::max<uint64_t>(S, 1) * sizeof(Splat));
    unsigned long long *depth = (unsigned long long *)A.take(NP * sizeof(unsigned long long));
    uint32_t *bc = (uint32_t *)A.take(((size_t)ptiles + 1) * 4);
    uint32_t *stmp = (uint32_t *)A.take(scan_tmp_words(ptiles) * 4);
    uint32_t *tot = (uint32_t *)A.take(16);
    char *B = nullptr;
    uint32_t nrows = 0;
    do {
        if (cudaMemcpyAsync(d_parts, hp.data(), (size_t)nnodes * sizeof(SPart), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_st, hs.data(), (size_t)nnodes * sizeof(SState), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_pofs, pofs.data(), (size_t)nnodes * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_sets, hsets.data(), hsets.size() * sizeof(SSet), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_sofs, sofs.data(), sofs.size() * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemsetAsync(depth, 0xff, NP * sizeof(unsigned long long), stream) != cudaSuccess ||
            cudaMemsetAsync(tot, 0, 16, stream) != cudaSuccess) {
            set_error("%s: upload failed: %s", who, cudaGetErrorString(cudaGetLastError()));
            rc = BS_ECUDA;
            break;
        }
        if (S > 0) {
            k_splat_setup<<<(unsigned)std::min<uint64_t>((S + 255) / 256, (uint64_t)sms * 32), 256, 0, stream>>>(
                d_sets, d_sofs, nsets, S, d_st, d_splats);
            dim3 gr((unsigned)std::min<uint64_t>((S + 255) / 256, (uint64_t)sms * 16), ndirs);
            k_splat_raster<<<gr, 256, 0, stream>>>(d_parts, S, d_splats, views, depth);
        }
        k_cover_count<<<ptiles, 256, 0, stream>>>(depth, NP, bc);
        scan_excl(bc, ptiles, tot, stmp, stream);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&nrows, tot, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            set_error("%s: raster phase failed: %s", who, cudaGetErrorString(cudaGetLastError()));
            rc = BS_ECUDA;
            break;
        }
        rc = merge_rows(nrows, nnodes, d_parts, d_st, tot, sms, stream, &B, [&](const Rows &rows) {
            k_splat_resolve<<<ptiles, 256, 0, stream>>>(depth, NP, d_parts, d_pofs, nnodes, d_splats, views, bc, rows);
        });
        if (rc != BS_OK) break;
        rc = finish_parts(nnodes, d_st, hs, out, stream, who);
    } while (0);
    if (B) cudaFreeAsync(B, stream);
    cudaFreeAsync(A.base, stream);
    return rc;
}

// Headless render of a mesh for one direction: the depth pass of bs_sample_visible alone.
bs_status render_mesh(const bs_mesh *mesh, const bs_dir *dir, int res, unsigned long long *image, cudaStream_t stream) {
    if (!mesh || !dir || !image) { set_error("bs_render_mesh: NULL argument"); return BS_EINVAL; }
    bs_surfels out;
    memset(&out, 0, sizeof(out));
    return sample_visible_parts(mesh, &res, 1, dir, 1, &out, stream, image);
}

// Headless render of discs for one axis direction: the depth pass of bs_sample_splats
// alone, into the caller's res x res image.
bs_status render_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *node, const bs_dir *dir,
                        unsigned long long *image, cudaStream_t stream) {
    const char *who = "bs_render_splats";
    if ((nsets > 0 && !sets) || nsets < 0 || !node || !dir || !image) { set_error("%s: NULL or bad argument", who); return BS_EINVAL; }
    const int nz = (dir->x != 0) + (dir->y != 0) + (dir->z != 0);
    if (nz != 1 || dir->x < -1 || dir->x > 1 || dir->y < -1 || dir->y > 1 || dir->z < -1 || dir->z > 1) {
        set_error("%s: not an axis direction", who);
        return BS_EINVAL;
    }
    if (node->res < 1 || node->res > BS_MAX_RES || !(node->scale > 0.0) || !std::isfinite(node->scale)) {
        set_error("%s: bad node resolution or scale", who);
        return BS_EINVAL;
    }
    Views views;
    views.ndirs = 1;
    make_frame(*dir, views.v[0]);
    SPart hp;
    memset(&hp, 0, sizeof(hp));
    hp.res = node->res;
    SState hs;
    memset(&hs, 0, sizeof(hs));
    for (int a = 0; a < 3; ++a) hs.mn[a] = node->frame_min[a];
    hs.scale = node->scale;
    std::vector<SSet> hsets((size_t)std::max(nsets, 1));
    std::vector<uint64_t> sofs((size_t)std::max(nsets, 1));
    uint64_t S = 0;
    for (int i = 0; i < nsets; ++i) {
        const bs_splat_set &T = sets[i];
        if (T.n > 0 && (!T.key || !T.nrm)) { set_error("%s: set %d: NULL key or normal array", who, i); return BS_EINVAL; }
        if (T.r2 < 0 || !(T.scale > 0.0) || !std::isfinite(T.scale)) { set_error("%s: set %d: bad radius or scale", who, i); return BS_EINVAL; }
        SSet &D = hsets[(size_t)i];
        D.key = T.key; D.nrm = T.nrm; D.rgb = T.rgb; D.perm = T.perm;
        for (int a = 0; a < 3; ++a) D.bmin[a] = T.bbox_min[a];
        D.node = 0; D.scale = T.scale; D.r2 = T.r2;
        sofs[(size_t)i] = S;
        S += T.n;
        if (S >= 0xFFFFFFFFull) { set_error("%s: more than 2^32 - 1 splats", who); return BS_EINVAL; }
    }
    const uint64_t npix = (uint64_t)node->res * node->res;
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    Scratch A;
    {
        Scratch probe;
        probe.take(sizeof(SPart));
        probe.take(sizeof(SState));
        probe.take(hsets.size() * sizeof(SSet));
        probe.take(sofs.size() * 8);
        probe.take((size_t)std::max<uint64_t>(S, 1) * sizeof(Splat));
        bs_status rc = alloc_async(&A.base, probe.off, stream, "splat render");
        if (rc != BS_OK) return rc;
    }
    SPart *d_parts = (SPart *)A.take(sizeof(SPart));
    SState *d_st = (SState *)A.take(sizeof(SState));
    SSet *d_sets = (SSet *)A.take(hsets.size() * sizeof(SSet));
    uint64_t *d_sofs = (uint64_t *)A.take(sofs.size() * 8);
    Splat *d_splats = (Splat *)A.take((size_t)std::max<uint64_t>(S, 1) * sizeof(Splat));
    bs_status rc = BS_OK;
    if (cudaMemcpyAsync(d_parts, &hp, sizeof(SPart), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(d_st, &hs, sizeof(SState), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(d_sets, hsets.data(), hsets.size() * sizeof(SSet), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(d_sofs, sofs.data(), sofs.size() * 8, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemsetAsync(image, 0xff, npix * sizeof(unsigned long long), stream) != cudaSuccess) {
        set_error("%s: upload failed: %s", who, cudaGetErrorString(cudaGetLastError()));
        rc = BS_ECUDA;
    } else if (S > 0) {
        k_splat_setup<<<(unsigned)std::min<uint64_t>((S + 255) / 256, (uint64_t)sms * 32), 256, 0, stream>>>(
            d_sets, d_sofs, nsets, S, d_st, d_splats);
        dim3 gr((unsigned)std::min<uint64_t>((S + 255) / 256, (uint64_t)sms * 16), 1);
        k_splat_raster<<<gr, 256, 0, stream>>>(d_parts, S, d_splats, views, image);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("%s: launch failed", who);
            rc = BS_ECUDA;
        }
    }
    cudaFreeAsync(A.base, stream);
    return rc;
}

}  // namespace bs
