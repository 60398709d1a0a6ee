// bs_sample.cu -- visible-surface sampling (Sec. 3.1): quantise a mesh, rasterise it
// orthographically from several integer directions with an integer rasteriser,
// emit one surfel per covered pixel, merge identical positions and sort the
// surfels into ascending Morton order.
//
// Pipeline (all on the caller's stream):
//   k_bbox -> k_scale -> k_quantise              node-local 21-bit integer positions
//   k_setup   (dir x triangle)                   snapped screen coords, winding, area
//   k_raster  (warp per dir x triangle)          64-bit atomicMin(depth << 32 | tri)
//   k_cover_count -> scan -> k_resolve           covered pixels in emission order
//   radix sort (Morton code, row)                stable LSD, 8-bit digits
//   k_unique_count -> scan -> k_unique_write     keep the first row of each position
//
// Arithmetic: integers throughout, except the quantiser (IEEE double subtract and
// multiply, written with explicit round-to-nearest intrinsics so nothing is fused)
// and the unit normal (IEEE double multiply/add/sqrt/divide, same intrinsics).
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
};

struct Views {
    View v[BS_MAX_DIRS];
    int ndirs;
    int res;
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
}

// ---------------------------------------------------------------------------
// Quantisation: bbox over float32 vertices, isotropic scale S = (2^21-1)/E.
// ---------------------------------------------------------------------------
struct QuantState {
    uint32_t mn_ord[3], mx_ord[3];  // order-preserving encodings of the float bounds
    uint32_t nonfinite;
    uint32_t invalid;
    uint32_t badtri;  // triangles with a vertex index >= nverts
    float mn[3];
    double scale;
    uint32_t count;  // surfels after dedup
    uint32_t rows;   // covered pixels before dedup
};

__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__global__ void k_bbox(const float *__restrict__ xyz, uint32_t nverts, QuantState *st) {
    uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u}, bad = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nverts; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float f = xyz[3ull * i + a];
            if (!isfinite(f)) {
                ++bad;
            } else {
                const uint32_t o = f2ord(f);
                mn[a] = min(mn[a], o);
                mx[a] = max(mx[a], o);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(0xffffffffu, mn[a]);
        mx[a] = __reduce_max_sync(0xffffffffu, mx[a]);
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&st->mn_ord[a], mn[a]);
            atomicMax(&st->mx_ord[a], mx[a]);
        }
        if (bad) atomicAdd(&st->nonfinite, bad);
    }
}

__global__ void k_scale(QuantState *st) {
    double E = 0.0;
    for (int a = 0; a < 3; ++a) {
        const float mn = ord2f(st->mn_ord[a]);
        const float mx = ord2f(st->mx_ord[a]);
        const double e = __dsub_rn((double)mx, (double)mn);
        if (e > E) E = e;
        st->mn[a] = __fadd_rn(mn, 0.0f);  // report -0.0 as +0.0
    }
    st->invalid = (st->nonfinite != 0u || !(E > 0.0)) ? 1u : 0u;
    st->scale = st->invalid ? 0.0 : __ddiv_rn(2097151.0, E);
}

__global__ void k_quantise(const float *__restrict__ xyz, uint32_t nverts, const QuantState *st,
                           int32_t *__restrict__ q) {
    if (st->invalid) return;
    const double S = st->scale;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < 3ull * nverts;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i % 3);
        const double t = __dmul_rn(__dsub_rn((double)xyz[i], (double)st->mn[a]), S);
        int64_t v = (int64_t)floor(t);
        v = v < 0 ? 0 : (v > QMAX ? QMAX : v);
        q[i] = (int32_t)v;
    }
}

// ---------------------------------------------------------------------------
// Triangle setup per (direction, triangle): snapped integer screen coordinates,
// biased depth, winding normalised so that area2 > 0 (vertex order kept in ord).
// ---------------------------------------------------------------------------
struct TriSetup {
    int32_t x[3], y[3];
    uint32_t w[3];
    uint32_t ord;  // bits 0-1: input vertex of slot 0, 2-3 slot 1, 4-5 slot 2; 0xffffffff = skip
    int64_t area2;
};

__device__ __forceinline__ void project(const View &V, int res, const int32_t *q, int32_t &X, int32_t &Y,
                                        uint32_t &W) {
    const int64_t x = q[0], y = q[1], z = q[2];
    const int64_t uq = V.u[0] * x + V.u[1] * y + V.u[2] * z;
    const int64_t vq = V.v[0] * x + V.v[1] * y + V.v[2] * z;
    const int64_t dq = V.d[0] * x + V.d[1] * y + V.d[2] * z;
    X = (int32_t)(((uq - V.ulo) * res * 512 + V.U1) / (2 * V.U1));
    Y = (int32_t)(((vq - V.vlo) * res * 512 + V.V1) / (2 * V.V1));
    W = (uint32_t)(-dq + V.wbias);
}

__global__ void k_setup(const int32_t *__restrict__ q, const uint32_t *__restrict__ tri, uint32_t ntris,
                        uint32_t nverts, QuantState *st, const Views views, TriSetup *__restrict__ out) {
    if (st->invalid) return;
    const int dir = blockIdx.y;
    const View &V = views.v[dir];
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntris; t += gridDim.x * blockDim.x) {
        if (tri[3ull * t] >= nverts || tri[3ull * t + 1] >= nverts || tri[3ull * t + 2] >= nverts) {
            TriSetup bad{};
            bad.ord = 0xffffffffu;
            out[(uint64_t)dir * ntris + t] = bad;
            if (dir == 0) atomicAdd(&st->badtri, 1u);
            continue;
        }
        int32_t X[3], Y[3];
        uint32_t W[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) project(V, views.res, q + 3ull * tri[3ull * t + i], X[i], Y[i], W[i]);
        int64_t a2 = (int64_t)(X[1] - X[0]) * (Y[2] - Y[0]) - (int64_t)(Y[1] - Y[0]) * (X[2] - X[0]);
        int o1 = 1, o2 = 2;
        if (a2 < 0) { o1 = 2; o2 = 1; a2 = -a2; }
        TriSetup s;
        s.x[0] = X[0]; s.y[0] = Y[0]; s.w[0] = W[0];
        s.x[1] = X[o1]; s.y[1] = Y[o1]; s.w[1] = W[o1];
        s.x[2] = X[o2]; s.y[2] = Y[o2]; s.w[2] = W[o2];
        s.ord = a2 == 0 ? 0xffffffffu : (uint32_t)(0 | (o1 << 2) | (o2 << 4));
        s.area2 = a2;
        out[(uint64_t)dir * ntris + t] = s;
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

// One warp per (direction, triangle); lanes stride over the pixels of its screen bbox.
__global__ void __launch_bounds__(256) k_raster(const TriSetup *__restrict__ setup, uint32_t ntris, int res,
                                                const QuantState *st, unsigned long long *__restrict__ depth) {
    if (st->invalid) return;
    const int dir = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const uint32_t warps_per_grid = gridDim.x * (blockDim.x >> 5);
    unsigned long long *dbuf = depth + (uint64_t)dir * res * res;
    for (uint32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntris; t += warps_per_grid) {
        const TriSetup s = setup[(uint64_t)dir * ntris + t];
        if (s.ord == 0xffffffffu) continue;
        const int32_t xmin = min(s.x[0], min(s.x[1], s.x[2])), xmax = max(s.x[0], max(s.x[1], s.x[2]));
        const int32_t ymin = min(s.y[0], min(s.y[1], s.y[2])), ymax = max(s.y[0], max(s.y[1], s.y[2]));
        int32_t px0, px1, py0, py1;
        pixel_span(xmin, xmax, res, px0, px1);
        pixel_span(ymin, ymax, res, py0, py1);
        if (px1 < px0 || py1 < py0) continue;
        const uint32_t wdt = (uint32_t)(px1 - px0 + 1);
        const uint32_t npx = wdt * (uint32_t)(py1 - py0 + 1);
        for (uint32_t p = lane; p < npx; p += 32) {
            const int32_t py = py0 + (int32_t)(p / wdt), px = px0 + (int32_t)(p % wdt);
            int64_t lam[3];
            if (!cover(s, px, py, lam)) continue;
            const uint64_t num = (uint64_t)lam[0] * s.w[0] + (uint64_t)lam[1] * s.w[1] + (uint64_t)lam[2] * s.w[2];
            const uint64_t z = num / (uint64_t)s.area2;
            atomicMin(dbuf + (uint64_t)py * res + px, (unsigned long long)((z << 32) | t));
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

__global__ void k_cover_count(const unsigned long long *__restrict__ depth, uint64_t npix, const QuantState *st,
                              uint32_t *__restrict__ blockcnt) {
    if (st->invalid) return;
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

struct Rows {
    uint64_t *morton;
    uint64_t *key;
    uint64_t *nrm;  // 3 x int16 packed little-endian in the low 48 bits
    uint32_t *rgb;  // 3 bytes packed
    uint32_t *e;
    uint32_t *idx;
};

// Resolve one covered pixel of direction dir: integer barycentric interpolation of
// the quantised vertices (floor), normal of the triangle turned toward the camera
// (snorm16, round half to even), face colour, Morton code.
__device__ void resolve_pixel(const View &V, const TriSetup &s, const int32_t *__restrict__ q,
                              const uint32_t *__restrict__ tri, const uint8_t *__restrict__ rgb, uint32_t t,
                              int32_t px, int32_t py, uint64_t &key, uint64_t &nrm_packed, uint32_t &rgb_packed) {
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
        pos[a] = num / (uint64_t)s.area2;
    }
    key = pack_pos(pos[0], pos[1], pos[2]);
    int64_t e1[3], e2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e1[a] = (int64_t)q[3ull * vi[1] + a] - q[3ull * vi[0] + a];
        e2[a] = (int64_t)q[3ull * vi[2] + a] - q[3ull * vi[0] + a];
    }
    int64_t n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const int64_t nd = n[0] * V.d[0] + n[1] * V.d[1] + n[2] * V.d[2];
    if (nd < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
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
    nrm_packed = np;
    rgb_packed = rgb ? ((uint32_t)rgb[3ull * t] | ((uint32_t)rgb[3ull * t + 1] << 8) | ((uint32_t)rgb[3ull * t + 2] << 16))
                     : 0u;
}

__global__ void __launch_bounds__(256) k_resolve(const unsigned long long *__restrict__ depth, uint64_t npix, int res,
                                                 const int32_t *__restrict__ q, const uint32_t *__restrict__ tri,
                                                 const uint8_t *__restrict__ rgb, const TriSetup *__restrict__ setup,
                                                 uint32_t ntris, const Views views, const QuantState *st,
                                                 const uint32_t *__restrict__ blockofs, Rows rows) {
    if (st->invalid) return;
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
    const uint64_t res2 = (uint64_t)res * res;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        const unsigned long long dv = i < npix ? depth[i] : ~0ull;
        const bool hit = dv != ~0ull;
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        if (hit) {
            const uint32_t o = out + __popc(m & ((1u << lane) - 1u));
            const int dir = (int)(i / res2);
            const uint64_t pix = i - (uint64_t)dir * res2;
            const int32_t py = (int32_t)(pix / res), px = (int32_t)(pix % res);
            const uint32_t t = (uint32_t)(dv & 0xffffffffull);
            const TriSetup s = setup[(uint64_t)dir * ntris + t];
            uint64_t key, np;
            uint32_t cp;
            resolve_pixel(views.v[dir], s, q, tri, rgb, t, px, py, key, np, cp);
            rows.morton[o] = morton_of(key);
            rows.key[o] = key;
            rows.nrm[o] = np;
            rows.rgb[o] = cp;
            rows.e[o] = (uint32_t)i;
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

__global__ void __launch_bounds__(256) k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                    uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                    uint32_t n, int shift, const uint32_t *__restrict__ offsets,
                                                    uint32_t ntiles) {
    __shared__ uint32_t cnt[TILE_WARPS][257];
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
    // exclusive prefix over warps for each digit
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < TILE_WARPS; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)((k[r] >> shift) & 255u);
            const uint32_t dst = offsets[(uint64_t)d * ntiles + blockIdx.x] + cnt[warp][d] + rank[r];
            kout[dst] = k[r];
            vout[dst] = v[r];
        }
    }
}

// Sorts (keys, vals) by the low `bits` bits of keys; bits must be a multiple of 8
// and the number of passes even, so the result ends in (keys, vals).
static bs_status radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *ktmp, uint32_t *vtmp, uint32_t n, int bits,
                            uint32_t *counts, cudaStream_t stream) {
    if (n == 0) return BS_OK;
    const uint32_t ntiles = (n + TILE - 1) / TILE;
    uint64_t *ka = keys, *kb = ktmp;
    uint32_t *va = vals, *vb = vtmp;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<ntiles, 256, 0, stream>>>(ka, n, shift, counts, ntiles);
        k_scan_excl<<<1, 1024, 0, stream>>>(counts, 256u * ntiles, nullptr);
        k_rs_scatter<<<ntiles, 256, 0, stream>>>(ka, va, kb, vb, n, shift, counts, ntiles);
        BS_CHECK_LAUNCH();
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    return BS_OK;
}

// ---------------------------------------------------------------------------
// Dedup: keep the first row of each Morton code (rows are stable-sorted by Morton
// code and were emitted in increasing e, so the first row has the smallest e).
// ---------------------------------------------------------------------------
__global__ void k_unique_count(const uint64_t *__restrict__ m, uint32_t n, uint32_t *__restrict__ blockcnt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    uint32_t c = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        c += (i < n && (i == 0 || m[i] != m[i - 1])) ? 1u : 0u;
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

__global__ void k_unique_write(const uint64_t *__restrict__ m, const uint32_t *__restrict__ idx, uint32_t n,
                               const uint32_t *__restrict__ blockofs, const uint32_t *__restrict__ total,
                               uint64_t cap, Rows rows, uint64_t *__restrict__ okey, int16_t *__restrict__ onrm,
                               uint8_t *__restrict__ orgb, uint32_t *__restrict__ osrc) {
    if ((uint64_t)*total > cap) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t base = (uint64_t)blockIdx.x * TILE + (uint64_t)warp * TILE_ROUNDS * 32;
    __shared__ uint32_t wc[TILE_WARPS];
    uint32_t c = 0;
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        c += (i < n && (i == 0 || m[i] != m[i - 1])) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) wc[warp] = c;
    __syncthreads();
    uint32_t out = blockofs[blockIdx.x];
    for (int w = 0; w < warp; ++w) out += wc[w];
    for (int r = 0; r < TILE_ROUNDS; ++r) {
        const uint64_t i = base + (uint64_t)r * 32 + lane;
        const bool keep = i < n && (i == 0 || m[i] != m[i - 1]);
        const uint32_t msk = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint32_t o = out + __popc(msk & ((1u << lane) - 1u));
            const uint32_t row = idx[i];
            okey[o] = rows.key[row];
            if (onrm) {
                const uint64_t np = rows.nrm[row];
                onrm[3ull * o + 0] = (int16_t)(uint16_t)(np & 0xffffu);
                onrm[3ull * o + 1] = (int16_t)(uint16_t)((np >> 16) & 0xffffu);
                onrm[3ull * o + 2] = (int16_t)(uint16_t)((np >> 32) & 0xffffu);
            }
            if (orgb) {
                const uint32_t cp = rows.rgb[row];
                orgb[3ull * o + 0] = (uint8_t)(cp & 0xffu);
                orgb[3ull * o + 1] = (uint8_t)((cp >> 8) & 0xffu);
                orgb[3ull * o + 2] = (uint8_t)((cp >> 16) & 0xffu);
            }
            if (osrc) osrc[o] = rows.e[row];
        }
        out += __popc(msk);
    }
}

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

bs_status sample_visible(const bs_mesh *mesh, const bs_dir *dirs, int ndirs, int res, bs_surfels *out,
                         cudaStream_t stream) {
    if (!mesh || !dirs || !out) { set_error("bs_sample_visible: NULL argument"); return BS_EINVAL; }
    if (ndirs < 1 || ndirs > BS_MAX_DIRS) { set_error("bs_sample_visible: ndirs=%d outside [1,%d]", ndirs, BS_MAX_DIRS); return BS_EINVAL; }
    if (res < 1 || res > BS_MAX_RES) { set_error("bs_sample_visible: res=%d outside [1,%d]", res, BS_MAX_RES); return BS_EINVAL; }
    if (mesh->nverts == 0 || !mesh->xyz) { set_error("bs_sample_visible: empty mesh"); return BS_EINVAL; }
    if (mesh->ntris > 0 && !mesh->tri) { set_error("bs_sample_visible: NULL triangle array"); return BS_EINVAL; }
    if (out->cap > 0 && !out->key) { set_error("bs_sample_visible: NULL key output"); return BS_EINVAL; }
    Views views;
    views.ndirs = ndirs;
    views.res = res;
    for (int i = 0; i < ndirs; ++i) {
        const bs_dir &d = dirs[i];
        const bool okc = d.x >= -1 && d.x <= 1 && d.y >= -1 && d.y <= 1 && d.z >= -1 && d.z <= 1;
        if (!okc || (d.x == 0 && d.y == 0 && d.z == 0)) {
            set_error("bs_sample_visible: direction %d is not a nonzero vector in {-1,0,1}^3", i);
            return BS_EINVAL;
        }
        make_frame(d, views.v[i]);
    }
    const uint32_t nv = mesh->nverts, nt = mesh->ntris;
    const uint64_t npix = (uint64_t)ndirs * res * res;
    if (npix >= (1ull << 32)) { set_error("bs_sample_visible: too many pixels"); return BS_EINVAL; }
    const uint32_t ptiles = (uint32_t)((npix + TILE - 1) / TILE);
    const uint32_t rs_tiles_max = ptiles;

    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    const size_t o_st = take(sizeof(QuantState));
    const size_t o_q = take(3ull * nv * sizeof(int32_t));
    const size_t o_setup = take((size_t)ndirs * nt * sizeof(TriSetup));
    const size_t o_depth = take(npix * sizeof(unsigned long long));
    const size_t o_bc = take(((size_t)ptiles + 1) * sizeof(uint32_t));
    const size_t o_tot = take(4 * sizeof(uint32_t));
    const size_t o_cnt = take(256ull * rs_tiles_max * sizeof(uint32_t));
    // rows (capacity npix; only `rows` of them used)
    const size_t o_m = take(npix * 8), o_k = take(npix * 8), o_n = take(npix * 8);
    const size_t o_c = take(npix * 4), o_e = take(npix * 4), o_i = take(npix * 4);
    const size_t o_m2 = take(npix * 8), o_i2 = take(npix * 4);
    char *ws = nullptr;
    {
        cudaError_t e = cudaMallocAsync((void **)&ws, off, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("bs_sample_visible: scratch allocation of %zu bytes failed: %s", off, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA;
        }
    }
    bs_status rc = BS_OK;
    QuantState *st = (QuantState *)(ws + o_st);
    int32_t *q = (int32_t *)(ws + o_q);
    TriSetup *setup = (TriSetup *)(ws + o_setup);
    unsigned long long *depth = (unsigned long long *)(ws + o_depth);
    uint32_t *bc = (uint32_t *)(ws + o_bc);
    uint32_t *tot = (uint32_t *)(ws + o_tot);
    uint32_t *cnt = (uint32_t *)(ws + o_cnt);
    Rows rows{(uint64_t *)(ws + o_m), (uint64_t *)(ws + o_k), (uint64_t *)(ws + o_n),
              (uint32_t *)(ws + o_c), (uint32_t *)(ws + o_e), (uint32_t *)(ws + o_i)};
    QuantState h{};
    int sms = 152;
    do {
        {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        }
        QuantState init{};
        for (int a = 0; a < 3; ++a) { init.mn_ord[a] = 0xffffffffu; init.mx_ord[a] = 0u; }
        if ((rc = cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, stream) == cudaSuccess ? BS_OK : BS_ECUDA)) {
            set_error("bs_sample_visible: state upload failed");
            break;
        }
        const int gb = (int)std::min<uint64_t>((nv + 255) / 256, (uint64_t)sms * 8);
        k_bbox<<<gb, 256, 0, stream>>>(mesh->xyz, nv, st);
        k_scale<<<1, 1, 0, stream>>>(st);
        k_quantise<<<(int)std::min<uint64_t>((3ull * nv + 255) / 256, (uint64_t)sms * 16), 256, 0, stream>>>(mesh->xyz, nv, st, q);
        if (cudaMemsetAsync(depth, 0xff, npix * sizeof(unsigned long long), stream) != cudaSuccess) {
            rc = BS_ECUDA; set_error("bs_sample_visible: memset failed"); break;
        }
        if (nt > 0) {
            dim3 gs((unsigned)std::min<uint64_t>((nt + 255) / 256, 4096), ndirs);
            k_setup<<<gs, 256, 0, stream>>>(q, mesh->tri, nt, nv, st, views, setup);
            dim3 gr((unsigned)std::min<uint64_t>((nt + 7) / 8, (uint64_t)sms * 64), ndirs);
            k_raster<<<gr, 256, 0, stream>>>(setup, nt, res, st, depth);
        }
        k_cover_count<<<ptiles, 256, 0, stream>>>(depth, npix, st, bc);
        k_scan_excl<<<1, 1024, 0, stream>>>(bc, ptiles, tot + 0);
        k_resolve<<<ptiles, 256, 0, stream>>>(depth, npix, res, q, mesh->tri, mesh->face_rgb, setup, nt, views, st, bc, rows);
        if ((rc = cudaGetLastError() == cudaSuccess ? BS_OK : BS_ECUDA)) { set_error("bs_sample_visible: launch failed"); break; }
        // number of rows is needed on the host to size the sort
        uint32_t nrows = 0;
        if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaMemcpyAsync(&nrows, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) {
            rc = BS_ECUDA; set_error("bs_sample_visible: readback failed: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        if (h.badtri) {
            rc = BS_EINVAL;
            set_error("bs_sample_visible: %u triangles reference a vertex index >= nverts", h.badtri);
            break;
        }
        if (h.invalid) {
            rc = BS_EINVAL;
            set_error(h.nonfinite ? "bs_sample_visible: non-finite vertex coordinate" : "bs_sample_visible: mesh has zero extent");
            break;
        }
        if (h.invalid == 0 && nrows > 0) {
            if ((rc = radix_sort(rows.morton, rows.idx, (uint64_t *)(ws + o_m2), (uint32_t *)(ws + o_i2), nrows, 64, cnt, stream)) != BS_OK) break;
            const uint32_t utiles = (nrows + TILE - 1) / TILE;
            k_unique_count<<<utiles, 256, 0, stream>>>(rows.morton, nrows, bc);
            k_scan_excl<<<1, 1024, 0, stream>>>(bc, utiles, tot + 1);
            k_unique_write<<<utiles, 256, 0, stream>>>(rows.morton, rows.idx, nrows, bc, tot + 1, out->cap, rows,
                                                       out->key, out->nrm, out->rgb, out->src);
            if ((rc = cudaGetLastError() == cudaSuccess ? BS_OK : BS_ECUDA)) { set_error("bs_sample_visible: launch failed"); break; }
        }
        uint32_t nout = 0;
        if (nrows > 0) {
            if (cudaMemcpyAsync(&nout, tot + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                rc = BS_ECUDA; set_error("bs_sample_visible: readback failed"); break;
            }
        }
        out->n = nout;
        for (int a = 0; a < 3; ++a) out->bbox_min[a] = h.mn[a];
        out->scale = h.scale;
        if ((uint64_t)nout > out->cap) {
            rc = BS_EOVERFLOW;
            set_error("bs_sample_visible: %u surfels exceed capacity %llu", nout, (unsigned long long)out->cap);
        }
    } while (0);
    cudaFreeAsync(ws, stream);
    if (rc == BS_OK) {
        cudaError_t e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) { set_error("bs_sample_visible: %s", cudaGetErrorString(e)); rc = BS_ECUDA; }
    }
    return rc;
}

}  // namespace bs
