/*
 * bs_oracle.c -- CPU oracle for visible-surface surfel sampling and progressive
 * (greedy-permutation) ordering, after Brandt et al., "Rendering of Complex
 * Heterogenous Scenes using Progressive Blue Surfels".
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * statement of what the surfel path computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline / reference legs load it; the product
 * path never does.  It shares no code, header, table or helper with the CUDA
 * library: every step below is written out here on its own, in the order the
 * method states it.
 *
 * Arithmetic: everything is integer (int64 / uint64) except
 *   - the quantiser (Sec. 3.1: positions in the node-local frame), which uses
 *     IEEE double subtraction and multiplication, and
 *   - the unit normal (Sec. 3.1: a normal buffer), which uses IEEE double
 *     multiply, add, sqrt and divide.
 * Build with -ffp-contract=off so no multiply-add is fused.
 *
 * Readings of the paper that fix details it leaves open (frame, pixel centres,
 * coverage tie rule, depth and position interpolation, normal format,
 * duplicate merge, tie-break, start index) are stated next to each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_Q ((int64_t)2097151) /* 2^21 - 1: largest quantised coordinate */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11).  Round: two 32x32->64 products of the counter   */
/* words 0 and 2 with the multipliers, outputs permuted and xored with the   */
/* odd counter words and the key; the key is bumped by the Weyl constants    */
/* between rounds.  Used for the "random starting surfel" of Sec. 3.2.       */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Morton code of a quantised point: bit 3i holds x_i, 3i+1 y_i, 3i+2 z_i. */
uint64_t or_morton3(uint32_t x, uint32_t y, uint32_t z)
{
    uint64_t m = 0;
    for (int i = 0; i < 21; i++) {
        m |= (uint64_t)((x >> i) & 1u) << (3 * i);
        m |= (uint64_t)((y >> i) & 1u) << (3 * i + 1);
        m |= (uint64_t)((z >> i) & 1u) << (3 * i + 2);
    }
    return m;
}

/* Packed surfel key: x in bits 42..62, y in 21..41, z in 0..20. */
static uint64_t pack_key(int64_t x, int64_t y, int64_t z)
{
    return ((uint64_t)x << 42) | ((uint64_t)y << 21) | (uint64_t)z;
}
static void unpack_key(uint64_t k, int64_t p[3])
{
    p[0] = (int64_t)((k >> 42) & 0x1FFFFF);
    p[1] = (int64_t)((k >> 21) & 0x1FFFFF);
    p[2] = (int64_t)(k & 0x1FFFFF);
}

/* ------------------------------------------------------------------------ */
/* Quantisation (Sec. 3.1: surfel positions live in the node's local frame). */
/* bbox over the float32 vertices; one isotropic scale S = (2^21-1)/E for    */
/* the largest side E (double); q = clamp(floor((x - min) * S), 0, 2^21-1).  */
/* Returns 0, or 1 for a non-finite vertex or a zero extent.                 */
/* ------------------------------------------------------------------------ */
int or_quantise(const float *xyz, uint64_t nverts, int32_t *q, float *bbox_min, double *scale)
{
    if (nverts == 0) return 1;
    float mn[3], mx[3];
    for (int a = 0; a < 3; a++) { mn[a] = xyz[a]; mx[a] = xyz[a]; }
    for (uint64_t i = 0; i < nverts; i++)
        for (int a = 0; a < 3; a++) {
            float x = xyz[3 * i + a];
            if (!isfinite(x)) return 1;
            if (x < mn[a]) mn[a] = x;
            if (x > mx[a]) mx[a] = x;
        }
    double E = 0.0;
    for (int a = 0; a < 3; a++) {
        double e = (double)mx[a] - (double)mn[a];
        if (e > E) E = e;
    }
    if (!(E > 0.0)) return 1;
    /* a -0.0 minimum is reported as +0.0 (x + 0 turns -0 into +0; no q changes) */
    for (int a = 0; a < 3; a++) mn[a] = mn[a] + 0.0f;
    double S = 2097151.0 / E;
    for (uint64_t i = 0; i < nverts; i++)
        for (int a = 0; a < 3; a++) {
            double t = ((double)xyz[3 * i + a] - (double)mn[a]) * S;
            double f = floor(t);
            int64_t v = (int64_t)f;
            if (v < 0) v = 0;
            if (v > OR_Q) v = OR_Q;
            q[3 * i + a] = (int32_t)v;
        }
    for (int a = 0; a < 3; a++) bbox_min[a] = mn[a];
    *scale = S;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* View frame for an integer direction d (Sec. 3.1: orthographic views of    */
/* the node from outside, e.g. its bounding-box corners, toward its centre). */
/* The camera sits on the +d side looking along -d.  k = first axis with the */
/* smallest |d_k|; u = d x e_k, v = d x u; depth w = -(d . q) (smaller is    */
/* nearer).  frame[0..2] = u, frame[3..5] = v, frame[6..8] = d.              */
/* ------------------------------------------------------------------------ */
static void cross3(const int64_t a[3], const int64_t b[3], int64_t c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

void or_frame(const int8_t d8[3], int64_t frame[9])
{
    int64_t d[3] = {d8[0], d8[1], d8[2]};
    int k = 0;
    for (int a = 1; a < 3; a++)
        if (llabs(d[a]) < llabs(d[k])) k = a;
    int64_t e[3] = {0, 0, 0};
    e[k] = 1;
    int64_t u[3], v[3];
    cross3(d, e, u);
    cross3(d, u, v);
    for (int a = 0; a < 3; a++) { frame[a] = u[a]; frame[3 + a] = v[a]; frame[6 + a] = d[a]; }
}

/* Screen mapping of one direction: the projection of the quantisation cube   */
/* [0,Q]^3 onto u (resp. v) spans res pixels; vertices are snapped to 1/256   */
/* pixel by round-half-up.  Pixel px has its centre at 256*px + 128.          */
typedef struct {
    int64_t u[3], v[3], d[3];
    int64_t ulo, vlo, U1, V1; /* lower end and span+1 of u.q, v.q */
    int64_t wbias;            /* Q * sum(max(0, d_a)) so that w + wbias >= 0 */
    int64_t res;
} or_view;

static void make_view(const int8_t d8[3], int res, or_view *vw)
{
    int64_t f[9];
    or_frame(d8, f);
    int64_t ulo = 0, uspan = 0, vlo = 0, vspan = 0, wb = 0;
    for (int a = 0; a < 3; a++) {
        vw->u[a] = f[a]; vw->v[a] = f[3 + a]; vw->d[a] = f[6 + a];
        if (f[a] < 0) ulo += f[a] * OR_Q;
        uspan += llabs(f[a]) * OR_Q;
        if (f[3 + a] < 0) vlo += f[3 + a] * OR_Q;
        vspan += llabs(f[3 + a]) * OR_Q;
        if (f[6 + a] > 0) wb += f[6 + a] * OR_Q;
    }
    vw->ulo = ulo; vw->vlo = vlo; vw->U1 = uspan + 1; vw->V1 = vspan + 1;
    vw->wbias = wb; vw->res = res;
}

static void project(const or_view *vw, const int32_t *q, int64_t *X, int64_t *Y, int64_t *W)
{
    int64_t uq = 0, vq = 0, dq = 0;
    for (int a = 0; a < 3; a++) {
        uq += vw->u[a] * (int64_t)q[a];
        vq += vw->v[a] * (int64_t)q[a];
        dq += vw->d[a] * (int64_t)q[a];
    }
    *X = ((uq - vw->ulo) * vw->res * 512 + vw->U1) / (2 * vw->U1);
    *Y = ((vq - vw->vlo) * vw->res * 512 + vw->V1) / (2 * vw->V1);
    *W = -dq + vw->wbias;
}

/* Edge function of the directed edge a->b at p (positive on its left). */
static int64_t edge(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}
/* Tie rule for a sample exactly on an edge: the edge owns it when its       */
/* direction points down (dy<0) or, if horizontal, right (dx>0).  This equals */
/* sampling at p + eps*(1, eta), so a shared edge is covered exactly once.    */
static int owned(int64_t ax, int64_t ay, int64_t bx, int64_t by)
{
    int64_t dx = bx - ax, dy = by - ay;
    return dy < 0 || (dy == 0 && dx > 0);
}

typedef struct {
    int ok;                 /* 0: zero screen area, skipped */
    int idx[3];             /* vertex order after winding normalisation */
    int64_t x[3], y[3], w[3];
    int64_t area2;
} or_tri;

static void setup_tri(const or_view *vw, const int32_t *q, const uint32_t *t, or_tri *T)
{
    int64_t X[3], Y[3], W[3];
    for (int i = 0; i < 3; i++) project(vw, q + 3 * (uint64_t)t[i], &X[i], &Y[i], &W[i]);
    int64_t a2 = edge(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
    T->ok = a2 != 0;
    int o[3] = {0, 1, 2};
    if (a2 < 0) { o[1] = 2; o[2] = 1; a2 = -a2; }
    for (int i = 0; i < 3; i++) { T->idx[i] = o[i]; T->x[i] = X[o[i]]; T->y[i] = Y[o[i]]; T->w[i] = W[o[i]]; }
    T->area2 = a2;
}

/* Barycentric weights at pixel centre (px,py): returns 1 if covered. */
static int cover(const or_tri *T, int64_t px, int64_t py, int64_t lam[3])
{
    const int64_t *x = T->x, *y = T->y;
    int64_t sx = 256 * px + 128, sy = 256 * py + 128;
    lam[0] = edge(x[1], y[1], x[2], y[2], sx, sy);
    lam[1] = edge(x[2], y[2], x[0], y[0], sx, sy);
    lam[2] = edge(x[0], y[0], x[1], y[1], sx, sy);
    int in0 = lam[0] > 0 || (lam[0] == 0 && owned(x[1], y[1], x[2], y[2]));
    int in1 = lam[1] > 0 || (lam[1] == 0 && owned(x[2], y[2], x[0], y[0]));
    int in2 = lam[2] > 0 || (lam[2] == 0 && owned(x[0], y[0], x[1], y[1]));
    return in0 && in1 && in2;
}

static void pixel_range(int64_t lo, int64_t hi, int64_t res, int64_t *p0, int64_t *p1)
{
    /* pixels whose centre 256p+128 lies in [lo, hi] */
    *p0 = lo <= 128 ? 0 : (lo - 128 + 255) / 256;
    *p1 = hi < 128 ? -1 : (hi - 128) / 256;
    if (*p1 > res - 1) *p1 = res - 1;
}

/* Depth pass of one direction (Sec. 3.1's render into G-buffers, as an     */
/* integer rasteriser): every triangle, every pixel centre of its screen    */
/* bbox; covered fragments keep the minimum of (depth << 32 | triangle id). */
/* depth[res*res] is initialised to all ones.  frag (nullable) returns the  */
/* number of covered fragments before the depth test; cover_cnt (nullable,  */
/* res*res) counts them per pixel.                                         */
void or_raster_dir(const int32_t *q, uint64_t nverts, const uint32_t *tri, uint64_t ntris,
                   const int8_t d[3], int res, uint64_t *depth, uint64_t *frag, uint32_t *cover_cnt)
{
    (void)nverts;
    or_view vw;
    make_view(d, res, &vw);
    uint64_t nf = 0;
    for (uint64_t p = 0; p < (uint64_t)res * res; p++) depth[p] = ~(uint64_t)0;
    for (uint64_t t = 0; t < ntris; t++) {
        or_tri T;
        setup_tri(&vw, q, tri + 3 * t, &T);
        if (!T.ok) continue;
        int64_t xmin = T.x[0], xmax = T.x[0], ymin = T.y[0], ymax = T.y[0];
        for (int i = 1; i < 3; i++) {
            if (T.x[i] < xmin) xmin = T.x[i];
            if (T.x[i] > xmax) xmax = T.x[i];
            if (T.y[i] < ymin) ymin = T.y[i];
            if (T.y[i] > ymax) ymax = T.y[i];
        }
        int64_t px0, px1, py0, py1;
        pixel_range(xmin, xmax, res, &px0, &px1);
        pixel_range(ymin, ymax, res, &py0, &py1);
        for (int64_t py = py0; py <= py1; py++)
            for (int64_t px = px0; px <= px1; px++) {
                int64_t lam[3];
                if (!cover(&T, px, py, lam)) continue;
                uint64_t num = (uint64_t)lam[0] * (uint64_t)T.w[0] + (uint64_t)lam[1] * (uint64_t)T.w[1] +
                               (uint64_t)lam[2] * (uint64_t)T.w[2];
                uint64_t z = num / (uint64_t)T.area2;
                uint64_t key = (z << 32) | (uint64_t)t;
                uint64_t pix = (uint64_t)py * res + (uint64_t)px;
                if (key < depth[pix]) depth[pix] = key;
                nf++;
                if (cover_cnt) cover_cnt[pix]++;
            }
    }
    if (frag) *frag = nf;
}

/* One surfel candidate per covered pixel (Sec. 3.1, last paragraph). */
typedef struct {
    uint64_t morton;
    uint32_t e;
    uint32_t pad;
    uint64_t key;
    int16_t nrm[3];
    uint8_t rgb[3];
    uint8_t pad2;
} or_row;

static int row_cmp(const void *pa, const void *pb)
{
    const or_row *a = (const or_row *)pa, *b = (const or_row *)pb;
    if (a->morton != b->morton) return a->morton < b->morton ? -1 : 1;
    if (a->e != b->e) return a->e < b->e ? -1 : 1;
    return 0;
}

/* Resolve one pixel: position by integer barycentric interpolation of the   */
/* quantised vertices (floor), unit normal of the triangle turned toward the */
/* camera as snorm16 (round half to even of 32767*n/|n|), face colour.       */
static void resolve_pixel(const or_view *vw, const int32_t *q, const uint32_t *tri, const uint8_t *face_rgb,
                          uint32_t t, int64_t px, int64_t py, or_row *r)
{
    or_tri T;
    setup_tri(vw, q, tri + 3 * (uint64_t)t, &T);
    int64_t lam[3];
    cover(&T, px, py, lam);
    int64_t pos[3];
    for (int a = 0; a < 3; a++) {
        uint64_t num = 0;
        for (int i = 0; i < 3; i++) num += (uint64_t)lam[i] * (uint64_t)q[3 * (uint64_t)tri[3 * (uint64_t)t + T.idx[i]] + a];
        pos[a] = (int64_t)(num / (uint64_t)T.area2);
    }
    const int32_t *q0 = q + 3 * (uint64_t)tri[3 * (uint64_t)t + 0];
    const int32_t *q1 = q + 3 * (uint64_t)tri[3 * (uint64_t)t + 1];
    const int32_t *q2 = q + 3 * (uint64_t)tri[3 * (uint64_t)t + 2];
    int64_t e1[3], e2[3], n[3];
    for (int a = 0; a < 3; a++) { e1[a] = (int64_t)q1[a] - q0[a]; e2[a] = (int64_t)q2[a] - q0[a]; }
    cross3(e1, e2, n);
    int64_t nd = n[0] * vw->d[0] + n[1] * vw->d[1] + n[2] * vw->d[2];
    if (nd < 0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
    double s = (double)n[0] * (double)n[0] + (double)n[1] * (double)n[1];
    s = s + (double)n[2] * (double)n[2];
    if (s == 0.0) {
        r->nrm[0] = r->nrm[1] = r->nrm[2] = 0;
    } else {
        double len = sqrt(s);
        for (int a = 0; a < 3; a++) {
            double c = (32767.0 * (double)n[a]) / len;
            r->nrm[a] = (int16_t)rint(c);
        }
    }
    for (int a = 0; a < 3; a++) r->rgb[a] = face_rgb ? face_rgb[3 * (uint64_t)t + a] : 0;
    r->key = pack_key(pos[0], pos[1], pos[2]);
    r->morton = or_morton3((uint32_t)pos[0], (uint32_t)pos[1], (uint32_t)pos[2]);
}

/* Visible-surface sampling of a quantised mesh (Sec. 3.1): raster every      */
/* direction, emit one row per covered pixel with emission index              */
/* e = dir*res^2 + py*res + px, then sort rows by (Morton code, e) and keep   */
/* the first row of every distinct position.  Returns the surfel count N;     */
/* the arrays are written only when N <= cap.  Returns -1 on bad arguments,   */
/* -2 when out of memory.                                                     */
int64_t or_sample_visible(const int32_t *q, uint64_t nverts, const uint32_t *tri, uint64_t ntris,
                          const uint8_t *face_rgb, const int8_t *dirs, int ndirs, int res,
                          uint64_t *key, int16_t *nrm, uint8_t *rgb, uint32_t *src, uint64_t cap)
{
    if (res < 1 || res > 4096 || ndirs < 1) return -1;
    uint64_t npix = (uint64_t)res * res;
    uint64_t *depth = (uint64_t *)malloc(npix * sizeof(uint64_t));
    uint64_t rcap = 1024, nrow = 0;
    or_row *rows = (or_row *)malloc(rcap * sizeof(or_row));
    if (!depth || !rows) { free(depth); free(rows); return -2; }
    for (int di = 0; di < ndirs; di++) {
        const int8_t *d = dirs + 3 * di;
        if (d[0] == 0 && d[1] == 0 && d[2] == 0) { free(depth); free(rows); return -1; }
        or_raster_dir(q, nverts, tri, ntris, d, res, depth, NULL, NULL);
        or_view vw;
        make_view(d, res, &vw);
        for (int64_t py = 0; py < res; py++)
            for (int64_t px = 0; px < res; px++) {
                uint64_t v = depth[(uint64_t)py * res + px];
                if (v == ~(uint64_t)0) continue;
                if (nrow == rcap) {
                    rcap *= 2;
                    or_row *nr = (or_row *)realloc(rows, rcap * sizeof(or_row));
                    if (!nr) { free(depth); free(rows); return -2; }
                    rows = nr;
                }
                or_row *r = &rows[nrow++];
                memset(r, 0, sizeof(*r));
                resolve_pixel(&vw, q, tri, face_rgb, (uint32_t)(v & 0xFFFFFFFFu), px, py, r);
                r->e = (uint32_t)((uint64_t)di * npix + (uint64_t)py * res + (uint64_t)px);
            }
    }
    free(depth);
    qsort(rows, nrow, sizeof(or_row), row_cmp);
    uint64_t n = 0;
    for (uint64_t i = 0; i < nrow; i++) {
        if (i > 0 && rows[i].morton == rows[i - 1].morton) continue;
        if (n < cap) {
            key[n] = rows[i].key;
            for (int a = 0; a < 3; a++) { nrm[3 * n + a] = rows[i].nrm[a]; rgb[3 * n + a] = rows[i].rgb[a]; }
            src[n] = rows[i].e;
        }
        n++;
    }
    free(rows);
    return (int64_t)n;
}

/* ------------------------------------------------------------------------ */
/* Hierarchical generation from child surfels (Sec. 3.4: a parent node's      */
/* initial set may be rendered from its children's surfel approximations     */
/* instead of their triangles), with each surfel drawn as the oriented disc  */
/* of Sec. 4.2 (position, normal, radius).  Readings:                        */
/*  - a set of splats carries its own frame (bbox_min float32, scale double) */
/*    and one squared disc radius r2 in its own quantised units;            */
/*  - a splat centre moves to the parent frame by IEEE double operations in   */
/*    this order: t = q / s_child; t = bmin_child + t; t = t - fmin;          */
/*    t = t * s_parent; c = clamp(floor(t), 0, 2^21 - 1);                     */
/*  - the radius likewise: r = sqrt(r2) / s_child * s_parent (double);        */
/*    R2 = ceil(r * r), at most 3 (2^21 - 1)^2;                              */
/*  - views are the six axis directions; a pixel centre's ray hits the disc  */
/*    plane n.(p - c) = 0 (n = the splat's snorm16 normal turned toward the   */
/*    camera, nw = n.d > 0; discs seen edge-on, nw = 0, are skipped) and the  */
/*    pixel is covered when the hit point lies within R2 of c -- an exact    */
/*    integer test in units of 1/(2 res) of a pixel-centre step;             */
/*  - depth of the hit point = floor of the exact rational depth; the        */
/*    smallest (depth << 32 | global splat index) wins a pixel;              */
/*  - the emitted surfel is the hit point (floor per axis), the splat's       */
/*    turned normal and colour; emission index, duplicate merge and Morton   */
/*    order as for triangles.                                                 */
/* ------------------------------------------------------------------------ */
static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q--;
    return q;
}

typedef struct {
    int64_t c[3];  /* centre in the parent frame */
    int64_t R2;    /* squared radius in parent units */
} or_splat;

static void splat_to_parent(uint64_t key, const float bmin[3], double s_child, int64_t r2, const float fmin[3],
                            double s_parent, or_splat *o)
{
    int64_t q[3];
    unpack_key(key, q);
    for (int a = 0; a < 3; a++) {
        double t = (double)q[a] / s_child;
        t = (double)bmin[a] + t;
        t = t - (double)fmin[a];
        t = t * s_parent;
        double f = floor(t);
        int64_t v = f < 0.0 ? 0 : (f > (double)OR_Q ? OR_Q : (int64_t)f);
        o->c[a] = v;
    }
    const double rmax2 = 3.0 * (double)OR_Q * (double)OR_Q;
    double r = sqrt((double)r2) / s_child;
    r = r * s_parent;
    double rr = r * r;
    o->R2 = rr >= rmax2 ? (int64_t)rmax2 : (int64_t)ceil(rr);
}

/* Pixels of one axis direction covered by one splat, with their depth keys. */
static void splat_dir(const or_view *vw, const or_splat *sp, const int16_t n16[3], uint32_t g, uint64_t *depth)
{
    int64_t n[3] = {n16[0], n16[1], n16[2]};
    int64_t nu = 0, nv = 0, nw = 0, cu = 0, cv = 0, cd = 0;
    for (int a = 0; a < 3; a++) {
        nu += vw->u[a] * n[a]; nv += vw->v[a] * n[a]; nw += vw->d[a] * n[a];
        cu += vw->u[a] * sp->c[a]; cv += vw->v[a] * sp->c[a]; cd += vw->d[a] * sp->c[a];
    }
    if (nw == 0) return;
    if (nw < 0) { nu = -nu; nv = -nv; nw = -nw; }
    const int64_t res = vw->res, two_res = 2 * res;
    const int64_t cu2 = (cu - vw->ulo) * two_res, cv2 = (cv - vw->vlo) * two_res;
    const int64_t dc = -cd + vw->wbias;
    /* a covered pixel has DU^2 <= R2 (2 res)^2 (and the same for DV), so only  */
    /* the pixels with |DU|, |DV| <= 2 res Rb, Rb = ceil(sqrt(R2)), are tested  */
    int64_t Rb = (int64_t)sqrt((double)sp->R2);
    while (Rb * Rb < sp->R2) Rb++;
    int64_t px0 = -floor_div(-(cu2 - two_res * Rb - vw->U1), 2 * vw->U1), px1 = floor_div(cu2 + two_res * Rb - vw->U1, 2 * vw->U1);
    int64_t py0 = -floor_div(-(cv2 - two_res * Rb - vw->V1), 2 * vw->V1), py1 = floor_div(cv2 + two_res * Rb - vw->V1, 2 * vw->V1);
    if (px0 < 0) px0 = 0;
    if (py0 < 0) py0 = 0;
    if (px1 > res - 1) px1 = res - 1;
    if (py1 > res - 1) py1 = res - 1;
    for (int64_t py = py0; py <= py1; py++) {
        const int64_t DV = (2 * py + 1) * vw->V1 - cv2;
        for (int64_t px = px0; px <= px1; px++) {
            const int64_t DU = (2 * px + 1) * vw->U1 - cu2;
            __int128 lhs = ((__int128)DU * DU + (__int128)DV * DV) * ((__int128)nw * nw);
            const __int128 t = (__int128)nu * DU + (__int128)nv * DV;
            lhs += t * t;
            const __int128 rhs = (__int128)sp->R2 * ((__int128)two_res * two_res) * ((__int128)nw * nw);
            if (lhs > rhs) continue;
            int64_t z = floor_div(dc * nw * two_res + nu * DU + nv * DV, nw * two_res);
            if (z < 0) z = 0;
            if (z > 0xFFFFFFFFll) z = 0xFFFFFFFFll;
            const uint64_t v = ((uint64_t)z << 32) | g;
            uint64_t *dp = &depth[(uint64_t)py * res + px];
            if (v < *dp) *dp = v;
        }
    }
}

/* The surfel of a pixel won by splat sp: the hit point, the turned normal. */
static void splat_resolve(const or_view *vw, const or_splat *sp, const int16_t n16[3], const uint8_t *rgb3,
                          int64_t px, int64_t py, or_row *r)
{
    int64_t n[3] = {n16[0], n16[1], n16[2]};
    int64_t nu = 0, nv = 0, nw = 0, cu = 0, cv = 0;
    for (int a = 0; a < 3; a++) {
        nu += vw->u[a] * n[a]; nv += vw->v[a] * n[a]; nw += vw->d[a] * n[a];
        cu += vw->u[a] * sp->c[a]; cv += vw->v[a] * sp->c[a];
    }
    const int flip = nw < 0;
    if (flip) { nu = -nu; nv = -nv; nw = -nw; }
    const int64_t two_res = 2 * vw->res;
    const int64_t DU = (2 * px + 1) * vw->U1 - (cu - vw->ulo) * two_res;
    const int64_t DV = (2 * py + 1) * vw->V1 - (cv - vw->vlo) * two_res;
    /* hit point = c + u DU/(2res) + v DV/(2res) - d (nu DU + nv DV)/(nw 2res); */
    /* u, v, d are signed unit axis vectors, so each axis gets one term         */
    const int64_t W = nu * DU + nv * DV;
    int64_t pos[3];
    for (int a = 0; a < 3; a++) {
        int64_t p = sp->c[a];
        if (vw->u[a] != 0) p += floor_div(vw->u[a] * DU, two_res);
        if (vw->v[a] != 0) p += floor_div(vw->v[a] * DV, two_res);
        if (vw->d[a] != 0) p += floor_div(-vw->d[a] * W, nw * two_res);
        pos[a] = p < 0 ? 0 : (p > OR_Q ? OR_Q : p);
    }
    for (int a = 0; a < 3; a++) {
        r->nrm[a] = (int16_t)(flip ? -n16[a] : n16[a]);
        r->rgb[a] = rgb3 ? rgb3[a] : 0;
    }
    r->key = pack_key(pos[0], pos[1], pos[2]);
    r->morton = or_morton3((uint32_t)pos[0], (uint32_t)pos[1], (uint32_t)pos[2]);
}

/* Headless render of discs for one axis direction: depth[py * res + px] gets the   */
/* smallest (depth << 32 | global splat index) of the discs covering the pixel, or  */
/* all ones (the depth pass of or_sample_splats on its own).  Returns 0, or -1.      */
int or_render_splats(uint64_t nsplat, const uint64_t *skey, const int16_t *snrm, int nsets, const uint64_t *set_ofs,
                     const float *bmin, const double *scale, const int64_t *r2, const float fmin[3], double fscale,
                     const int8_t dir[3], int res, uint64_t *depth)
{
    if (res < 1 || res > 4096 || nsets < 0 || nsplat >= 0xFFFFFFFFull) return -1;
    if ((dir[0] != 0) + (dir[1] != 0) + (dir[2] != 0) != 1) return -1;
    if (set_ofs[0] != 0 || set_ofs[nsets] != nsplat) return -1;
    or_view vw;
    make_view(dir, res, &vw);
    for (uint64_t i = 0; i < (uint64_t)res * res; i++) depth[i] = ~(uint64_t)0;
    for (int i = 0; i < nsets; i++)
        for (uint64_t g = set_ofs[i]; g < set_ofs[i + 1]; g++) {
            or_splat sp;
            splat_to_parent(skey[g], bmin + 3 * i, scale[i], r2[i], fmin, fscale, &sp);
            splat_dir(&vw, &sp, snrm + 3 * g, (uint32_t)g, depth);
        }
    return 0;
}

/* Splat sampling of one parent node.  Splats are concatenated over nsets   */
/* sets; set i holds splats [set_ofs[i], set_ofs[i+1]) with frame bmin[3i..],  */
/* scale[i] and squared radius r2[i].  The parent frame is (fmin, fscale).    */
/* dirs must be axis directions.  Returns N as or_sample_visible does, -1 on  */
/* bad arguments, -2 when out of memory.                                     */
int64_t or_sample_splats(uint64_t nsplat, const uint64_t *skey, const int16_t *snrm, const uint8_t *srgb, int nsets,
                         const uint64_t *set_ofs, const float *bmin, const double *scale, const int64_t *r2,
                         const float fmin[3], double fscale, const int8_t *dirs, int ndirs, int res,
                         uint64_t *key, int16_t *nrm, uint8_t *rgb, uint32_t *src, uint64_t cap)
{
    if (res < 1 || res > 4096 || ndirs < 1 || nsets < 0 || nsplat >= 0xFFFFFFFFull) return -1;
    if (set_ofs[0] != 0 || set_ofs[nsets] != nsplat) return -1;
    for (int di = 0; di < ndirs; di++) {
        const int8_t *d = dirs + 3 * di;
        const int nz = (d[0] != 0) + (d[1] != 0) + (d[2] != 0);
        if (nz != 1) return -1;
    }
    or_splat *sp = (or_splat *)malloc((nsplat ? nsplat : 1) * sizeof(or_splat));
    const uint64_t npix = (uint64_t)res * res;
    uint64_t *depth = (uint64_t *)malloc(npix * sizeof(uint64_t));
    uint64_t rcap = 1024, nrow = 0;
    or_row *rows = (or_row *)malloc(rcap * sizeof(or_row));
    if (!sp || !depth || !rows) { free(sp); free(depth); free(rows); return -2; }
    for (int i = 0; i < nsets; i++)
        for (uint64_t g = set_ofs[i]; g < set_ofs[i + 1]; g++)
            splat_to_parent(skey[g], bmin + 3 * i, scale[i], r2[i], fmin, fscale, &sp[g]);
    for (int di = 0; di < ndirs; di++) {
        or_view vw;
        make_view(dirs + 3 * di, res, &vw);
        for (uint64_t i = 0; i < npix; i++) depth[i] = ~(uint64_t)0;
        for (uint64_t g = 0; g < nsplat; g++) splat_dir(&vw, &sp[g], snrm + 3 * g, (uint32_t)g, depth);
        for (int64_t py = 0; py < res; py++)
            for (int64_t px = 0; px < res; px++) {
                const uint64_t v = depth[(uint64_t)py * res + px];
                if (v == ~(uint64_t)0) continue;
                if (nrow == rcap) {
                    rcap *= 2;
                    or_row *nr = (or_row *)realloc(rows, rcap * sizeof(or_row));
                    if (!nr) { free(sp); free(depth); free(rows); return -2; }
                    rows = nr;
                }
                or_row *r = &rows[nrow++];
                memset(r, 0, sizeof(*r));
                const uint32_t g = (uint32_t)(v & 0xFFFFFFFFu);
                splat_resolve(&vw, &sp[g], snrm + 3 * (uint64_t)g, srgb ? srgb + 3 * (uint64_t)g : NULL, px, py, r);
                r->e = (uint32_t)((uint64_t)di * npix + (uint64_t)py * res + (uint64_t)px);
            }
    }
    free(sp);
    free(depth);
    qsort(rows, nrow, sizeof(or_row), row_cmp);
    uint64_t n = 0;
    for (uint64_t i = 0; i < nrow; i++) {
        if (i > 0 && rows[i].morton == rows[i - 1].morton) continue;
        if (n < cap) {
            key[n] = rows[i].key;
            for (int a = 0; a < 3; a++) { nrm[3 * n + a] = rows[i].nrm[a]; rgb[3 * n + a] = rows[i].rgb[a]; }
            src[n] = rows[i].e;
        }
        n++;
    }
    free(rows);
    return (int64_t)n;
}

/* ------------------------------------------------------------------------ */
/* Progressive ordering: the exact greedy permutation (farthest-first        */
/* traversal) that Sec. 3.2 sets as the goal and Sec. 3.3 uses as the quality */
/* reference.  perm[0] = s; for k >= 1, perm[k] is the unchosen point whose   */
/* squared distance to the nearest chosen point is largest, ties to the       */
/* lowest index; rad2[k] is that squared distance; rad2[0] = INT64_MAX.       */
/* The loop keeps D[i] = min over chosen j of |q_i - q_j|^2, and each step    */
/* does an O(N) argmax followed by an O(N) min-update (O(N^2) in total).      */
/* ------------------------------------------------------------------------ */

/* Start index (Sec. 3.2: a random starting surfel): start >= 0 is taken as  */
/* given; otherwise x = Philox4x32-10(ctr={part_id,0,0,0}, key={seed_lo,     */
/* seed_hi}) word 0 and s = (x * N) >> 32.  Returns 0, or 1 if start >= N.    */
int or_start_index(uint64_t n, uint64_t seed, uint32_t part_id, int64_t start, uint64_t *out)
{
    if (n == 0) return 1;
    if (start >= 0) {
        if ((uint64_t)start >= n) return 1;
        *out = (uint64_t)start;
        return 0;
    }
    uint32_t ctr[4] = {part_id, 0, 0, 0};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    *out = (uint64_t)(((unsigned __int128)r[0] * n) >> 32);
    return 0;
}

static int64_t d2key(uint64_t a, uint64_t b)
{
    int64_t p[3], r[3];
    unpack_key(a, p);
    unpack_key(b, r);
    int64_t dx = p[0] - r[0], dy = p[1] - r[1], dz = p[2] - r[2];
    return dx * dx + dy * dy + dz * dz;
}

/* Orders the first m = (max_count ? min(max_count, n) : n) entries.  visits */
/* (nullable) returns N + sum over steps k>=1 of the number of unchosen      */
/* points strictly inside the ball of squared radius rad2[k] around the new  */
/* point (what a spatially pruned update must examine); improved (nullable)  */
/* returns how many D[i] the updates lowered.  Returns 0, or 1 on bad input. */
int or_greedy(const uint64_t *key, uint64_t n, uint64_t s, uint64_t max_count, uint32_t *perm, int64_t *rad2,
              uint64_t *visits, uint64_t *improved, int nthreads)
{
    if (n == 0 || s >= n) return 1;
    uint64_t m = (max_count == 0 || max_count > n) ? n : max_count;
    int64_t *D = (int64_t *)malloc(n * sizeof(int64_t));
    uint8_t *chosen = (uint8_t *)calloc(n, 1);
    if (!D || !chosen) { free(D); free(chosen); return 1; }
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#else
    (void)nthreads;
#endif
    uint64_t vis = n, imp = 0;
    perm[0] = (uint32_t)s;
    rad2[0] = INT64_MAX;
    chosen[s] = 1;
    for (uint64_t i = 0; i < n; i++) D[i] = d2key(key[i], key[s]);
    for (uint64_t k = 1; k < m; k++) {
        /* argmax over unchosen of (D[i], -i) */
        int64_t bestD = -1;
        uint64_t besti = n;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            int64_t lD = -1;
            uint64_t li = n;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
            for (uint64_t i = 0; i < n; i++)
                if (!chosen[i] && D[i] > lD) { lD = D[i]; li = i; }
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (li < n && (lD > bestD || (lD == bestD && li < besti))) { bestD = lD; besti = li; }
            }
        }
        uint64_t j = besti;
        perm[k] = (uint32_t)j;
        rad2[k] = bestD;
        chosen[j] = 1;
        /* min-update of every unchosen point against the new point */
        uint64_t vk = 0, ik = 0;
        const int64_t R = bestD;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(+ : vk, ik)
#endif
        for (uint64_t i = 0; i < n; i++) {
            if (chosen[i]) continue;
            int64_t d = d2key(key[i], key[j]);
            if (d < R) vk++;
            if (d < D[i]) { D[i] = d; ik++; }
        }
        vis += vk;
        imp += ik;
    }
    free(D);
    free(chosen);
    if (visits) *visits = vis;
    if (improved) *improved = imp;
    return 0;
}

/* Per-prefix splat radius in the part's world units: sqrt(rad2)/S with IEEE */
/* double sqrt and divide, rounded to float; +inf for the first entry.       */
void or_radius(const int64_t *rad2, uint64_t m, double scale, float *radius)
{
    for (uint64_t k = 0; k < m; k++) {
        if (rad2[k] == INT64_MAX) { radius[k] = INFINITY; continue; }
        if (rad2[k] < 0) { radius[k] = NAN; continue; }
        double r = sqrt((double)rad2[k]) / scale;
        radius[k] = (float)r;
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* The paper's randomised progressive sampling (Sec. 3.2): start from a random */
/* surfel; each round draw a random subset of the remaining input set, append */
/* the candidate(s) farthest from every surfel chosen before the round, and   */
/* remove them; after every `step` rounds one more candidate is taken per     */
/* round (the speed-up heuristic of Sec. 3.2); stop at max_count or when the  */
/* input set is empty.  Vicinity removal is not used (no threshold is given). */
/* Reading of the unstated details:                                          */
/*  - remaining set: array R of indices, removal by swap with the last entry; */
/*    picks are removed in the order they are appended;                      */
/*  - round t draws sample_size positions with replacement, position u is    */
/*    (w * |R|) >> 32 with w = word 0 of Philox4x32-10(ctr = {part_id, t, u, */
/*    1}, key = {seed_lo, seed_hi}); sample_size = 0 takes the whole set;     */
/*  - the round takes the m_t = 1 + t / step (step = 0: 1) distinct sampled  */
/*    points with the largest distance to the chosen set, ties to the lowest */
/*    index, in that order; distances are not refreshed inside a round;     */
/*  - rad2 of a pick is its squared distance to every earlier pick.          */
/* ------------------------------------------------------------------------ */
int or_sampled(const uint64_t *key, uint64_t n, uint64_t s, uint64_t max_count, uint64_t seed, uint32_t part_id,
               uint32_t sample_size, uint32_t step, uint32_t *perm, int64_t *rad2, uint32_t *round_of)
{
    if (n == 0 || s >= n) return 1;
    uint64_t m = (max_count == 0 || max_count > n) ? n : max_count;
    int64_t *D = (int64_t *)malloc(n * sizeof(int64_t));
    uint32_t *R = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *pos = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *cand = (uint32_t *)malloc((sample_size ? sample_size : n) * sizeof(uint32_t));
    uint8_t *mark = (uint8_t *)calloc(n, 1);
    if (!D || !R || !pos || !cand || !mark) { free(D); free(R); free(pos); free(cand); free(mark); return 1; }
    uint64_t L = n;
    for (uint64_t i = 0; i < n; i++) { R[i] = (uint32_t)i; pos[i] = (uint32_t)i; }
    /* remove x from the remaining set */
#define OR_REMOVE(x)                                   \
    do {                                               \
        uint32_t p_ = pos[(x)], y_ = R[L - 1];         \
        R[p_] = y_;                                    \
        pos[y_] = p_;                                  \
        L--;                                           \
    } while (0)
    perm[0] = (uint32_t)s;
    rad2[0] = INT64_MAX;
    if (round_of) round_of[0] = 0;
    OR_REMOVE((uint32_t)s);
    for (uint64_t i = 0; i < n; i++) D[i] = d2key(key[i], key[s]);
    uint64_t out = 1;
    uint32_t seed_key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t t = 0; out < m && L > 0; t++) {
        /* the round's random subset of the remaining set */
        uint64_t nc = 0;
        if (sample_size == 0) {
            for (uint64_t u = 0; u < L; u++) cand[nc++] = R[u];
        } else {
            for (uint32_t u = 0; u < sample_size; u++) {
                uint32_t ctr[4] = {part_id, t, u, 1u}, w[4];
                or_philox4x32_10(ctr, seed_key, w);
                uint64_t p = ((uint64_t)w[0] * L) >> 32;
                uint32_t c = R[p];
                if (!mark[c]) { mark[c] = 1; cand[nc++] = c; }
            }
            for (uint64_t u = 0; u < nc; u++) mark[cand[u]] = 0;
        }
        uint64_t mt = 1 + (step ? t / step : 0);
        uint64_t first = out;
        /* the mt candidates farthest from the surfels chosen before this round */
        for (uint64_t r = 0; r < mt && out < m && r < nc; r++) {
            uint64_t best = nc;
            for (uint64_t u = 0; u < nc; u++) {
                uint32_t c = cand[u];
                if (mark[c]) continue;
                if (best == nc || D[c] > D[cand[best]] || (D[c] == D[cand[best]] && c < cand[best])) best = u;
            }
            uint32_t c = cand[best];
            mark[c] = 1;
            int64_t r2 = D[c];
            for (uint64_t q = first; q < out; q++) {
                int64_t d = d2key(key[c], key[perm[q]]);
                if (d < r2) r2 = d;
            }
            perm[out] = c;
            rad2[out] = r2;
            if (round_of) round_of[out] = t;
            out++;
        }
        for (uint64_t q = first; q < out; q++) {
            mark[perm[q]] = 0;
            OR_REMOVE(perm[q]);
        }
        /* distances of every point to the chosen set */
        for (uint64_t q = first; q < out; q++) {
            uint64_t j = perm[q];
            for (uint64_t i = 0; i < n; i++) {
                int64_t d = d2key(key[i], key[j]);
                if (d < D[i]) D[i] = d;
            }
        }
    }
#undef OR_REMOVE
    free(D); free(R); free(pos); free(cand); free(mark);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Prefix selection (Sec. 4.1).                                              */
/* r_m: the median of the nearest-neighbour distances inside the first pm    */
/* surfels of an ordering (the lower median, the ceil(pm/2)-th smallest      */
/* squared distance; 0 for pm < 2).                                          */
/* Exact prefix for a radius: prefix p (entries 0..p-1) reaches every point  */
/* within sqrt(rad2[p]); the shortest prefix whose reach is at most r is     */
/* the smallest p >= 1 with rad2[p] <= r^2, or m if no ordered entry has it. */
/* ------------------------------------------------------------------------ */
static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int64_t or_prefix_median_nn(const uint64_t *key, const uint32_t *perm, uint64_t pm)
{
    if (pm < 2) return 0;
    int64_t *nn = (int64_t *)malloc(pm * sizeof(int64_t));
    if (!nn) return -1;
    for (uint64_t a = 0; a < pm; a++) {
        int64_t best = INT64_MAX;
        for (uint64_t b = 0; b < pm; b++) {
            if (a == b) continue;
            int64_t d = d2key(key[perm[a]], key[perm[b]]);
            if (d < best) best = d;
        }
        nn[a] = best;
    }
    qsort(nn, pm, sizeof(int64_t), cmp_i64);
    int64_t r = nn[(pm + 1) / 2 - 1];
    free(nn);
    return r;
}

uint64_t or_prefix_for_radius(const int64_t *rad2, uint64_t m, int64_t r2)
{
    for (uint64_t p = 1; p < m; p++)
        if (rad2[p] <= r2) return p;
    return m;
}

/* ------------------------------------------------------------------------ */
/* Bottom-up generation (Sec. 3.4) with the prefix rule of Sec. 4.1: the     */
/* frame a parent node is sampled in, and the child prefix it draws.         */
/* Reading (the paper leaves both open):                                     */
/*  - child c's quantisation cube is [m_c, m_c + Q / s_c] on every axis     */
/*    (bbox minimum m_c, float32; scale s_c, double; Q = 2^21 - 1);          */
/*  - the parent frame's minimum is the per-axis smallest m_c (a float32,   */
/*    so it is one of the children's own corners) and its scale maps the    */
/*    largest child cube extent from that minimum, max over c and axes of   */
/*    (m_c + Q / s_c) - min, onto Q: S = Q / extent (IEEE double, in this   */
/*    order);                                                               */
/*  - a child is drawn with the shortest prefix of its ordering that        */
/*    reaches every child surfel within one pixel step of the parent's      */
/*    raster: 2^21 / res parent units = (2^21 / res) * (s_c / S) child      */
/*    units; the target is the square of that, truncated to an integer.    */
/* ------------------------------------------------------------------------ */
int or_parent_frame(const float *mins, const double *scales, uint64_t nchildren, float *frame_min,
                    double *frame_scale)
{
    if (nchildren == 0) return 1;
    for (int a = 0; a < 3; a++) {
        float lo = mins[a];
        for (uint64_t c = 1; c < nchildren; c++)
            if (mins[3 * c + a] < lo) lo = mins[3 * c + a];
        frame_min[a] = lo;
    }
    double ext = 0.0;
    for (uint64_t c = 0; c < nchildren; c++) {
        if (!(scales[c] > 0.0)) return 1;
        double side = (double)OR_Q / scales[c];
        for (int a = 0; a < 3; a++) {
            double hi = (double)mins[3 * c + a] + side;
            double e = hi - (double)frame_min[a];
            if (e > ext) ext = e;
        }
    }
    if (!(ext > 0.0)) return 1;
    *frame_scale = (double)OR_Q / ext;
    return 0;
}

int64_t or_child_target_r2(double child_scale, double parent_scale, int parent_res)
{
    double step = 2097152.0 / (double)parent_res;  /* one parent pixel, parent units */
    double h = step * (child_scale / parent_scale);  /* the same length, child units */
    return (int64_t)(h * h);
}
