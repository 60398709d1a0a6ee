// bs_scene.cu -- scene-scale driver support: CAD-like parts (boxes and cylinders)
// regenerated on the device from a seed, so a scene of production lines (Sec. 5's
// evaluation scene) is sampled and ordered node by node without ever holding all of
// its triangles.  The float32 recipe (operation order, tables, Philox counters) is
// fixed so that a host implementation can reproduce every vertex bit for bit:
//   w(part, prim, k) = Philox4x32-10(ctr = {part_lo, part_hi, prim, k}, key = seed);
//   u(x) = float(x >> 8) * 2^-24;  sizes = size_table[x >> 22];
//   box: h = s * 0.5, lo = c - h, mid = lo + h, hi = c + h; 6 faces of 2x2 quads;
//   cylinder: ring j = cos_table[j] * r + c, sin_table[j] * r + c; levels c -/+ L * 0.5;
//   placement: + (slot * dx, line * dy, 0).
#include "bs_internal.cuh"

namespace bs {

constexpr int BOX_V = 54, BOX_T = 48, CYL_V = 98, CYL_T = 192;

struct SceneTables {
    float size[1024];
    float cosv[32];
    float sinv[32];
};

struct ScenePart {
    uint64_t part;
    int32_t line, slot;
};

__device__ __forceinline__ float unit(uint32_t x) { return __fmul_rn((float)(x >> 8), 5.9604644775390625e-08f); }

__device__ __forceinline__ void words(uint64_t part, uint32_t prim, uint32_t k, uint64_t seed, uint32_t w[4]) {
    const uint32_t c[4] = {(uint32_t)part, (uint32_t)(part >> 32), prim, k};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    philox4x32_10(c, key, w);
}

__global__ void k_scene_generate(const ScenePart *__restrict__ parts, int nparts, uint64_t seed, int nb, int nc,
                                 const SceneTables *__restrict__ tab, float dx, float dy, int local_indices,
                                 float *__restrict__ xyz, uint32_t *__restrict__ tri, uint8_t *__restrict__ rgb) {
    const int prims = nb + nc;
    const uint64_t vper = (uint64_t)nb * BOX_V + (uint64_t)nc * CYL_V;
    const uint64_t tper = (uint64_t)nb * BOX_T + (uint64_t)nc * CYL_T;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < (uint64_t)nparts * prims;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const int q = (int)(g / prims), prim = (int)(g % prims);
        const ScenePart P = parts[q];
        const float off[3] = {__fmul_rn((float)P.slot, dx), __fmul_rn((float)P.line, dy), 0.0f};
        const bool box = prim < nb;
        const uint64_t v0 = q * vper + (box ? (uint64_t)prim * BOX_V : (uint64_t)nb * BOX_V + (uint64_t)(prim - nb) * CYL_V);
        const uint64_t t0 = q * tper + (box ? (uint64_t)prim * BOX_T : (uint64_t)nb * BOX_T + (uint64_t)(prim - nb) * CYL_T);
        // vertex index of the primitive's first vertex: within its part, or within the whole mesh
        const uint32_t vbase = (uint32_t)(local_indices ? v0 - q * vper : v0);
        uint32_t w0[4], w1[4], w2[4], w3[4];
        words(P.part, (uint32_t)prim, 0, seed, w0);
        words(P.part, (uint32_t)prim, 1, seed, w1);
        words(P.part, (uint32_t)prim, 2, seed, w2);
        if (box) {
            words(P.part, (uint32_t)prim, 3, seed, w3);
            float lvl[3][3];  // [level][axis]
            for (int a = 0; a < 3; ++a) {
                const float c = unit(w0[a]);
                const float h = __fmul_rn(tab->size[w1[a] >> 22], 0.5f);
                lvl[0][a] = __fsub_rn(c, h);
                lvl[1][a] = __fadd_rn(lvl[0][a], h);
                lvl[2][a] = __fadd_rn(c, h);
            }
            const int faces[6][4] = {{0, 0, 1, 2}, {0, 2, 2, 1}, {1, 0, 2, 0}, {1, 2, 0, 2}, {2, 0, 0, 1}, {2, 2, 1, 0}};
            const uint32_t cw[6] = {w2[0], w2[1], w2[2], w2[3], w3[0], w3[1]};
            for (int f = 0; f < 6; ++f) {
                const int ax = faces[f][0], lev = faces[f][1], ua = faces[f][2], va = faces[f][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        float v[3];
                        v[ax] = lvl[lev][ax];
                        v[ua] = lvl[i][ua];
                        v[va] = lvl[j][va];
                        const uint64_t vi = v0 + f * 9 + i * 3 + j;
                        for (int a = 0; a < 3; ++a) xyz[3 * vi + a] = __fadd_rn(v[a], off[a]);
                    }
                const uint32_t fb = vbase + f * 9;
                int t = 0;
                for (int I = 0; I < 2; ++I)
                    for (int J = 0; J < 2; ++J) {
                        const uint32_t a = fb + I * 3 + J, b = fb + (I + 1) * 3 + J, c = fb + (I + 1) * 3 + J + 1,
                                       d = fb + I * 3 + J + 1;
                        const uint64_t ti = t0 + f * 8 + t;
                        tri[3 * ti] = a; tri[3 * ti + 1] = b; tri[3 * ti + 2] = c;
                        tri[3 * ti + 3] = a; tri[3 * ti + 4] = c; tri[3 * ti + 5] = d;
                        t += 2;
                    }
                for (int t8 = 0; t8 < 8; ++t8) {
                    const uint64_t ti = t0 + f * 8 + t8;
                    rgb[3 * ti] = (uint8_t)(cw[f] & 255u);
                    rgb[3 * ti + 1] = (uint8_t)((cw[f] >> 8) & 255u);
                    rgb[3 * ti + 2] = (uint8_t)((cw[f] >> 16) & 255u);
                }
            }
        } else {
            const int axis = (int)(w0[0] % 3u), a1 = (axis + 1) % 3, a2 = (axis + 2) % 3;
            const float cc[3] = {unit(w0[1]), unit(w0[2]), unit(w0[3])};
            const float r = tab->size[w1[0] >> 22];
            const float hl = __fmul_rn(tab->size[w1[1] >> 22], 0.5f);
            const float lev[3] = {__fsub_rn(cc[axis], hl), cc[axis], __fadd_rn(cc[axis], hl)};
            for (int k = 0; k < 3; ++k)
                for (int j = 0; j < 32; ++j) {
                    float v[3];
                    v[a1] = __fadd_rn(__fmul_rn(tab->cosv[j], r), cc[a1]);
                    v[a2] = __fadd_rn(__fmul_rn(tab->sinv[j], r), cc[a2]);
                    v[axis] = lev[k];
                    const uint64_t vi = v0 + k * 32 + j;
                    for (int a = 0; a < 3; ++a) xyz[3 * vi + a] = __fadd_rn(v[a], off[a]);
                }
            for (int e = 0; e < 2; ++e) {
                float v[3];
                v[a1] = cc[a1];
                v[a2] = cc[a2];
                v[axis] = lev[e ? 2 : 0];
                const uint64_t vi = v0 + 96 + e;
                for (int a = 0; a < 3; ++a) xyz[3 * vi + a] = __fadd_rn(v[a], off[a]);
            }
            int t = 0;
            for (int I = 0; I < 2; ++I)
                for (int J = 0; J < 32; ++J) {
                    const int J1 = (J + 1) % 32;
                    const uint32_t a = vbase + I * 32 + J, b = vbase + (I + 1) * 32 + J, c = vbase + (I + 1) * 32 + J1,
                                   d = vbase + I * 32 + J1;
                    const uint64_t ti = t0 + t;
                    tri[3 * ti] = a; tri[3 * ti + 1] = b; tri[3 * ti + 2] = c;
                    tri[3 * ti + 3] = a; tri[3 * ti + 4] = c; tri[3 * ti + 5] = d;
                    t += 2;
                }
            for (int j = 0; j < 32; ++j) {
                const uint64_t ti = t0 + 128 + j;
                tri[3 * ti] = vbase + 96; tri[3 * ti + 1] = vbase + j; tri[3 * ti + 2] = vbase + (j + 1) % 32;
            }
            for (int j = 0; j < 32; ++j) {
                const uint64_t ti = t0 + 160 + j;
                tri[3 * ti] = vbase + 97; tri[3 * ti + 1] = vbase + 64 + (j + 1) % 32; tri[3 * ti + 2] = vbase + 64 + j;
            }
            for (int t2 = 0; t2 < CYL_T; ++t2) {
                const uint32_t c = t2 < 128 ? w2[0] : (t2 < 160 ? w2[1] : w2[2]);
                const uint64_t ti = t0 + t2;
                rgb[3 * ti] = (uint8_t)(c & 255u);
                rgb[3 * ti + 1] = (uint8_t)((c >> 8) & 255u);
                rgb[3 * ti + 2] = (uint8_t)((c >> 16) & 255u);
            }
        }
    }
}

bs_status scene_generate(uint64_t seed, const uint64_t *part_ids, const int32_t *lines, const int32_t *slots, int nparts,
                         int nboxes, int ncyl, const float *size_table, const float *cos32, const float *sin32,
                         float dx, float dy, int local_indices, float *xyz, uint32_t *tri, uint8_t *rgb,
                         cudaStream_t stream) {
    if (nparts < 0 || nboxes < 0 || ncyl < 0 || (nparts > 0 && (!part_ids || !lines || !slots || !xyz || !tri || !rgb)) ||
        !size_table || !cos32 || !sin32) {
        set_error("bs_scene_generate: bad arguments");
        return BS_EINVAL;
    }
    if (nboxes == 0 && ncyl == 0) { set_error("bs_scene_generate: a part needs at least one primitive"); return BS_EINVAL; }
    const uint64_t vper = (uint64_t)nboxes * BOX_V + (uint64_t)ncyl * CYL_V;
    if ((uint64_t)nparts * vper >= (1ull << 32)) { set_error("bs_scene_generate: more than 2^32 vertices"); return BS_EINVAL; }
    if (nparts == 0) return BS_OK;
    std::vector<ScenePart> hp((size_t)nparts);
    for (int i = 0; i < nparts; ++i) hp[(size_t)i] = ScenePart{part_ids[i], lines[i], slots[i]};
    SceneTables ht;
    memcpy(ht.size, size_table, sizeof(ht.size));
    memcpy(ht.cosv, cos32, sizeof(ht.cosv));
    memcpy(ht.sinv, sin32, sizeof(ht.sinv));
    char *buf = nullptr;
    const size_t bytes = sizeof(SceneTables) + 256 + (size_t)nparts * sizeof(ScenePart);
    cudaError_t e = pool_malloc_async((void **)&buf, bytes, stream);
    if (e != cudaSuccess) { cudaGetLastError(); set_error("bs_scene_generate: scratch allocation failed"); return BS_ENOMEM; }
    SceneTables *dt = (SceneTables *)buf;
    ScenePart *dp = (ScenePart *)(buf + ((sizeof(SceneTables) + 255) & ~(size_t)255));
    e = cudaMemcpyAsync(dt, &ht, sizeof(ht), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, hp.data(), (size_t)nparts * sizeof(ScenePart), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        const uint64_t work = (uint64_t)nparts * (uint64_t)(nboxes + ncyl);
        k_scene_generate<<<(unsigned)std::min<uint64_t>((work + 127) / 128, 152 * 64), 128, 0, stream>>>(
            dp, nparts, seed, nboxes, ncyl, dt, dx, dy, local_indices, xyz, tri, rgb);
        e = cudaGetLastError();
    }
    cudaFreeAsync(buf, stream);
    if (e != cudaSuccess) { set_error("bs_scene_generate: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    return BS_OK;
}

}  // namespace bs
