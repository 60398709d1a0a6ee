// bs_internal.cuh -- shared pieces of the libbs CUDA implementation (sm_103a).
//
// Everything here is device/host plumbing for the kernels in bs_sample.cu,
// bs_order.cu and bs_server.cu: error reporting, the packed-position helpers,
// Philox4x32-10 and a few warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bs.h"

namespace bs {

// ---- error reporting (thread-local message behind bs_last_error) ----
void set_error(const char *fmt, ...);
void clear_error();

#define BS_CUDA_TRY(expr)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            bs::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return BS_ECUDA;                                                                     \
        }                                                                                        \
    } while (0)

#define BS_CHECK_LAUNCH()                                                                        \
    do {                                                                                         \
        cudaError_t e_ = cudaGetLastError();                                                     \
        if (e_ != cudaSuccess) {                                                                 \
            bs::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return BS_ECUDA;                                                                     \
        }                                                                                        \
    } while (0)

constexpr int64_t QMAX = 2097151;  // 2^21 - 1

// ---- packed quantised positions: x << 42 | y << 21 | z ----
__host__ __device__ __forceinline__ uint64_t pack_pos(uint64_t x, uint64_t y, uint64_t z) {
    return (x << 42) | (y << 21) | z;
}
__host__ __device__ __forceinline__ uint32_t pos_x(uint64_t k) { return (uint32_t)(k >> 42) & 0x1FFFFFu; }
__host__ __device__ __forceinline__ uint32_t pos_y(uint64_t k) { return (uint32_t)(k >> 21) & 0x1FFFFFu; }
__host__ __device__ __forceinline__ uint32_t pos_z(uint64_t k) { return (uint32_t)k & 0x1FFFFFu; }

// Squared distance of two packed positions (< 3 * 2^42, exact in int64).  The
// coordinate differences fit 22 bits, so each square is one 32x32->64 multiply.
__host__ __device__ __forceinline__ int64_t dist2(uint64_t a, uint64_t b) {
    const int32_t dx = (int32_t)pos_x(a) - (int32_t)pos_x(b);
    const int32_t dy = (int32_t)pos_y(a) - (int32_t)pos_y(b);
    const int32_t dz = (int32_t)pos_z(a) - (int32_t)pos_z(b);
    return (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
}

// Squared distance from q to the box [lo, hi] (packed corners), 0 inside.
__host__ __device__ __forceinline__ int64_t box_dist2(uint64_t lo, uint64_t hi, uint64_t q) {
    const int32_t cx = (int32_t)pos_x(q), cy = (int32_t)pos_y(q), cz = (int32_t)pos_z(q);
    const int32_t dx = max(max((int32_t)pos_x(lo) - cx, cx - (int32_t)pos_x(hi)), 0);
    const int32_t dy = max(max((int32_t)pos_y(lo) - cy, cy - (int32_t)pos_y(hi)), 0);
    const int32_t dz = max(max((int32_t)pos_z(lo) - cz, cz - (int32_t)pos_z(hi)), 0);
    return (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
}

// Spread the low 21 bits of v to every third bit (Morton interleave helper).
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1FFFFFull;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}
// Morton code: bit 3i = x_i, 3i+1 = y_i, 3i+2 = z_i.
__host__ __device__ __forceinline__ uint64_t morton_of(uint64_t key) {
    return spread3(pos_x(key)) | (spread3(pos_y(key)) << 1) | (spread3(pos_z(key)) << 2);
}

// ---- Philox4x32-10 (Salmon et al., SC'11), host and device ----
__host__ __device__ __forceinline__ void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                                       uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t a = (uint64_t)0xD2511F53u * c0;
        const uint64_t b = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)b;
        c3 = (uint32_t)a;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Starting index of a part: Philox word 0 scaled to [0, n) by multiply-shift.
inline uint64_t start_from_seed(uint64_t n, uint64_t seed, uint32_t part_id) {
    const uint32_t ctr[4] = {part_id, 0u, 0u, 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    philox4x32_10(ctr, key, r);
    return ((uint64_t)r[0] * n) >> 32;
}

// ---- one part of an ordering launch (device pointers; scratch carved by order_parts) ----
struct PartDesc {
    const uint64_t *key;
    uint32_t *perm;
    int64_t *rad2;
    float *radius;
    int64_t *D;
    uint64_t *bkey, *bq, *blo, *bhi;
    uint64_t *gkey, *gq, *glo, *ghi;
    uint32_t *R, *pos;  // variant 1: remaining set (index array) and each index's position in it
    uint32_t *done;     // optional completion flag (device view of host-mapped memory), set to 1 at the end
    double scale;
    uint64_t seed;
    uint32_t n, m, start, nb, ng;
    uint32_t variant, sample_size, sample_step, part_id;
};

}  // namespace bs

#include <algorithm>
#include <cstring>
#include <vector>

namespace bs {

// throughput: several parts of a launch share SMs as quarters of CTAs even when the
// launch is small (the server's launches), instead of one whole CTA per part
bs_status order_parts(std::vector<PartDesc> &parts, cudaStream_t stream, bool batched, bool throughput = false);
bs_status order_part_noalloc(PartDesc part, cudaStream_t stream);
bs_status prefix_median_nn(const bs_surfels *s, const uint32_t *perm, uint64_t pm, int64_t *rm2, cudaStream_t stream);
bs_status prefix_for_radius_batched(const int64_t *const *rad2, const uint64_t *m, const int64_t *r2, int nparts,
                                    uint64_t *p, int64_t *r2_at, cudaStream_t stream);
bs_status prefix_for_radius(const int64_t *rad2, uint64_t m, int64_t r2, uint64_t *p, cudaStream_t stream);
bs_status parent_frames(const float *child_min, const double *child_scale, const uint64_t *child_ofs, int nparents,
                        const int32_t *parent_res, float *frame_min, double *frame_scale, int64_t *child_r2);
bs_status scene_generate(uint64_t seed, const uint64_t *part_ids, const int32_t *lines, const int32_t *slots, int nparts,
                         int nboxes, int ncyl, const float *size_table, const float *cos32, const float *sin32,
                         float dx, float dy, int local_indices, float *xyz, uint32_t *tri, uint8_t *rgb,
                         cudaStream_t stream);
void order_set_tuning(int threads, int ctas_per_sm);
void order_set_quarters(int v);
void order_set_full_parts(int k);
void order_set_slots(int v);
void order_set_cluster(int c, int min_points);
void order_set_kernel_timing(bool on);
void order_set_algo(int algo);
bs_status order_last_launch_ms(int which, double *ms);
bs_status sample_visible(const bs_mesh *mesh, const bs_dir *dirs, int ndirs, int res, bs_surfels *out,
                         cudaStream_t stream);
bs_status render_mesh(const bs_mesh *mesh, const bs_dir *dir, int res, unsigned long long *image, cudaStream_t stream);
bs_status render_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *node, const bs_dir *dir,
                        unsigned long long *image, cudaStream_t stream);
// the library's stream-ordered pool (freed with cudaFreeAsync)
cudaError_t pool_malloc_async(void **ptr, size_t bytes, cudaStream_t stream);
void pool_set_keep(uint64_t bytes);
void pool_fail_next(int k);
bs_status sample_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *nodes, int nnodes, const bs_dir *dirs,
                        int ndirs, bs_surfels *out, cudaStream_t stream);
// host meshes (on_device == 0) copied into one device block (*block, freed by the caller
// with cudaFreeAsync on stream); dev receives the meshes with device pointers
bs_status stage_meshes(const bs_mesh *in, int n, std::vector<bs_mesh> &dev, char **block, cudaStream_t stream);
bs_status sample_order_batched(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs, int ndirs,
                               const bs_order_opts *opts, bs_part_result *out, int out_on_device, cudaStream_t stream);
bs_status sample_visible_parts(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs, int ndirs,
                               bs_surfels *out, cudaStream_t stream, unsigned long long *image = nullptr);

// ---- warp reductions ----
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
    uint32_t hi = (uint32_t)(v >> 32);
    uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
    uint32_t lo = hi == mhi ? (uint32_t)v : 0u;
    uint32_t mlo = __reduce_max_sync(0xffffffffu, lo);
    return ((uint64_t)mhi << 32) | mlo;
}

}  // namespace bs
