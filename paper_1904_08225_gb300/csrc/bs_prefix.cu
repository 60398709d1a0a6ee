// bs_prefix.cu -- prefix selection at render time (Sec. 4.1): the median nearest-
// neighbour distance r_m inside the first p_m surfels of an ordering, and the shortest
// prefix whose surfels reach every point of the part within a radius.
#include <cmath>
#include <vector>

#include "bs_internal.cuh"

namespace bs {

// nn[a] = squared distance from prefix point a to its nearest other prefix point
__global__ void __launch_bounds__(256) k_prefix_nn(const uint64_t *__restrict__ key, const uint32_t *__restrict__ perm,
                                                   uint32_t pm, int64_t *__restrict__ nn) {
    __shared__ int64_t red[8];
    for (uint32_t a = blockIdx.x; a < pm; a += gridDim.x) {
        const uint64_t qa = key[perm[a]];
        int64_t best = INT64_MAX;
        for (uint32_t b = threadIdx.x; b < pm; b += blockDim.x)
            if (b != a) best = min(best, dist2(qa, key[perm[b]]));
        const uint32_t hi = __reduce_min_sync(0xffffffffu, (uint32_t)((uint64_t)best >> 32));
        const uint32_t lo = __reduce_min_sync(0xffffffffu, (uint32_t)((uint64_t)best >> 32) == hi ? (uint32_t)best : 0xffffffffu);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (int64_t)(((uint64_t)hi << 32) | lo);
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t v = red[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = min(v, red[w]);
            nn[a] = v;
        }
        __syncthreads();
    }
}

// the (rank+1)-th smallest of v[0..n) (values in [0, 2^62)), by a bitwise radix select in one block
__global__ void __launch_bounds__(1024) k_select(const int64_t *__restrict__ v, uint32_t n, uint32_t rank,
                                                 int64_t *__restrict__ out) {
    __shared__ uint32_t red[32];
    uint64_t prefix = 0;
    uint32_t k = rank;
    for (int bit = 61; bit >= 0; --bit) {
        const uint64_t himask = bit == 61 ? 0ull : (~0ull << (bit + 1));
        uint32_t c = 0;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t x = (uint64_t)v[i];
            c += ((x & himask) == (prefix & himask) && ((x >> bit) & 1ull) == 0) ? 1u : 0u;
        }
        c = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        uint32_t total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += red[w];
        __syncthreads();
        if (k >= total) {
            k -= total;
            prefix |= 1ull << bit;
        }
    }
    if (threadIdx.x == 0) *out = (int64_t)prefix;
}

// count of k in [1, m) with rad2[k] > r2
__global__ void k_count_above(const int64_t *__restrict__ rad2, uint64_t m, int64_t r2,
                              unsigned long long *__restrict__ count) {
    uint32_t c = 0;
    for (uint64_t k = 1 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m; k += (uint64_t)gridDim.x * blockDim.x)
        c += rad2[k] > r2 ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

bs_status prefix_median_nn(const bs_surfels *s, const uint32_t *perm, uint64_t pm, int64_t *rm2, cudaStream_t stream) {
    if (!s || !s->key || !perm || !rm2) { set_error("bs_prefix_median_nn: NULL argument"); return BS_EINVAL; }
    if (pm > s->n || pm > 65536) { set_error("bs_prefix_median_nn: pm=%llu exceeds n or 65536", (unsigned long long)pm); return BS_EINVAL; }
    if (pm < 2) { *rm2 = 0; return BS_OK; }
    int64_t *buf = nullptr;
    cudaError_t e = pool_malloc_async((void **)&buf, (pm + 1) * sizeof(int64_t), stream);
    if (e != cudaSuccess) { cudaGetLastError(); set_error("bs_prefix_median_nn: scratch allocation failed"); return BS_ENOMEM; }
    k_prefix_nn<<<(unsigned)std::min<uint64_t>(pm, 4096), 256, 0, stream>>>(s->key, perm, (uint32_t)pm, buf);
    k_select<<<1, 1024, 0, stream>>>(buf, (uint32_t)pm, (uint32_t)((pm + 1) / 2 - 1), buf + pm);
    int64_t h = 0;
    e = cudaMemcpyAsync(&h, buf + pm, 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(buf, stream);
    if (e != cudaSuccess) { set_error("bs_prefix_median_nn: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    *rm2 = h;
    return BS_OK;
}

bs_status prefix_for_radius(const int64_t *rad2, uint64_t m, int64_t r2, uint64_t *p, cudaStream_t stream) {
    if (!rad2 || !p || m == 0) { set_error("bs_prefix_for_radius: NULL argument or m = 0"); return BS_EINVAL; }
    if (r2 < 0) { set_error("bs_prefix_for_radius: negative squared radius"); return BS_EINVAL; }
    unsigned long long *cnt = nullptr;
    cudaError_t e = pool_malloc_async((void **)&cnt, 8, stream);
    if (e != cudaSuccess) { cudaGetLastError(); set_error("bs_prefix_for_radius: scratch allocation failed"); return BS_ENOMEM; }
    unsigned long long h = 0;
    e = cudaMemsetAsync(cnt, 0, 8, stream);
    if (e == cudaSuccess && m > 1) {
        k_count_above<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 1216), 256, 0, stream>>>(rad2, m, r2, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(cnt, stream);
    if (e != cudaSuccess) { set_error("bs_prefix_for_radius: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    // rad2[1..m) does not increase: the entries above r2 are exactly [1, 1 + h)
    *p = std::min<uint64_t>(1 + h, m);
    return BS_OK;
}

// thread per part: binary search of the first k in [1, m) with rad2[k] <= r2 (rad2[1..m)
// does not increase), m when none
__global__ void k_prefix_batched(const int64_t *const *__restrict__ rad2, const uint64_t *__restrict__ m,
                                 const int64_t *__restrict__ r2, int nparts, uint64_t *__restrict__ p,
                                 int64_t *__restrict__ r2_at) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nparts) return;
    const int64_t *r = rad2[i];
    const uint64_t mi = m[i];
    uint64_t lo = 1, hi = mi;
    for (int it = 0; it < 64 && lo < hi; ++it) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (r[mid] <= r2[i]) hi = mid;
        else lo = mid + 1;
    }
    const uint64_t pi = lo < mi ? lo : mi;
    p[i] = pi;
    r2_at[i] = r[pi < mi ? pi : mi - 1];
}

bs_status prefix_for_radius_batched(const int64_t *const *rad2, const uint64_t *m, const int64_t *r2, int nparts,
                                    uint64_t *p, int64_t *r2_at, cudaStream_t stream) {
    if (nparts < 0 || (nparts > 0 && (!rad2 || !m || !r2 || !p))) {
        set_error("bs_prefix_for_radius_batched: NULL argument");
        return BS_EINVAL;
    }
    for (int i = 0; i < nparts; ++i)
        if (!rad2[i] || m[i] == 0 || r2[i] < 0) {
            set_error("bs_prefix_for_radius_batched: part %d: NULL rad2, m = 0 or negative r2", i);
            return BS_EINVAL;
        }
    if (nparts == 0) return BS_OK;
    const size_t n = (size_t)nparts;
    char *buf = nullptr;
    const size_t bytes = n * (8 + 8 + 8 + 8 + 8);
    cudaError_t e = pool_malloc_async((void **)&buf, bytes, stream);
    if (e != cudaSuccess) { cudaGetLastError(); set_error("bs_prefix_for_radius_batched: scratch allocation failed"); return BS_ENOMEM; }
    const int64_t **d_rad2 = (const int64_t **)buf;
    uint64_t *d_m = (uint64_t *)(buf + 8 * n);
    int64_t *d_r2 = (int64_t *)(buf + 16 * n);
    uint64_t *d_p = (uint64_t *)(buf + 24 * n);
    int64_t *d_at = (int64_t *)(buf + 32 * n);
    std::vector<int64_t> at(n);
    e = cudaMemcpyAsync(d_rad2, rad2, 8 * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_m, m, 8 * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_r2, r2, 8 * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        k_prefix_batched<<<(nparts + 255) / 256, 256, 0, stream>>>(d_rad2, d_m, d_r2, nparts, d_p, d_at);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, d_p, 8 * n, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(at.data(), d_at, 8 * n, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(buf, stream);
    if (e != cudaSuccess) { set_error("bs_prefix_for_radius_batched: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    if (r2_at)
        for (size_t i = 0; i < n; ++i) r2_at[i] = at[i];
    return BS_OK;
}

// Parent frames and child prefix targets of the bottom-up generation (Sec. 3.4 with the
// prefix rule of Sec. 4.1).  Host arithmetic on a handful of numbers per node: IEEE
// double operations in the stated order (the library's host code is compiled without
// floating-point contraction).
bs_status parent_frames(const float *child_min, const double *child_scale, const uint64_t *child_ofs, int nparents,
                        const int32_t *parent_res, float *frame_min, double *frame_scale, int64_t *child_r2) {
    if (nparents < 0 || (nparents > 0 && (!child_min || !child_scale || !child_ofs || !parent_res || !frame_min ||
                                          !frame_scale || !child_r2))) {
        set_error("bs_parent_frames: NULL argument or negative count");
        return BS_EINVAL;
    }
    const double Qd = (double)QMAX;
    for (int k = 0; k < nparents; ++k) {
        const uint64_t c0 = child_ofs[k], c1 = child_ofs[k + 1];
        if (c1 <= c0) { set_error("bs_parent_frames: parent %d has no children", k); return BS_EINVAL; }
        if (parent_res[k] < 1 || parent_res[k] > BS_MAX_RES) {
            set_error("bs_parent_frames: parent %d: resolution %d outside 1..%d", k, parent_res[k], BS_MAX_RES);
            return BS_EINVAL;
        }
        float lo[3] = {child_min[3 * c0], child_min[3 * c0 + 1], child_min[3 * c0 + 2]};
        for (uint64_t c = c0; c < c1; ++c) {
            const double s = child_scale[c];
            if (!(s > 0.0) || !std::isfinite(s)) { set_error("bs_parent_frames: child %llu: bad scale", (unsigned long long)c); return BS_EINVAL; }
            for (int a = 0; a < 3; ++a) {
                const float m = child_min[3 * c + a];
                if (!std::isfinite(m)) { set_error("bs_parent_frames: child %llu: non-finite corner", (unsigned long long)c); return BS_EINVAL; }
                lo[a] = m < lo[a] ? m : lo[a];
            }
        }
        double ext = 0.0;
        for (uint64_t c = c0; c < c1; ++c) {
            const double side = Qd / child_scale[c];
            for (int a = 0; a < 3; ++a) {
                const double hi = (double)child_min[3 * c + a] + side;
                const double e = hi - (double)lo[a];
                ext = e > ext ? e : ext;
            }
        }
        if (!(ext > 0.0) || !std::isfinite(ext)) { set_error("bs_parent_frames: parent %d: zero extent", k); return BS_EINVAL; }
        const double S = Qd / ext;
        for (int a = 0; a < 3; ++a) frame_min[3 * k + a] = lo[a];
        frame_scale[k] = S;
        const double step = 2097152.0 / (double)parent_res[k];
        for (uint64_t c = c0; c < c1; ++c) {
            const double h = step * (child_scale[c] / S);
            child_r2[c] = (int64_t)(h * h);
        }
    }
    return BS_OK;
}

}  // namespace bs
