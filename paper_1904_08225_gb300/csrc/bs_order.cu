// bs_order.cu -- progressive ordering (Sec. 3.2): the exact greedy permutation
// (farthest-first traversal) of each part's quantised surfel positions, with the
// per-prefix squared radius that makes every prefix an r-net (Sec. 4.1).
//
// Data layout per part (points in the caller's order, normally ascending Morton
// code, so consecutive points are spatially close):
//   D[i]      int64  squared distance of point i to the nearest chosen point; -1 once chosen
//   bucket b  = points [32b, 32b+32)   (one warp)   : bkey, bq, blo, bhi in global memory
//   group  g  = buckets [32g, 32g+32)  (1024 points): gkey, gq, glo, ghi in shared memory
// A record's key packs (D+1) above the complement of the local index of its best
// point, so one unsigned max gives the largest D with ties to the lowest index:
//   bkey = (D+1) << 5  | (31 - i_in_bucket)
//   gkey = (D+1) << 10 | (1023 - i_in_group)
//   top  = (D+1) << 13 | (8191 - g)
// bq / gq hold the packed position of that best point; blo/bhi and glo/ghi the
// bounding box of the points (fixed), used to skip records that cannot change:
// a point's D can only drop if |q_i - q_j|^2 < D_i <= record max, so a record
// with box_dist2(box, q_j) >= record max is left alone.
//
// Kernels:
//   k_order_init  one warp per group over all parts: D from the start point,
//                 bucket and group records.                       (HBM/L2 sweep)
//   k_order_loop  persistent, one CTA per part at a time (parts taken from an
//                 atomic counter): per step a block argmax over the group records,
//                 a scan of group boxes against the new point, and a warp per
//                 touched group updating its touched buckets.     (the update sweep)
//   k_radius      radius[k] = sqrt(rad2[k]) / scale in IEEE double, as float.
#include <algorithm>
#include <mutex>
#include <vector>

#include "bs_internal.cuh"

namespace bs {

constexpr uint32_t FULL = 0xffffffffu;
constexpr int MAX_GROUPS = 6144;  // BS_MAX_POINTS / 1024

__global__ void __launch_bounds__(256) k_order_init(const PartDesc *__restrict__ parts, const uint32_t *__restrict__ gofs,
                                                    int nparts, uint32_t total_groups) {
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= total_groups) return;
    const int lane = threadIdx.x & 31;
    int lo = 0, hi = nparts - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gofs[mid] <= gw) lo = mid; else hi = mid - 1;
    }
    const PartDesc P = parts[lo];
    const uint32_t g = gw - gofs[lo];
    const uint64_t qs = P.key[P.start];
    uint64_t gk = 0, gqv = 0;
    uint32_t glx = 0xffffffffu, gly = 0xffffffffu, glz = 0xffffffffu, ghx = 0, ghy = 0, ghz = 0;
    for (int b = 0; b < 32; ++b) {
        const uint32_t bucket = g * 32 + b;
        if (bucket >= P.nb) break;
        const uint32_t i = bucket * 32 + lane;
        const bool valid = i < P.n;
        const uint64_t k = valid ? P.key[i] : 0ull;
        int64_t d = -1;
        if (valid) {
            d = i == P.start ? -1 : dist2(k, qs);
            P.D[i] = d;
        }
        const uint64_t nk = valid ? (((uint64_t)(d + 1) << 5) | (uint64_t)(31 - lane)) : 0ull;
        const uint64_t bk = warp_max_u64(nk);
        const uint64_t bqv = __shfl_sync(FULL, k, 31 - (int)(bk & 31));
        const uint32_t lx = __reduce_min_sync(FULL, valid ? pos_x(k) : 0xffffffffu);
        const uint32_t ly = __reduce_min_sync(FULL, valid ? pos_y(k) : 0xffffffffu);
        const uint32_t lz = __reduce_min_sync(FULL, valid ? pos_z(k) : 0xffffffffu);
        const uint32_t hx = __reduce_max_sync(FULL, valid ? pos_x(k) : 0u);
        const uint32_t hy = __reduce_max_sync(FULL, valid ? pos_y(k) : 0u);
        const uint32_t hz = __reduce_max_sync(FULL, valid ? pos_z(k) : 0u);
        if (lane == 0) {
            P.bkey[bucket] = bk;
            P.bq[bucket] = bqv;
            P.blo[bucket] = pack_pos(lx, ly, lz);
            P.bhi[bucket] = pack_pos(hx, hy, hz);
        }
        const uint64_t cand = ((bk >> 5) << 10) | (uint64_t)(1023 - (b * 32 + (31 - (int)(bk & 31))));
        if (cand > gk) { gk = cand; gqv = bqv; }
        glx = min(glx, lx); gly = min(gly, ly); glz = min(glz, lz);
        ghx = max(ghx, hx); ghy = max(ghy, hy); ghz = max(ghz, hz);
    }
    if (lane == 0) {
        P.gkey[g] = gk;
        P.gq[g] = gqv;
        P.glo[g] = pack_pos(glx, gly, glz);
        P.ghi[g] = pack_pos(ghx, ghy, ghz);
    }
}

template <int T>
__global__ void __launch_bounds__(T) k_order_loop(const PartDesc *__restrict__ parts, int nparts,
                                                  uint32_t *__restrict__ next_part, int ngmax) {
    extern __shared__ uint64_t sm[];
    uint64_t *s_gkey = sm;
    uint64_t *s_gq = sm + ngmax;
    uint64_t *s_glo = sm + 2 * ngmax;
    uint64_t *s_ghi = sm + 3 * ngmax;
    uint32_t *s_list = (uint32_t *)(sm + 4 * ngmax);
    constexpr int NW = T / 32;
    __shared__ uint64_t s_red[NW];
    __shared__ uint32_t s_cnt, s_part;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_part = atomicAdd(next_part, 1u);
        __syncthreads();
        const uint32_t p = s_part;
        if (p >= (uint32_t)nparts) break;
        const PartDesc P = parts[p];
        for (uint32_t g = threadIdx.x; g < P.ng; g += T) {
            s_gkey[g] = P.gkey[g];
            s_gq[g] = P.gq[g];
            s_glo[g] = P.glo[g];
            s_ghi[g] = P.ghi[g];
        }
        if (threadIdx.x == 0) {
            P.perm[0] = P.start;
            P.rad2[0] = INT64_MAX;
            s_cnt = 0;
        }
        __syncthreads();
        for (uint32_t k = 1; k < P.m; ++k) {
            // A: argmax over group records
            uint64_t best = 0;
            for (uint32_t g = threadIdx.x; g < P.ng; g += T)
                best = max(best, ((s_gkey[g] >> 10) << 13) | (uint64_t)(8191 - g));
            best = warp_max_u64(best);
            if (lane == 0) s_red[warp] = best;
            __syncthreads();
            best = warp_max_u64(lane < NW ? s_red[lane] : 0ull);
            const uint32_t gj = 8191u - (uint32_t)(best & 8191u);
            const uint64_t gkj = s_gkey[gj];
            const uint32_t j = gj * 1024u + (1023u - (uint32_t)(gkj & 1023u));
            const int64_t Dj = (int64_t)(best >> 13) - 1;
            const uint64_t qj = s_gq[gj];
            if (threadIdx.x == 0) {
                P.perm[k] = j;
                P.rad2[k] = Dj;
            }
            // B: groups whose box can hold a point the new point moves closer
            for (uint32_t g = threadIdx.x; g < P.ng; g += T) {
                const int64_t gD = (int64_t)(s_gkey[g] >> 10) - 1;
                if (g == gj || box_dist2(s_glo[g], s_ghi[g], qj) < gD) s_list[atomicAdd(&s_cnt, 1u)] = g;
            }
            __syncthreads();
            // C: one warp per listed group; lane b owns bucket b of the group
            const uint32_t cnt = s_cnt;
            const uint32_t bj = j >> 5;
            for (uint32_t li = warp; li < cnt; li += NW) {
                const uint32_t g = s_list[li];
                const uint32_t b = g * 32 + lane;
                const bool vb = b < P.nb;
                uint64_t bk = vb ? P.bkey[b] : 0ull;
                uint64_t bqv = vb ? P.bq[b] : 0ull;
                const uint64_t blo = vb ? P.blo[b] : 0ull, bhi = vb ? P.bhi[b] : 0ull;
                const int64_t bD = (int64_t)(bk >> 5) - 1;
                const bool aff = vb && (b == bj || box_dist2(blo, bhi, qj) < bD);
                uint32_t mask = __ballot_sync(FULL, aff);
                while (mask) {
                    const int bb = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const uint32_t i = (g * 32 + bb) * 32 + lane;
                    const bool valid = i < P.n;
                    const uint64_t ki = valid ? P.key[i] : 0ull;
                    int64_t d = valid ? P.D[i] : -1;
                    if (d >= 0) {
                        if (i == j) {
                            d = -1;
                            P.D[i] = -1;
                        } else {
                            const int64_t dd = dist2(ki, qj);
                            if (dd < d) {
                                d = dd;
                                P.D[i] = dd;
                            }
                        }
                    }
                    const uint64_t nk = valid ? (((uint64_t)(d + 1) << 5) | (uint64_t)(31 - lane)) : 0ull;
                    const uint64_t nbk = warp_max_u64(nk);
                    const uint64_t nq = __shfl_sync(FULL, ki, 31 - (int)(nbk & 31));
                    if (lane == bb) { bk = nbk; bqv = nq; }
                }
                if (aff) { P.bkey[b] = bk; P.bq[b] = bqv; }
                const uint64_t cand = vb ? (((bk >> 5) << 10) | (uint64_t)(1023 - (lane * 32 + (31 - (int)(bk & 31))))) : 0ull;
                const uint64_t ngk = warp_max_u64(cand);
                const uint64_t ngq = __shfl_sync(FULL, bqv, (int)((1023u - (uint32_t)(ngk & 1023u)) >> 5));
                if (lane == 0) { s_gkey[g] = ngk; s_gq[g] = ngq; }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_cnt = 0;
        }
        __syncthreads();
    }
}

__global__ void k_radius(const PartDesc *__restrict__ parts, int nparts) {
    for (int p = blockIdx.y; p < nparts; p += gridDim.y) {
        const PartDesc P = parts[p];
        if (!P.radius) continue;
        for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < P.m; k += gridDim.x * blockDim.x) {
            const int64_t r2 = P.rad2[k];
            P.radius[k] = r2 == INT64_MAX ? __int_as_float(0x7f800000) : (float)__ddiv_rn(__dsqrt_rn((double)r2), P.scale);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct LoopCfg {
    int threads;
    int grid;
};

static int g_loop_threads_override = 0;   // set by bs_set_tuning("order_threads", v)
static int g_ctas_per_sm_override = 0;    // set by bs_set_tuning("order_ctas_per_sm", v)

void order_set_tuning(int threads, int ctas_per_sm) {
    g_loop_threads_override = threads;
    g_ctas_per_sm_override = ctas_per_sm;
}

// Optional per-kernel timing: events recorded on the launch stream around one kernel.
static bool g_kernel_timing = false;
static cudaEvent_t g_ev[3][2];
static bool g_ev_made = false, g_ev_used[3] = {false, false, false};
static int g_ev_device = -1;

void order_set_kernel_timing(bool on) { g_kernel_timing = on; }

static void timing_mark(int which, int edge, cudaStream_t stream) {
    if (!g_kernel_timing) return;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!g_ev_made || g_ev_device != dev) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 2; ++j) cudaEventCreate(&g_ev[i][j]);
        g_ev_made = true;
        g_ev_device = dev;
    }
    cudaEventRecord(g_ev[which][edge], stream);
    if (edge == 1) g_ev_used[which] = true;
}

bs_status order_last_launch_ms(int which, double *ms) {
    if (which < 0 || which > 2 || !g_ev_made || !g_ev_used[which]) return BS_ENOTREADY;
    if (cudaEventSynchronize(g_ev[which][1]) != cudaSuccess) return BS_ECUDA;
    float f = 0.f;
    if (cudaEventElapsedTime(&f, g_ev[which][0], g_ev[which][1]) != cudaSuccess) return BS_ECUDA;
    *ms = f;
    return BS_OK;
}

template <int T>
static cudaError_t launch_loop(const PartDesc *d_parts, int nparts, uint32_t *d_next, int ngmax, int grid,
                               cudaStream_t stream) {
    const size_t smem = (size_t)ngmax * 36;
    cudaError_t e = cudaFuncSetAttribute(k_order_loop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_order_loop<T><<<grid, T, smem, stream>>>(d_parts, nparts, d_next, ngmax);
    return cudaGetLastError();
}

template <int T>
static int occupancy(int ngmax) {
    int blocks = 0;
    const size_t smem = (size_t)ngmax * 36;
    cudaFuncSetAttribute(k_order_loop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_order_loop<T>, T, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(blocks, 1);
}

static int pick_threads(int ngmax, bool batched) {
    if (g_loop_threads_override) return g_loop_threads_override;
    if (batched) return ngmax > 256 ? 256 : 128;
    if (ngmax <= 32) return 128;
    if (ngmax <= 512) return 256;
    return 512;
}

// Orders nparts parts.  host descriptors: keys, outputs, n, m, start, scale filled in.
bs_status order_parts(std::vector<PartDesc> &hp, cudaStream_t stream, bool batched) {
    const int nparts = (int)hp.size();
    if (nparts == 0) return BS_OK;
    // LPT: largest parts first so the persistent CTAs finish together
    std::vector<int> order(nparts);
    for (int i = 0; i < nparts; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hp[a].n > hp[b].n; });
    size_t total = 0;
    uint32_t ngmax = 1, total_groups = 0;
    for (auto &p : hp) {
        p.nb = (p.n + 31) / 32;
        p.ng = (p.nb + 31) / 32;
        ngmax = std::max(ngmax, p.ng);
        total += align_up((size_t)p.n * 8) + 4 * align_up((size_t)p.nb * 8) + 4 * align_up((size_t)p.ng * 8);
        if (!p.rad2) total += align_up((size_t)p.m * 8);
    }
    const size_t desc_bytes = align_up((size_t)nparts * sizeof(PartDesc));
    const size_t gofs_bytes = align_up((size_t)nparts * 4);
    total += desc_bytes + gofs_bytes + 256;
    char *ws = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&ws, total, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("bs_order: scratch allocation of %zu bytes failed: %s", total, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? BS_ENOMEM : BS_ECUDA;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { char *p = ws + off; off += align_up(bytes); return p; };
    PartDesc *d_parts = (PartDesc *)take((size_t)nparts * sizeof(PartDesc));
    uint32_t *d_gofs = (uint32_t *)take((size_t)nparts * 4);
    uint32_t *d_next = (uint32_t *)take(256);
    std::vector<PartDesc> sorted(nparts);
    std::vector<uint32_t> gofs(nparts);
    for (int r = 0; r < nparts; ++r) {
        PartDesc p = hp[order[r]];
        p.D = (int64_t *)take((size_t)p.n * 8);
        p.bkey = (uint64_t *)take((size_t)p.nb * 8);
        p.bq = (uint64_t *)take((size_t)p.nb * 8);
        p.blo = (uint64_t *)take((size_t)p.nb * 8);
        p.bhi = (uint64_t *)take((size_t)p.nb * 8);
        p.gkey = (uint64_t *)take((size_t)p.ng * 8);
        p.gq = (uint64_t *)take((size_t)p.ng * 8);
        p.glo = (uint64_t *)take((size_t)p.ng * 8);
        p.ghi = (uint64_t *)take((size_t)p.ng * 8);
        if (!p.rad2) p.rad2 = (int64_t *)take((size_t)p.m * 8);
        gofs[r] = total_groups;
        total_groups += p.ng;
        sorted[r] = p;
    }
    bs_status rc = BS_OK;
    do {
        if (cudaMemcpyAsync(d_parts, sorted.data(), (size_t)nparts * sizeof(PartDesc), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_gofs, gofs.data(), (size_t)nparts * 4, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemsetAsync(d_next, 0, 4, stream) != cudaSuccess) {
            set_error("bs_order: descriptor upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = BS_ECUDA;
            break;
        }
        const uint32_t init_blocks = (total_groups + 7) / 8;
        timing_mark(0, 0, stream);
        k_order_init<<<init_blocks, 256, 0, stream>>>(d_parts, d_gofs, nparts, total_groups);
        timing_mark(0, 1, stream);
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int T = pick_threads((int)ngmax, batched);
        int per_sm = 1;
        switch (T) {
            case 64: per_sm = occupancy<64>(ngmax); break;
            case 128: per_sm = occupancy<128>(ngmax); break;
            case 256: per_sm = occupancy<256>(ngmax); break;
            case 512: per_sm = occupancy<512>(ngmax); break;
            default: per_sm = occupancy<1024>(ngmax); break;
        }
        if (g_ctas_per_sm_override) per_sm = std::min(per_sm, g_ctas_per_sm_override);
        const int grid = std::max(1, std::min(nparts, sms * per_sm));
        timing_mark(1, 0, stream);
        switch (T) {
            case 64: e = launch_loop<64>(d_parts, nparts, d_next, ngmax, grid, stream); break;
            case 128: e = launch_loop<128>(d_parts, nparts, d_next, ngmax, grid, stream); break;
            case 256: e = launch_loop<256>(d_parts, nparts, d_next, ngmax, grid, stream); break;
            case 512: e = launch_loop<512>(d_parts, nparts, d_next, ngmax, grid, stream); break;
            default: e = launch_loop<1024>(d_parts, nparts, d_next, ngmax, grid, stream); break;
        }
        timing_mark(1, 1, stream);
        if (e != cudaSuccess) {
            set_error("bs_order: loop launch failed: %s", cudaGetErrorString(e));
            rc = BS_ECUDA;
            break;
        }
        bool any_radius = false;
        uint32_t mmax = 0;
        for (auto &p : sorted) { any_radius |= p.radius != nullptr; mmax = std::max(mmax, p.m); }
        if (any_radius) {
            dim3 g(std::min<uint32_t>((mmax + 255) / 256, 64), std::min(nparts, 65535));
            timing_mark(2, 0, stream);
            k_radius<<<g, 256, 0, stream>>>(d_parts, nparts);
            timing_mark(2, 1, stream);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("bs_order: launch failed: %s", cudaGetErrorString(e));
            rc = BS_ECUDA;
        }
    } while (0);
    cudaFreeAsync(ws, stream);
    return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the single-part ordering.
//
// Some callers cannot allocate device memory while they run: a plugin or render
// thread inside a host application that owns the GPU memory budget, or a
// real-time loop where cudaMalloc / a stream-ordered pool growth may block or fail.
// bs_order_noalloc serves them: the caller passes keys and outputs as usual and all
// ordering scratch (distance array, bucket and group records, descriptor, part
// counter, and rad2 when the caller passes none) lives in the fixed device array
// below, which every GPU that loads the library holds until process exit.
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t NOALLOC_MAX_POINTS = BS_NOALLOC_MAX_POINTS;
constexpr uint32_t NOALLOC_MAX_BUCKETS = NOALLOC_MAX_POINTS / 32;
constexpr uint32_t NOALLOC_MAX_GROUPS = (NOALLOC_MAX_BUCKETS + 31) / 32;
constexpr size_t NA_DESC = 0;                                               // PartDesc
constexpr size_t NA_NEXT = 256;                                             // part counter
constexpr size_t NA_D = 512;                                                // int64 D[n]
constexpr size_t NA_RAD2 = NA_D + 8ull * NOALLOC_MAX_POINTS;                // int64 rad2[m]
constexpr size_t NA_BUCKETS = NA_RAD2 + 8ull * NOALLOC_MAX_POINTS;          // 4 x u64 [nb]
constexpr size_t NA_GROUPS = NA_BUCKETS + 4 * 8ull * NOALLOC_MAX_BUCKETS;   // 4 x u64 [ng]
constexpr size_t NA_BYTES = NA_GROUPS + 4 * 8ull * NOALLOC_MAX_GROUPS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_noalloc_mu;
char *g_noalloc_addr[64] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
bs_status noalloc_scratch(char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error("bs_order_noalloc: cudaGetDevice: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    if (dev < 0 || dev >= 64) { set_error("bs_order_noalloc: device %d out of range", dev); return BS_EINVAL; }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("bs_order_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return BS_ECUDA;
        }
        g_noalloc_addr[dev] = (char *)p;
    }
    *out = g_noalloc_addr[dev];
    return BS_OK;
}

}  // namespace

bs_status order_part_noalloc(PartDesc p, cudaStream_t stream) {
    if (p.n > NOALLOC_MAX_POINTS) {
        set_error("bs_order_noalloc: n=%u exceeds the fixed scratch limit of %u points", p.n, NOALLOC_MAX_POINTS);
        return BS_EOVERFLOW;
    }
    char *base = nullptr;
    bs_status st = noalloc_scratch(&base);
    if (st != BS_OK) return st;
    p.nb = (p.n + 31) / 32;
    p.ng = (p.nb + 31) / 32;
    p.D = (int64_t *)(base + NA_D);
    if (!p.rad2) p.rad2 = (int64_t *)(base + NA_RAD2);
    uint64_t *bk = (uint64_t *)(base + NA_BUCKETS);
    p.bkey = bk;
    p.bq = bk + NOALLOC_MAX_BUCKETS;
    p.blo = bk + 2 * NOALLOC_MAX_BUCKETS;
    p.bhi = bk + 3 * NOALLOC_MAX_BUCKETS;
    uint64_t *gk = (uint64_t *)(base + NA_GROUPS);
    p.gkey = gk;
    p.gq = gk + NOALLOC_MAX_GROUPS;
    p.glo = gk + 2 * NOALLOC_MAX_GROUPS;
    p.ghi = gk + 3 * NOALLOC_MAX_GROUPS;
    PartDesc *d_desc = (PartDesc *)(base + NA_DESC);
    uint32_t *d_next = (uint32_t *)(base + NA_NEXT);
    cudaError_t e = cudaMemcpyAsync(d_desc, &p, sizeof(PartDesc), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_next, 0, 8, stream);  // d_next[0] counter, d_next[1] = gofs[0] = 0
    if (e != cudaSuccess) { set_error("bs_order_noalloc: descriptor upload failed: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    k_order_init<<<(p.ng + 7) / 8, 256, 0, stream>>>(d_desc, d_next + 1, 1, p.ng);
    const int T = pick_threads((int)p.ng, false);
    switch (T) {
        case 64: e = launch_loop<64>(d_desc, 1, d_next, (int)p.ng, 1, stream); break;
        case 128: e = launch_loop<128>(d_desc, 1, d_next, (int)p.ng, 1, stream); break;
        case 256: e = launch_loop<256>(d_desc, 1, d_next, (int)p.ng, 1, stream); break;
        case 512: e = launch_loop<512>(d_desc, 1, d_next, (int)p.ng, 1, stream); break;
        default: e = launch_loop<1024>(d_desc, 1, d_next, (int)p.ng, 1, stream); break;
    }
    if (e == cudaSuccess && p.radius) {
        k_radius<<<dim3(std::min<uint32_t>((p.m + 255) / 256, 64), 1), 256, 0, stream>>>(d_desc, 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { set_error("bs_order_noalloc: launch failed: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    return BS_OK;
}

}  // namespace bs
