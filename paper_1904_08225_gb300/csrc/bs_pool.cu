// bs_pool.cu -- the library's stream-ordered memory pool, one per device.
//
// Every scratch allocation of the library comes from this pool.  Unlike the device's
// default pool (which returns freed memory to the system at each synchronisation, so
// the next large call maps it again), this pool keeps up to `keep` bytes of freed
// memory for the next call (bs_set_tuning("pool_keep_mb", v); 64 GiB by default).
#include <atomic>
#include <mutex>

#include "bs_internal.cuh"

namespace bs {

// Failure injection for tests of the error paths (bs_set_tuning("fail_next_allocs", k)):
// the next k pool allocations fail as if the device were out of memory.  Host-side only.
static std::atomic<int> g_fail_allocs{0};

void pool_fail_next(int k) { g_fail_allocs.store(k < 0 ? 0 : k); }

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64];
static bool g_pool_made[64];
static uint64_t g_pool_keep = 64ull << 30;

static cudaMemPool_t current_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_made[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = g_pool_keep;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = p;
        g_pool_made[dev] = true;
    }
    return g_pool[dev];
}

cudaError_t pool_malloc_async(void **ptr, size_t bytes, cudaStream_t stream) {
    for (int left = g_fail_allocs.load(); left > 0; left = g_fail_allocs.load())
        if (g_fail_allocs.compare_exchange_weak(left, left - 1)) {
            *ptr = nullptr;
            return cudaErrorMemoryAllocation;
        }
    cudaMemPool_t p = current_pool();
    if (!p) return cudaMallocAsync(ptr, bytes, stream);
    return cudaMallocFromPoolAsync(ptr, bytes, p, stream);
}

void pool_set_keep(uint64_t bytes) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    g_pool_keep = bytes;
    for (int d = 0; d < 64; ++d)
        if (g_pool_made[d]) {
            uint64_t keep = bytes;
            cudaMemPoolSetAttribute(g_pool[d], cudaMemPoolAttrReleaseThreshold, &keep);
            cudaMemPoolTrimTo(g_pool[d], (size_t)bytes);
        }
}

}  // namespace bs
