// bs_api.cu -- the extern "C" entry points of libbs (declared in include/bs.h):
// argument validation, start-index selection, and the serving loop.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bs_internal.cuh"

namespace bs {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

// Validates one part and fills a descriptor (device pointers from the caller).
static bs_status make_part(const bs_surfels *s, const bs_order_opts *opts, uint32_t *perm, int64_t *rad2,
                           float *radius, PartDesc &p) {
    if (!s || !opts) { set_error("bs_order: NULL argument"); return BS_EINVAL; }
    if (s->n == 0 || s->n > BS_MAX_POINTS) {
        set_error("bs_order: n=%llu outside [1, %u]", (unsigned long long)s->n, BS_MAX_POINTS);
        return s->n == 0 ? BS_EINVAL : BS_EOVERFLOW;
    }
    if (!s->key || !perm) { set_error("bs_order: NULL key or perm array"); return BS_EINVAL; }
    if (radius && !(s->scale > 0.0)) { set_error("bs_order: radius requested but scale <= 0"); return BS_EINVAL; }
    uint64_t start;
    if (opts->start >= 0) {
        if ((uint64_t)opts->start >= s->n) {
            set_error("bs_order: start %lld >= n %llu", (long long)opts->start, (unsigned long long)s->n);
            return BS_EINVAL;
        }
        start = (uint64_t)opts->start;
    } else {
        start = start_from_seed(s->n, opts->seed, opts->part_id);
    }
    const uint64_t m = (opts->max_count == 0 || opts->max_count > s->n) ? s->n : opts->max_count;
    if (opts->variant != 0 && opts->variant != 1) { set_error("bs_order: variant=%d not 0 or 1", opts->variant); return BS_EINVAL; }
    if (opts->variant == 1 && (opts->sample_size < 1 || opts->sample_size > 256)) {
        set_error("bs_order: sample_size=%u outside [1, 256]", opts->sample_size);
        return BS_EINVAL;
    }
    memset(&p, 0, sizeof(p));
    p.variant = (uint32_t)opts->variant;
    p.sample_size = opts->sample_size;
    p.sample_step = opts->sample_step;
    p.part_id = opts->part_id;
    p.seed = opts->seed;
    p.key = s->key;
    p.perm = perm;
    p.rad2 = rad2;
    p.radius = radius;
    p.scale = s->scale;
    p.n = (uint32_t)s->n;
    p.m = (uint32_t)m;
    p.start = (uint32_t)start;
    return BS_OK;
}

}  // namespace bs

using namespace bs;

namespace bs {
// launch slots of servers created from now on (bs_set_tuning("server_slots", v))
int g_server_slots = 16;
// request timeout of servers created from now on (bs_set_tuning("server_timeout_ms", v); 0 = none)
int g_server_timeout_ms = 0;
}  // namespace bs
using bs::g_server_slots;
using bs::g_server_timeout_ms;

extern "C" {

const char *bs_last_error(void) { return g_err; }

bs_status bs_set_tuning(const char *name, int value) {
    if (name && !strcmp(name, "server_timeout_ms")) {
        if (value < 0) { set_error("bs_set_tuning: server_timeout_ms=%d negative", value); return BS_EINVAL; }
        g_server_timeout_ms = value;
        return BS_OK;
    }
    if (name && !strcmp(name, "fail_next_allocs")) {
        if (value < 0) { set_error("bs_set_tuning: fail_next_allocs=%d negative", value); return BS_EINVAL; }
        pool_fail_next(value);
        return BS_OK;
    }
    if (name && !strcmp(name, "server_slots")) {
        if (value < 1 || value > 256) { set_error("bs_set_tuning: server_slots=%d outside [1, 256]", value); return BS_EINVAL; }
        g_server_slots = value;
        return BS_OK;
    }
    static int threads = 0, ctas = 0;
    if (!name) { set_error("bs_set_tuning: NULL name"); return BS_EINVAL; }
    if (!strcmp(name, "order_threads")) {
        if (value != 0 && value != 64 && value != 128 && value != 256 && value != 512 && value != 1024) {
            set_error("bs_set_tuning: order_threads=%d not in {0,64,128,256,512,1024}", value);
            return BS_EINVAL;
        }
        threads = value;
    } else if (!strcmp(name, "order_algo")) {
        if (value != 1 && value != 2) { set_error("bs_set_tuning: order_algo=%d not 1 or 2", value); return BS_EINVAL; }
        order_set_algo(value);
        return BS_OK;
    } else if (!strcmp(name, "kernel_timing")) {
        if (value != 0 && value != 1) { set_error("bs_set_tuning: kernel_timing=%d not 0 or 1", value); return BS_EINVAL; }
        order_set_kernel_timing(value == 1);
        return BS_OK;
    } else if (!strcmp(name, "pool_keep_mb")) {
        if (value < 0) { set_error("bs_set_tuning: pool_keep_mb=%d negative", value); return BS_EINVAL; }
        pool_set_keep((uint64_t)value << 20);
        return BS_OK;
    } else if (!strcmp(name, "order_quarters")) {
        if (value != 0 && value != 1 && value != 2) { set_error("bs_set_tuning: order_quarters=%d not 0, 1 or 2", value); return BS_EINVAL; }
        order_set_quarters(value);
        return BS_OK;
    } else if (!strcmp(name, "order_full_parts")) {
        if (value < 0) { set_error("bs_set_tuning: order_full_parts=%d negative", value); return BS_EINVAL; }
        order_set_full_parts(value);
        return BS_OK;
    } else if (!strcmp(name, "order_slots")) {
        if (value != 0 && value != 2 && value != 4 && value != 8) {
            set_error("bs_set_tuning: order_slots=%d not 0, 2, 4 or 8", value);
            return BS_EINVAL;
        }
        order_set_slots(value == 0 ? 4 : value);
        return BS_OK;
    } else if (!strcmp(name, "order_cluster")) {
        if (value < 0 || value > 16) { set_error("bs_set_tuning: order_cluster=%d outside [0,16]", value); return BS_EINVAL; }
        order_set_cluster(value, 0);
        return BS_OK;
    } else if (!strcmp(name, "order_cluster_min")) {
        if (value < 1) { set_error("bs_set_tuning: order_cluster_min=%d not positive", value); return BS_EINVAL; }
        order_set_cluster(-1, value);
        return BS_OK;
    } else if (!strcmp(name, "order_ctas_per_sm")) {
        if (value < 0 || value > 32) { set_error("bs_set_tuning: order_ctas_per_sm=%d outside [0,32]", value); return BS_EINVAL; }
        ctas = value;
    } else {
        set_error("bs_set_tuning: unknown knob '%s'", name);
        return BS_EINVAL;
    }
    order_set_tuning(threads, ctas);
    return BS_OK;
}

bs_status bs_last_launch_ms(const char *kernel, double *ms) {
    clear_error();
    if (!kernel || !ms) { set_error("bs_last_launch_ms: NULL argument"); return BS_EINVAL; }
    int which = -1;
    if (!strcmp(kernel, "order_init")) which = 0;
    else if (!strcmp(kernel, "order_loop")) which = 1;
    else if (!strcmp(kernel, "order_radius")) which = 2;
    if (which < 0) { set_error("bs_last_launch_ms: unknown kernel '%s'", kernel); return BS_EINVAL; }
    bs_status st = order_last_launch_ms(which, ms);
    if (st == BS_ENOTREADY) set_error("bs_last_launch_ms: no timed launch of %s yet", kernel);
    if (st == BS_ECUDA) set_error("bs_last_launch_ms: event query failed");
    return st;
}

// The scalar arguments of a sampling call, checked before any mesh is staged.
static bs_status check_sample_args(const char *fn, const int *res, int nparts, const bs_dir *dirs, int ndirs) {
    if (nparts < 1 || nparts > 65535 || !res || !dirs) { set_error("%s: NULL argument or nparts outside [1, 65535]", fn); return BS_EINVAL; }
    if (ndirs < 1 || ndirs > BS_MAX_DIRS) { set_error("%s: ndirs=%d outside [1,%d]", fn, ndirs, BS_MAX_DIRS); return BS_EINVAL; }
    for (int i = 0; i < ndirs; ++i) {
        const bs_dir &d = dirs[i];
        if (d.x < -1 || d.x > 1 || d.y < -1 || d.y > 1 || d.z < -1 || d.z > 1 || (d.x == 0 && d.y == 0 && d.z == 0)) {
            set_error("%s: direction %d is not a nonzero vector in {-1,0,1}^3", fn, i);
            return BS_EINVAL;
        }
    }
    for (int p = 0; p < nparts; ++p)
        if (res[p] < 1 || res[p] > BS_MAX_RES) { set_error("%s: part %d: res=%d outside [1,%d]", fn, p, res[p], BS_MAX_RES); return BS_EINVAL; }
    return BS_OK;
}

bs_status bs_sample_visible(const bs_mesh *mesh, const bs_dir *dirs, int ndirs, int res, bs_surfels *out,
                            void *cuda_stream) {
    clear_error();
    if (!mesh || !out) { set_error("bs_sample_visible: NULL argument"); return BS_EINVAL; }
    if (check_sample_args("bs_sample_visible", &res, 1, dirs, ndirs) != BS_OK) return BS_EINVAL;
    std::vector<bs_mesh> dm;
    char *block = nullptr;
    bs_status st = stage_meshes(mesh, 1, dm, &block, (cudaStream_t)cuda_stream);
    if (st != BS_OK) return st;
    st = sample_visible(dm.data(), dirs, ndirs, res, out, (cudaStream_t)cuda_stream);
    if (block) cudaFreeAsync(block, (cudaStream_t)cuda_stream);
    return st;
}

bs_status bs_sample_visible_batched(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs, int ndirs,
                                    bs_surfels *out, void *cuda_stream) {
    clear_error();
    if (!meshes || !out) { set_error("bs_sample_visible_batched: NULL argument"); return BS_EINVAL; }
    if (check_sample_args("bs_sample_visible_batched", res, nparts, dirs, ndirs) != BS_OK) return BS_EINVAL;
    std::vector<bs_mesh> dm;
    char *block = nullptr;
    bs_status st = stage_meshes(meshes, nparts, dm, &block, (cudaStream_t)cuda_stream);
    if (st != BS_OK) return st;
    st = sample_visible_parts(dm.data(), res, nparts, dirs, ndirs, out, (cudaStream_t)cuda_stream);
    if (block) cudaFreeAsync(block, (cudaStream_t)cuda_stream);
    return st;
}

bs_status bs_sample_order_batched(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs, int ndirs,
                                  const bs_order_opts *opts, bs_part_result *out, int out_on_device,
                                  void *cuda_stream) {
    clear_error();
    if (!meshes || !opts || !out) { set_error("bs_sample_order_batched: NULL argument"); return BS_EINVAL; }
    if (check_sample_args("bs_sample_order_batched", res, nparts, dirs, ndirs) != BS_OK) return BS_EINVAL;
    return sample_order_batched(meshes, res, nparts, dirs, ndirs, opts, out, out_on_device, (cudaStream_t)cuda_stream);
}

bs_status bs_order(const bs_surfels *s, const bs_order_opts *opts, uint32_t *perm, int64_t *rad2, float *radius,
                   void *cuda_stream) {
    clear_error();
    std::vector<PartDesc> parts(1);
    bs_status st = make_part(s, opts, perm, rad2, radius, parts[0]);
    if (st != BS_OK) return st;
    return order_parts(parts, (cudaStream_t)cuda_stream, false);
}

bs_status bs_prefix_median_nn(const bs_surfels *s, const uint32_t *perm, uint64_t pm, int64_t *rm2, void *cuda_stream) {
    clear_error();
    return prefix_median_nn(s, perm, pm, rm2, (cudaStream_t)cuda_stream);
}

bs_status bs_prefix_for_radius(const int64_t *rad2, uint64_t m, int64_t r2, uint64_t *p, void *cuda_stream) {
    clear_error();
    return prefix_for_radius(rad2, m, r2, p, (cudaStream_t)cuda_stream);
}

bs_status bs_scene_generate(uint64_t seed, const uint64_t *part_ids, const int32_t *lines, const int32_t *slots,
                            int nparts, int nboxes, int ncyl, const float *size_table, const float *cos32,
                            const float *sin32, float dx, float dy, int local_indices, float *xyz, uint32_t *tri,
                            uint8_t *rgb, void *cuda_stream) {
    clear_error();
    return scene_generate(seed, part_ids, lines, slots, nparts, nboxes, ncyl, size_table, cos32, sin32, dx, dy,
                          local_indices, xyz, tri, rgb, (cudaStream_t)cuda_stream);
}

bs_status bs_render_mesh(const bs_mesh *mesh, const bs_dir *dir, int res, unsigned long long *image, void *cuda_stream) {
    clear_error();
    if (!mesh || !dir || !image) { set_error("bs_render_mesh: NULL argument"); return BS_EINVAL; }
    if (check_sample_args("bs_render_mesh", &res, 1, dir, 1) != BS_OK) return BS_EINVAL;
    std::vector<bs_mesh> dm;
    char *block = nullptr;
    bs_status st = stage_meshes(mesh, 1, dm, &block, (cudaStream_t)cuda_stream);
    if (st != BS_OK) return st;
    st = render_mesh(dm.data(), dir, res, image, (cudaStream_t)cuda_stream);
    if (block) cudaFreeAsync(block, (cudaStream_t)cuda_stream);
    return st;
}

bs_status bs_render_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *node, const bs_dir *dir,
                           unsigned long long *image, void *cuda_stream) {
    clear_error();
    return render_splats(sets, nsets, node, dir, image, (cudaStream_t)cuda_stream);
}

bs_status bs_sample_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *nodes, int nnodes,
                           const bs_dir *dirs, int ndirs, bs_surfels *out, void *cuda_stream) {
    clear_error();
    return sample_splats(sets, nsets, nodes, nnodes, dirs, ndirs, out, (cudaStream_t)cuda_stream);
}

bs_status bs_prefix_for_radius_batched(const int64_t *const *rad2, const uint64_t *m, const int64_t *r2, int nparts,
                                       uint64_t *p, int64_t *r2_at, void *cuda_stream) {
    clear_error();
    return prefix_for_radius_batched(rad2, m, r2, nparts, p, r2_at, (cudaStream_t)cuda_stream);
}

double bs_prefix_estimate(uint64_t pm, int64_t rm2, int64_t r2) {
    if (r2 <= 0) return (double)INFINITY;
    return (double)pm * (double)rm2 / (double)r2;
}

bs_status bs_parent_frames(const float *child_min, const double *child_scale, const uint64_t *child_ofs, int nparents,
                           const int32_t *parent_res, float *frame_min, double *frame_scale, int64_t *child_r2) {
    clear_error();
    return parent_frames(child_min, child_scale, child_ofs, nparents, parent_res, frame_min, frame_scale, child_r2);
}

bs_status bs_order_noalloc(const bs_surfels *s, const bs_order_opts *opts, uint32_t *perm, int64_t *rad2,
                           float *radius, void *cuda_stream) {
    clear_error();
    PartDesc p;
    bs_status st = make_part(s, opts, perm, rad2, radius, p);
    if (st != BS_OK) return st;
    return order_part_noalloc(p, (cudaStream_t)cuda_stream);
}

bs_status bs_order_batched(const bs_surfels *parts, int nparts, const bs_order_opts *opts, uint32_t *const *perm,
                           int64_t *const *rad2, float *const *radius, void *cuda_stream) {
    clear_error();
    if (nparts < 0 || (nparts > 0 && (!parts || !opts || !perm))) { set_error("bs_order_batched: bad arguments"); return BS_EINVAL; }
    std::vector<PartDesc> hp((size_t)nparts);
    for (int i = 0; i < nparts; ++i) {
        bs_status st = make_part(&parts[i], &opts[i], perm[i], rad2 ? rad2[i] : nullptr, radius ? radius[i] : nullptr, hp[i]);
        if (st != BS_OK) {
            char msg[512];
            snprintf(msg, sizeof(msg), "part %d: %s", i, bs_last_error());
            set_error("%s", msg);
            return st;
        }
    }
    return order_parts(hp, (cudaStream_t)cuda_stream, true);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Server: continuous batching.  A host thread admits queued requests while their
// device footprint fits the budget and a stream is free, launches them as one
// batched ordering on that stream (so batches on different streams overlap on
// the device), and retires a batch when its completion event fires.
// ---------------------------------------------------------------------------
namespace bs {

struct SrvReq {
    uint64_t ticket;
    std::vector<uint64_t> key;
    double scale;
    bs_order_opts opts;
    uint64_t n, m, bytes;
    uint64_t *dk;   // its keys and outputs inside the launch's device block
    uint32_t *dp;
    int64_t *dr;
    float *df;
    size_t stage_off;
    std::vector<uint32_t> perm;
    std::vector<int64_t> rad2;
    std::vector<float> radius;
    double t[3];
    int state;  // 0 queued, 1 running, 5 copying its result, 2 done, 3 failed, 4 collected, 6 cancelled
    bool cancel;  // cancelled while on the device: its result is dropped when the launch ends
    bs_status err;
    uint32_t flag;          // index of its completion flag in the slot
    cudaEvent_t copied;     // recorded on the copy stream after its result copies
};

constexpr uint32_t SLOT_FLAGS = 4096;  // requests per launch (one completion flag each)
constexpr size_t SLOT_STAGE_BYTES = 64ull << 20;  // pinned result staging per launch slot, grown on demand

struct SrvSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<SrvReq *> reqs;
    char *stage = nullptr;  // pinned host staging for results
    size_t stage_cap = 0;
    char *kstage = nullptr;  // pinned host staging for the launch's keys (one upload)
    size_t kstage_cap = 0;
    char *dblock = nullptr;  // the launch's device block: every request's keys, then outputs
    std::vector<char *> retired_pinned;  // outgrown staging, freed with the server
    uint32_t *flags_h = nullptr;  // host-mapped completion flags, set by the ordering kernel
    uint32_t *flags_d = nullptr;  // the same memory as the device sees it
    bool busy = false;
};

}  // namespace bs

struct bs_server {
    int device = 0;
    uint64_t budget = 0, used = 0;
    int max_inflight = 4096, inflight = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<bs::SrvReq *> queue;
    std::unordered_map<uint64_t, bs::SrvReq *> all;
    std::vector<bs::SrvSlot> slots;
    cudaStream_t copy = nullptr;  // device-to-host copies of finished requests
    cudaEvent_t copy_tail = nullptr;  // the copy stream's last work, ordered before a launch's memory is freed
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread driver;
    std::chrono::steady_clock::time_point t0;
    size_t max_queue = 1u << 20;
    double timeout_s = 0.0;  // a request on the device longer than this fails with BS_ETIMEOUT (0: none)
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace bs {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t req_bytes(uint64_t n) {
    // key + outputs + ordering scratch (D, bucket and group records) + slack
    const uint64_t nb = (n + 31) / 32, ng = (nb + 31) / 32;
    return (size_t)(n * 8 + n * 4 + n * 8 + n * 4) + (size_t)(n * 8 + n * 8 + nb * 32 + ng * 32) + 4096;
}

// Releases a finished launch: device memory and budget (every request's result has
// been copied by then, see driver_loop).  A request cancelled on the device ends here.
static void retire(bs_server *S, SrvSlot &slot) {
    // a request that timed out may still have its result copy in flight on the copy
    // stream: the block is freed after it
    if (slot.dblock && cudaEventRecord(S->copy_tail, S->copy) == cudaSuccess)
        cudaStreamWaitEvent(slot.stream, S->copy_tail, 0);
    if (slot.dblock) cudaFreeAsync(slot.dblock, slot.stream);
    slot.dblock = nullptr;
    for (SrvReq *r : slot.reqs) {
        r->dk = nullptr; r->dp = nullptr; r->dr = nullptr; r->df = nullptr;
        if (r->cancel && r->state != 4) {
            r->state = 6;
            std::vector<uint32_t>().swap(r->perm);
            std::vector<int64_t>().swap(r->rad2);
            std::vector<float>().swap(r->radius);
        }
        if (r->copied) {
            cudaEventDestroy(r->copied);
            r->copied = nullptr;
        }
        S->used -= r->bytes;
        S->inflight -= 1;
    }
    slot.reqs.clear();
    slot.busy = false;
}

// Starts the device-to-host copy of a request whose part has finished (its flag is
// set) on the copy stream, while the rest of the launch keeps running.
static void start_copy(bs_server *S, SrvSlot &slot, SrvReq *r) {
    char *st = slot.stage + r->stage_off;
    cudaMemcpyAsync(st, r->dp, r->m * 4, cudaMemcpyDeviceToHost, S->copy);
    cudaMemcpyAsync(st + align256(r->m * 4), r->dr, r->m * 8, cudaMemcpyDeviceToHost, S->copy);
    cudaMemcpyAsync(st + align256(r->m * 4) + align256(r->m * 8), r->df, r->m * 4, cudaMemcpyDeviceToHost, S->copy);
    if (!r->copied && cudaEventCreateWithFlags(&r->copied, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        r->copied = nullptr;
    }
    if (r->copied) cudaEventRecord(r->copied, S->copy);
}

// Moves a request's copied result from the slot's pinned staging into its own buffers.
static void finish_copy(SrvSlot &slot, SrvReq *r) {
    const char *st = slot.stage + r->stage_off;
    memcpy(r->perm.data(), st, r->m * 4);
    memcpy(r->rad2.data(), st + align256(r->m * 4), r->m * 8);
    memcpy(r->radius.data(), st + align256(r->m * 4) + align256(r->m * 8), r->m * 4);
}

// Grows a pinned host staging buffer to at least `need` bytes (twice that when it grows).
// The outgrown buffer is kept until the server is destroyed: cudaFreeHost would wait for
// all work on the device, stalling every launch in flight.
static bool ensure_pinned(SrvSlot &slot, char **buf, size_t *cap, size_t need) {
    if (need <= *cap) return true;
    if (*buf) slot.retired_pinned.push_back(*buf);
    *buf = nullptr;
    *cap = 0;
    if (cudaHostAlloc((void **)buf, need * 2, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return false;
    }
    *cap = need * 2;
    return true;
}

// The device work of a launch: one device block for every request's keys and outputs,
// the keys gathered into pinned staging and uploaded in one copy, the ordering launch.
// Runs without the server lock; it touches only the slot and fields of the batch's
// requests that no other thread reads (the requests are still "queued" to poll and
// times).  err[i] receives each request's outcome (BS_OK when it runs); when the block
// cannot be had, every request of the launch fails with BS_ENOMEM and the device is
// left as it was.
static void launch_batch(bs_server *S, SrvSlot &slot, std::vector<SrvReq *> &batch, std::vector<bs_status> &err) {
    size_t stage = 0, keys = 0, outs = 0;
    for (SrvReq *r : batch) {
        r->stage_off = stage;
        stage += align256(r->m * 4) + align256(r->m * 8) + align256(r->m * 4);
        keys += align256(r->n * 8);
        outs += align256(r->m * 4) + align256(r->m * 8) + align256(r->m * 4);
    }
    err.assign(batch.size(), BS_OK);
    bool ok = ensure_pinned(slot, &slot.stage, &slot.stage_cap, stage) &&
              ensure_pinned(slot, &slot.kstage, &slot.kstage_cap, keys);
    if (ok && pool_malloc_async((void **)&slot.dblock, keys + outs, slot.stream) != cudaSuccess) {
        cudaGetLastError();
        slot.dblock = nullptr;
        ok = false;
    }
    if (!ok) {
        for (size_t i = 0; i < batch.size(); ++i) err[i] = BS_ENOMEM;
        cudaEventRecord(slot.done, slot.stream);
        return;
    }
    std::vector<PartDesc> parts;
    parts.reserve(batch.size());
    size_t ko = 0, oo = keys;
    for (size_t i = 0; i < batch.size(); ++i) {
        SrvReq *r = batch[i];
        memcpy(slot.kstage + ko, r->key.data(), r->n * 8);
        std::vector<uint64_t>().swap(r->key);
        r->dk = (uint64_t *)(slot.dblock + ko);
        ko += align256(r->n * 8);
        r->dp = (uint32_t *)(slot.dblock + oo);
        r->dr = (int64_t *)(slot.dblock + oo + align256(r->m * 4));
        r->df = (float *)(slot.dblock + oo + align256(r->m * 4) + align256(r->m * 8));
        oo += align256(r->m * 4) + align256(r->m * 8) + align256(r->m * 4);
        PartDesc p;
        memset(&p, 0, sizeof(p));
        p.key = r->dk; p.perm = r->dp; p.rad2 = r->dr; p.radius = r->df; p.scale = r->scale;
        r->flag = (uint32_t)parts.size();
        slot.flags_h[r->flag] = 0u;
        p.done = slot.flags_d + r->flag;
        p.n = (uint32_t)r->n; p.m = (uint32_t)r->m;
        p.start = (uint32_t)(r->opts.start >= 0 ? (uint64_t)r->opts.start : start_from_seed(r->n, r->opts.seed, r->opts.part_id));
        p.variant = (uint32_t)r->opts.variant;
        p.sample_size = r->opts.sample_size;
        p.sample_step = r->opts.sample_step;
        p.part_id = r->opts.part_id;
        p.seed = r->opts.seed;
        parts.push_back(p);
    }
    if (cudaMemcpyAsync(slot.dblock, slot.kstage, keys, cudaMemcpyHostToDevice, slot.stream) != cudaSuccess) {
        set_error("bs_server: key upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        for (size_t i = 0; i < batch.size(); ++i) err[i] = BS_ECUDA;
    } else {
        // several requests share the GPU as quarters of CTAs, like a large batch
        const bs_status st = order_parts(parts, slot.stream, true, true);
        if (st != BS_OK)
            for (size_t i = 0; i < batch.size(); ++i) err[i] = st;
    }
    cudaEventRecord(slot.done, slot.stream);
}

// The driver thread.  The server lock guards the queue, the budget and every request's
// state; the driver holds it only to read and change those, and drops it for the CUDA
// calls and copies, so that submit and poll from other threads never wait on them.  The
// requests it works on meanwhile stay in a state (queued, running, copying) that poll
// and times answer without touching their buffers, and only this thread changes slots.
static void driver_loop(bs_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    std::vector<SrvReq *> to_copy, to_finish;
    std::vector<SrvSlot *> copy_owner, finish_owner;
    std::vector<bs_status> err;
    while (!S->stop) {
        bool progressed = false;
        // 1. requests whose part has finished (flag set) or whose result copy has landed
        to_copy.clear();
        to_finish.clear();
        copy_owner.clear();
        finish_owner.clear();
        const double tnow = S->now();
        for (SrvSlot &slot : S->slots) {
            if (!slot.busy) continue;
            for (SrvReq *r : slot.reqs) {
                if ((r->state == 1 || r->state == 5) && S->timeout_s > 0.0 && tnow - r->t[1] > S->timeout_s) {
                    // a bounded wait: the request fails now; its launch keeps running and its
                    // memory and budget are released when the launch ends
                    r->state = 3;
                    r->err = BS_ETIMEOUT;
                    r->t[2] = tnow;
                    progressed = true;
                    continue;
                }
                if (r->state == 1 && ((volatile uint32_t *)slot.flags_h)[r->flag] != 0u) {
                    to_copy.push_back(r);
                    copy_owner.push_back(&slot);
                } else if (r->state == 5 && (!r->copied || cudaEventQuery(r->copied) == cudaSuccess)) {
                    to_finish.push_back(r);
                    finish_owner.push_back(&slot);
                }
            }
        }
        if (!to_copy.empty() || !to_finish.empty()) {
            lk.unlock();
            for (size_t i = 0; i < to_copy.size(); ++i) start_copy(S, *copy_owner[i], to_copy[i]);
            bool sync = false;
            for (SrvReq *r : to_finish) sync |= !r->copied;
            if (sync) cudaStreamSynchronize(S->copy);
            for (size_t i = 0; i < to_finish.size(); ++i) finish_copy(*finish_owner[i], to_finish[i]);
            lk.lock();
            const double t = S->now();
            // (a request that timed out meanwhile keeps its failed state)
            for (SrvReq *r : to_copy)
                if (r->state == 1) r->state = 5;
            for (SrvReq *r : to_finish)
                if (r->state == 5) { r->t[2] = t; r->state = 2; }
            progressed = true;
        }
        // 2. launches whose every request is finished
        for (SrvSlot &slot : S->slots) {
            if (!slot.busy) continue;
            bool all_done = true;
            for (SrvReq *r : slot.reqs) all_done &= r->state == 2 || r->state == 3 || r->state == 4 || r->state == 6;
            if (all_done && cudaEventQuery(slot.done) == cudaSuccess) {
                retire(S, slot);
                progressed = true;
            }
        }
        if (progressed) S->cv.notify_all();
        // 3. new launches on free slots
        for (SrvSlot &slot : S->slots) {
            if (slot.busy || S->queue.empty()) continue;
            std::vector<SrvReq *> batch;
            while (!S->queue.empty() && S->inflight < S->max_inflight && batch.size() < SLOT_FLAGS) {
                SrvReq *r = S->queue.front();
                if (S->used + r->bytes > S->budget) break;  // FIFO admission under the memory budget
                S->queue.pop_front();
                S->used += r->bytes;
                S->inflight += 1;
                batch.push_back(r);
            }
            if (batch.empty()) break;
            slot.busy = true;
            const double t1 = S->now();
            lk.unlock();
            launch_batch(S, slot, batch, err);
            lk.lock();
            const double t2 = S->now();
            for (size_t i = 0; i < batch.size(); ++i) {
                SrvReq *r = batch[i];
                r->t[1] = t1;
                if (err[i] == BS_OK) r->state = 1;
                else { r->state = 3; r->err = err[i]; r->t[2] = t2; }
            }
            slot.reqs = std::move(batch);
            progressed = true;
        }
        if (!progressed) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace bs

extern "C" {

bs_server *bs_server_create(uint64_t device_budget_bytes, int max_inflight, bs_status *st) {
    clear_error();
    if (device_budget_bytes == 0 || max_inflight < 0) {
        set_error("bs_server_create: budget must be > 0 and max_inflight >= 0");
        if (st) *st = BS_EINVAL;
        return nullptr;
    }
    bs_server *S = new (std::nothrow) bs_server();
    if (!S) { if (st) *st = BS_ENOMEM; return nullptr; }
    cudaGetDevice(&S->device);
    S->budget = device_budget_bytes;
    S->max_inflight = max_inflight ? max_inflight : 4096;
    S->timeout_s = g_server_timeout_ms * 1e-3;
    S->t0 = std::chrono::steady_clock::now();
    S->slots.resize((size_t)g_server_slots);  // launches in flight at once: each holds the requests queued when it started
    if (cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->copy_tail, cudaEventDisableTiming) != cudaSuccess) {
        set_error("bs_server_create: stream creation failed: %s", cudaGetErrorString(cudaGetLastError()));
        if (st) *st = BS_ECUDA;
        delete S;
        return nullptr;
    }
    for (SrvSlot &slot : S->slots) {
        if (cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc((void **)&slot.flags_h, SLOT_FLAGS * sizeof(uint32_t), cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&slot.flags_d, slot.flags_h, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&slot.stage, SLOT_STAGE_BYTES, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&slot.kstage, SLOT_STAGE_BYTES, cudaHostAllocDefault) != cudaSuccess) {
            set_error("bs_server_create: stream/event creation failed: %s", cudaGetErrorString(cudaGetLastError()));
            if (st) *st = BS_ECUDA;
            for (SrvSlot &s2 : S->slots) {
                if (s2.stream) cudaStreamDestroy(s2.stream);
                if (s2.done) cudaEventDestroy(s2.done);
                if (s2.flags_h) cudaFreeHost(s2.flags_h);
                if (s2.stage) cudaFreeHost(s2.stage);
                if (s2.kstage) cudaFreeHost(s2.kstage);
            }
            cudaStreamDestroy(S->copy);
            delete S;
            return nullptr;
        }
        slot.stage_cap = SLOT_STAGE_BYTES;
        slot.kstage_cap = SLOT_STAGE_BYTES;
    }
    S->driver = std::thread(driver_loop, S);
    if (st) *st = BS_OK;
    return S;
}

bs_status bs_server_submit(bs_server *S, const uint64_t *key, uint64_t n, double scale, const bs_order_opts *opts,
                           uint64_t *ticket) {
    clear_error();
    if (!S || !key || !opts || !ticket) { set_error("bs_server_submit: NULL argument"); return BS_EINVAL; }
    if (n == 0 || n > BS_MAX_POINTS) { set_error("bs_server_submit: n=%llu outside [1,%u]", (unsigned long long)n, BS_MAX_POINTS); return BS_EINVAL; }
    if (opts->start >= 0 && (uint64_t)opts->start >= n) { set_error("bs_server_submit: start >= n"); return BS_EINVAL; }
    if (opts->variant != 0 && opts->variant != 1) { set_error("bs_server_submit: variant must be 0 or 1"); return BS_EINVAL; }
    if (opts->variant == 1 && (opts->sample_size < 1 || opts->sample_size > 256)) {
        set_error("bs_server_submit: sample_size outside [1, 256]");
        return BS_EINVAL;
    }
    if (!(scale > 0.0)) { set_error("bs_server_submit: scale must be > 0"); return BS_EINVAL; }
    SrvReq *r = new (std::nothrow) SrvReq();
    if (!r) return BS_ENOMEM;
    r->n = n;
    r->m = (opts->max_count == 0 || opts->max_count > n) ? n : opts->max_count;
    r->bytes = req_bytes(n);
    if (r->bytes > S->budget) {
        delete r;
        set_error("bs_server_submit: request needs %llu bytes, budget is %llu", (unsigned long long)req_bytes(n),
                  (unsigned long long)S->budget);
        return BS_ENOMEM;
    }
    r->key.assign(key, key + n);
    r->scale = scale;
    r->opts = *opts;
    r->perm.resize(r->m);
    r->rad2.resize(r->m);
    r->radius.resize(r->m);
    r->state = 0;
    r->err = BS_OK;
    r->dk = nullptr; r->dp = nullptr; r->dr = nullptr; r->df = nullptr;
    r->cancel = false;
    r->flag = 0;
    r->copied = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queue.size() >= S->max_queue) { delete r; set_error("bs_server_submit: queue full"); return BS_EBUSY; }
    r->ticket = S->next_ticket++;
    r->t[0] = S->now();
    r->t[1] = r->t[2] = 0.0;
    S->queue.push_back(r);
    S->all[r->ticket] = r;
    *ticket = r->ticket;
    return BS_OK;
}

bs_status bs_server_poll(bs_server *S, uint64_t ticket, uint32_t *perm, int64_t *rad2, float *radius) {
    clear_error();
    if (!S) { set_error("bs_server_poll: NULL server"); return BS_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("bs_server_poll: unknown ticket %llu", (unsigned long long)ticket); return BS_EINVAL; }
    SrvReq *r = it->second;
    if (r->state == 0 || r->state == 1 || r->state == 5) return BS_ENOTREADY;
    if (r->state == 3) {
        set_error("bs_server_poll: request %llu failed", (unsigned long long)ticket);
        return r->err == BS_OK ? BS_ECUDA : r->err;
    }
    if (r->state == 4) { set_error("bs_server_poll: ticket %llu already collected", (unsigned long long)ticket); return BS_EINVAL; }
    if (r->state == 6 || r->cancel) {
        set_error("bs_server_poll: request %llu was cancelled", (unsigned long long)ticket);
        return BS_ECANCELED;
    }
    if (!perm) return BS_OK;  // status query only
    memcpy(perm, r->perm.data(), r->m * 4);
    if (rad2) memcpy(rad2, r->rad2.data(), r->m * 8);
    if (radius) memcpy(radius, r->radius.data(), r->m * 4);
    r->state = 4;
    std::vector<uint64_t>().swap(r->key);
    std::vector<uint32_t>().swap(r->perm);
    std::vector<int64_t>().swap(r->rad2);
    std::vector<float>().swap(r->radius);
    return BS_OK;
}

bs_status bs_server_times(bs_server *S, uint64_t ticket, double t[3]) {
    clear_error();
    if (!S || !t) { set_error("bs_server_times: NULL argument"); return BS_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("bs_server_times: unknown ticket"); return BS_EINVAL; }
    SrvReq *r = it->second;
    if (r->state != 2 && r->state != 3 && r->state != 4 && r->state != 6) return BS_ENOTREADY;
    t[0] = r->t[0]; t[1] = r->t[1]; t[2] = r->t[2];
    return BS_OK;
}

bs_status bs_server_cancel(bs_server *S, uint64_t ticket) {
    clear_error();
    if (!S) { set_error("bs_server_cancel: NULL server"); return BS_EINVAL; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) { set_error("bs_server_cancel: unknown ticket %llu", (unsigned long long)ticket); return BS_EINVAL; }
    SrvReq *r = it->second;
    switch (r->state) {
        case 0: {  // queued: leaves the queue now (no budget was charged yet)
            for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
                if (*q == r) { S->queue.erase(q); break; }
            r->state = 6;
            r->t[1] = r->t[2] = S->now();
            std::vector<uint64_t>().swap(r->key);
            std::vector<uint32_t>().swap(r->perm);
            std::vector<int64_t>().swap(r->rad2);
            std::vector<float>().swap(r->radius);
            return BS_OK;
        }
        case 1:
        case 5:  // on the device: dropped when its launch ends, which releases its memory and budget
            r->cancel = true;
            return BS_OK;
        case 2:  // finished, not collected: the result is dropped
            r->state = 6;
            std::vector<uint32_t>().swap(r->perm);
            std::vector<int64_t>().swap(r->rad2);
            std::vector<float>().swap(r->radius);
            return BS_OK;
        case 6:
            return BS_OK;
        default:
            set_error("bs_server_cancel: request %llu already failed or collected", (unsigned long long)ticket);
            return BS_EINVAL;
    }
}

void bs_server_destroy(bs_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    if (S->driver.joinable()) S->driver.join();
    for (SrvSlot &slot : S->slots) {
        if (slot.busy) {
            cudaEventSynchronize(slot.done);
            cudaStreamSynchronize(S->copy);
            retire(S, slot);
        }
        if (slot.stage) cudaFreeHost(slot.stage);
        if (slot.kstage) cudaFreeHost(slot.kstage);
        for (char *b : slot.retired_pinned) cudaFreeHost(b);
        if (slot.flags_h) cudaFreeHost(slot.flags_h);
        cudaEventDestroy(slot.done);
        cudaStreamDestroy(slot.stream);
    }
    cudaEventDestroy(S->copy_tail);
    cudaStreamDestroy(S->copy);
    for (auto &kv : S->all) delete kv.second;
    delete S;
}

}  // extern "C"
