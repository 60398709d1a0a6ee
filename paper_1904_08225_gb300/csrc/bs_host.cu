// bs_host.cu -- host buffers at the boundary: meshes given in host memory are uploaded
// by the library (the node geometry of Sec. 3.1), and bs_sample_order_batched runs the
// whole path -- sampling (Sec. 3.1), ordering (Sec. 3.2) and radii (Sec. 4.1) -- from
// host meshes to host results in one call.
//
// Copies: arrays of consecutive meshes (or parts) that lie back to back in host memory
// move as one copy.  A page-locked host array is copied directly on the call's stream;
// a pageable one goes through pinned staging that the library owns (one buffer per
// device, grown on demand, reused once its previous copies have finished).
#include <mutex>
#include <vector>

#include "bs_internal.cuh"

namespace bs {

namespace {

struct PinnedStage {
    std::mutex mu;
    char *buf = nullptr;
    size_t cap = 0;
    cudaEvent_t last = nullptr;  // the last copies out of (or into) buf
    bool pending = false;
};
PinnedStage g_stage[64];

std::mutex g_copy_mu;
cudaStream_t g_copy_stream[64] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return -1;
    }
    return dev;
}

// True for page-locked host memory (cudaHostAlloc'd or registered).
bool is_pinned(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// One contiguous host range and where it goes (or comes from) on the device.
struct Run {
    const char *host;  // host start (a const pointer for uploads; the destination for downloads)
    char *dev;
    size_t bytes;
};

// Groups segments (host pointer, bytes) into runs of back-to-back host ranges of the
// same array kind; each run gets the next 256-aligned offset of a device block.
// Returns the block size.
size_t plan_runs(const std::vector<std::pair<const char *, size_t>> &segs, const std::vector<int> &kind,
                 std::vector<Run> &runs, std::vector<size_t> &seg_off) {
    size_t off = 0;
    seg_off.assign(segs.size(), 0);
    for (size_t i = 0; i < segs.size(); ++i) {
        const char *h = segs[i].first;
        const size_t b = segs[i].second;
        if (!runs.empty() && kind[i] == kind[i - 1] && runs.back().host + runs.back().bytes == h) {
            seg_off[i] = (size_t)runs.back().dev + runs.back().bytes;  // an offset until the block exists
            runs.back().bytes += b;
            off += b;
            continue;
        }
        off = align256(off);
        runs.push_back(Run{h, (char *)off, b});
        seg_off[i] = off;
        off += b;
    }
    return align256(off);
}

// Copies runs host -> device on `stream`: page-locked sources directly, the others
// through the device's pinned staging.
bs_status upload_runs(std::vector<Run> &runs, cudaStream_t stream) {
    size_t pageable = 0;
    for (const Run &r : runs)
        if (!is_pinned(r.host)) pageable += align256(r.bytes);
    for (const Run &r : runs)
        if (is_pinned(r.host) && cudaMemcpyAsync(r.dev, r.host, r.bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
            set_error("host upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            return BS_ECUDA;
        }
    if (pageable == 0) return BS_OK;
    const int dev = current_device();
    if (dev < 0) { set_error("host upload: no current device"); return BS_ECUDA; }
    PinnedStage &S = g_stage[dev];
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.pending && cudaEventSynchronize(S.last) != cudaSuccess) {
        set_error("host upload: staging wait failed: %s", cudaGetErrorString(cudaGetLastError()));
        return BS_ECUDA;
    }
    S.pending = false;
    if (!S.last && cudaEventCreateWithFlags(&S.last, cudaEventDisableTiming) != cudaSuccess) {
        set_error("host upload: event creation failed");
        return BS_ECUDA;
    }
    if (pageable > S.cap) {
        if (S.buf) cudaFreeHost(S.buf);
        S.buf = nullptr;
        S.cap = 0;
        if (cudaHostAlloc((void **)&S.buf, pageable, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            set_error("host upload: %zu bytes of pinned staging unavailable", pageable);
            return BS_ENOMEM;
        }
        S.cap = pageable;
    }
    size_t off = 0;
    for (const Run &r : runs) {
        if (is_pinned(r.host)) continue;
        memcpy(S.buf + off, r.host, r.bytes);
        if (cudaMemcpyAsync(r.dev, S.buf + off, r.bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) {
            set_error("host upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            return BS_ECUDA;
        }
        off += align256(r.bytes);
    }
    cudaEventRecord(S.last, stream);
    S.pending = true;
    return BS_OK;
}

// The device's stream for reading results back beside the ordering.
cudaStream_t copy_stream() {
    const int dev = current_device();
    if (dev < 0) return nullptr;
    std::lock_guard<std::mutex> lk(g_copy_mu);
    if (!g_copy_stream[dev] && cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        g_copy_stream[dev] = nullptr;
    }
    return g_copy_stream[dev];
}

}  // namespace

bs_status stage_meshes(const bs_mesh *in, int n, std::vector<bs_mesh> &dev, char **block, cudaStream_t stream) {
    *block = nullptr;
    dev.assign(in, in + n);
    // host segments in mesh order, one kind at a time so that packed arrays form runs
    std::vector<std::pair<const char *, size_t>> segs;
    std::vector<std::pair<int, int>> who;  // (mesh, kind)
    for (int kind = 0; kind < 3; ++kind)
        for (int i = 0; i < n; ++i) {
            const bs_mesh &m = in[i];
            if (m.on_device) continue;
            const void *p = kind == 0 ? (const void *)m.xyz : kind == 1 ? (const void *)m.tri : (const void *)m.face_rgb;
            const size_t b = kind == 0 ? (size_t)m.nverts * 12 : kind == 1 ? (size_t)m.ntris * 12 : (size_t)m.ntris * 3;
            if (!p || b == 0) continue;
            segs.emplace_back((const char *)p, b);
            who.emplace_back(i, kind);
        }
    for (bs_mesh &m : dev) m.on_device = 1;
    if (segs.empty()) return BS_OK;
    std::vector<Run> runs;
    std::vector<size_t> seg_off;
    std::vector<int> kinds(who.size());
    for (size_t s = 0; s < who.size(); ++s) kinds[s] = who[s].second;
    const size_t bytes = plan_runs(segs, kinds, runs, seg_off);
    char *base = nullptr;
    if (pool_malloc_async((void **)&base, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        set_error("host meshes: %zu bytes of device memory unavailable", bytes);
        return BS_ENOMEM;
    }
    for (Run &r : runs) r.dev = base + (size_t)r.dev;
    for (size_t s = 0; s < segs.size(); ++s) {
        bs_mesh &m = dev[(size_t)who[s].first];
        char *d = base + seg_off[s];
        if (who[s].second == 0) m.xyz = (const float *)d;
        else if (who[s].second == 1) m.tri = (const uint32_t *)d;
        else m.face_rgb = (const uint8_t *)d;
    }
    const bs_status st = upload_runs(runs, stream);
    if (st != BS_OK) {
        cudaFreeAsync(base, stream);
        return st;
    }
    *block = base;
    return BS_OK;
}

bs_status sample_order_batched(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs, int ndirs,
                               const bs_order_opts *opts, bs_part_result *out, int out_on_device,
                               cudaStream_t stream) {
    if (nparts < 1 || !meshes || !res || !dirs || !opts || !out) {
        set_error("bs_sample_order_batched: NULL argument or nparts < 1");
        return BS_EINVAL;
    }
    for (int p = 0; p < nparts; ++p)
        if (!out[p].perm && out[p].cap > 0) {
            set_error("bs_sample_order_batched: part %d: NULL perm", p);
            return BS_EINVAL;
        }
    std::vector<bs_mesh> dm;
    char *mblock = nullptr;
    bs_status st = stage_meshes(meshes, nparts, dm, &mblock, stream);
    if (st != BS_OK) return st;
    // surfel records: the caller's device arrays, or device scratch laid out part after
    // part with each part's cap rows (back to back, so packed host outputs read back as
    // one copy per array)
    uint64_t rows = 0;
    std::vector<uint64_t> rofs((size_t)nparts);
    for (int p = 0; p < nparts; ++p) { rofs[(size_t)p] = rows; rows += out[p].cap; }
    char *sblock = nullptr;
    uint64_t *skey = nullptr;
    int16_t *snrm = nullptr;
    uint8_t *srgb = nullptr;
    uint32_t *ssrc = nullptr;
    uint32_t *sperm = nullptr;
    int64_t *srad2 = nullptr;
    float *srad = nullptr;
    if (!out_on_device) {
        const size_t bytes = align256(rows * 8) * 2 + align256(rows * 6) + align256(rows * 3) + align256(rows * 4) * 3;
        if (pool_malloc_async((void **)&sblock, bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            if (mblock) cudaFreeAsync(mblock, stream);
            set_error("bs_sample_order_batched: %zu bytes of device scratch unavailable", bytes);
            return BS_ENOMEM;
        }
        size_t o = 0;
        skey = (uint64_t *)(sblock + o); o += align256(rows * 8);
        snrm = (int16_t *)(sblock + o); o += align256(rows * 6);
        srgb = (uint8_t *)(sblock + o); o += align256(rows * 3);
        ssrc = (uint32_t *)(sblock + o); o += align256(rows * 4);
        sperm = (uint32_t *)(sblock + o); o += align256(rows * 4);
        srad2 = (int64_t *)(sblock + o); o += align256(rows * 8);
        srad = (float *)(sblock + o);
    }
    std::vector<bs_surfels> sv((size_t)nparts);
    for (int p = 0; p < nparts; ++p) {
        bs_surfels &s = sv[(size_t)p];
        memset(&s, 0, sizeof(s));
        const uint64_t r = rofs[(size_t)p];
        s.key = out_on_device ? out[p].key : skey + r;
        s.nrm = out_on_device ? out[p].nrm : snrm + 3 * r;
        s.rgb = out_on_device ? out[p].rgb : srgb + 3 * r;
        s.src = out_on_device ? out[p].src : ssrc + r;
        s.cap = out[p].cap;
    }
    bool need_key_scratch = false;
    for (int p = 0; p < nparts && out_on_device; ++p) need_key_scratch |= !out[p].key;
    if (need_key_scratch) {  // device outputs without keys: the ordering still needs them
        if (pool_malloc_async((void **)&sblock, align256(rows * 8), stream) != cudaSuccess) {
            cudaGetLastError();
            if (mblock) cudaFreeAsync(mblock, stream);
            set_error("bs_sample_order_batched: device scratch unavailable");
            return BS_ENOMEM;
        }
        for (int p = 0; p < nparts; ++p)
            if (!out[p].key) sv[(size_t)p].key = (uint64_t *)sblock + rofs[(size_t)p];
    }
    st = sample_visible_parts(dm.data(), res, nparts, dirs, ndirs, sv.data(), stream);
    if (mblock) cudaFreeAsync(mblock, stream);
    for (int p = 0; p < nparts; ++p) {
        out[p].n = sv[(size_t)p].n;
        for (int a = 0; a < 3; ++a) out[p].bbox_min[a] = sv[(size_t)p].bbox_min[a];
        out[p].scale = sv[(size_t)p].scale;
    }
    if (st != BS_OK) {
        if (sblock) cudaFreeAsync(sblock, stream);
        return st;
    }
    // the surfel records go back on the copy stream while the ordering runs
    cudaStream_t cs = out_on_device ? nullptr : copy_stream();
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto fail = [&](const char *what) {
        set_error("bs_sample_order_batched: %s: %s", what, cudaGetErrorString(cudaGetLastError()));
        for (int i = 0; i < 2; ++i)
            if (ev[i]) cudaEventDestroy(ev[i]);
        if (sblock) cudaFreeAsync(sblock, stream);
        return BS_ECUDA;
    };
    // back-to-back host destinations (and sources) of consecutive parts form one copy
    auto download = [&](cudaStream_t s, size_t width, auto dst_of, const char *src_base, auto count_of) -> bool {
        int p = 0;
        while (p < nparts) {
            char *d0 = (char *)dst_of(p);
            if (!d0 || count_of(p) == 0) { ++p; continue; }
            const char *s0 = src_base + rofs[(size_t)p] * width;
            size_t bytes = count_of(p) * width;
            int q = p + 1;
            while (q < nparts && (char *)dst_of(q) == d0 + bytes && src_base + rofs[(size_t)q] * width == s0 + bytes &&
                   count_of(q) > 0) {
                bytes += count_of(q) * width;
                ++q;
            }
            if (cudaMemcpyAsync(d0, s0, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
            p = q;
        }
        return true;
    };
    auto n_of = [&](int p) { return (size_t)out[p].n; };
    if (!out_on_device) {
        if (!cs) return fail("copy stream");
        if (cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess)
            return fail("event creation");
        cudaEventRecord(ev[0], stream);
        cudaStreamWaitEvent(cs, ev[0], 0);
        if (!download(cs, 8, [&](int p) { return (void *)out[p].key; }, (const char *)skey, n_of) ||
            !download(cs, 6, [&](int p) { return (void *)out[p].nrm; }, (const char *)snrm, n_of) ||
            !download(cs, 3, [&](int p) { return (void *)out[p].rgb; }, (const char *)srgb, n_of) ||
            !download(cs, 4, [&](int p) { return (void *)out[p].src; }, (const char *)ssrc, n_of))
            return fail("surfel read-back");
    }
    // the ordering
    std::vector<PartDesc> hp((size_t)nparts);
    std::vector<uint64_t> ms((size_t)nparts);
    for (int p = 0; p < nparts; ++p) {
        const bs_order_opts &o = opts[p];
        const uint64_t n = out[p].n;
        const uint64_t m = (o.max_count == 0 || o.max_count > n) ? n : o.max_count;
        ms[(size_t)p] = m;
        if (n == 0 || n > BS_MAX_POINTS || (o.start >= 0 && (uint64_t)o.start >= n) || o.variant < 0 || o.variant > 1 ||
            (o.variant == 1 && (o.sample_size < 1 || o.sample_size > 256))) {
            set_error("bs_sample_order_batched: part %d: cannot order (n=%llu)", p, (unsigned long long)n);
            for (int i = 0; i < 2; ++i)
                if (ev[i]) { cudaStreamSynchronize(cs); cudaEventDestroy(ev[i]); ev[i] = nullptr; }
            if (sblock) cudaFreeAsync(sblock, stream);
            return BS_EINVAL;
        }
        PartDesc &d = hp[(size_t)p];
        memset(&d, 0, sizeof(d));
        const uint64_t r = rofs[(size_t)p];
        d.key = sv[(size_t)p].key;
        d.perm = out_on_device ? out[p].perm : sperm + r;
        d.rad2 = out_on_device ? out[p].rad2 : srad2 + r;
        d.radius = out_on_device ? out[p].radius : (out[p].radius ? srad + r : nullptr);
        d.scale = out[p].scale;
        d.n = (uint32_t)n;
        d.m = (uint32_t)m;
        d.start = (uint32_t)(o.start >= 0 ? (uint64_t)o.start : start_from_seed(n, o.seed, o.part_id));
        d.variant = (uint32_t)o.variant;
        d.sample_size = o.sample_size;
        d.sample_step = o.sample_step;
        d.part_id = o.part_id;
        d.seed = o.seed;
    }
    st = order_parts(hp, stream, true);
    if (st != BS_OK) {
        if (cs) cudaStreamSynchronize(cs);
        for (int i = 0; i < 2; ++i)
            if (ev[i]) cudaEventDestroy(ev[i]);
        if (sblock) cudaFreeAsync(sblock, stream);
        return st;
    }
    if (!out_on_device) {
        auto m_of = [&](int p) { return (size_t)ms[(size_t)p]; };
        if (!download(stream, 4, [&](int p) { return (void *)out[p].perm; }, (const char *)sperm, m_of) ||
            !download(stream, 8, [&](int p) { return (void *)out[p].rad2; }, (const char *)srad2, m_of) ||
            !download(stream, 4, [&](int p) { return (void *)out[p].radius; }, (const char *)srad, m_of))
            return fail("result read-back");
        cudaEventRecord(ev[1], cs);
        cudaStreamWaitEvent(stream, ev[1], 0);  // the records are read before the scratch is freed
    }
    if (sblock) cudaFreeAsync(sblock, stream);
    const cudaError_t e = cudaStreamSynchronize(stream);
    for (int i = 0; i < 2; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) {
        set_error("bs_sample_order_batched: %s", cudaGetErrorString(e));
        return BS_ECUDA;
    }
    return BS_OK;
}

}  // namespace bs
