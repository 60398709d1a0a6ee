/*
 * bs.h -- C ABI of libbs: visible-surface surfel sampling and progressive
 * (greedy-permutation) ordering on a GB300 GPU (sm_103a), after Brandt et al.,
 * "Rendering of Complex Heterogenous Scenes using Progressive Blue Surfels".
 *
 * Conventions shared by every call:
 *  - Plain pointers and sizes only.  Unless a field says otherwise, array
 *    pointers are CUDA DEVICE pointers owned by the caller; the library never
 *    frees or keeps them after the call's stream work completes.
 *  - Work is issued on the CUDA stream passed as `cuda_stream` (a cudaStream_t;
 *    NULL = the legacy default stream) and is ordered with the caller's other
 *    work on that stream.  Scratch memory is taken from the device's
 *    stream-ordered memory pool on that stream and returned on it.
 *  - The library never aborts.  Every failure returns a status and records a
 *    message readable through bs_last_error() on the calling thread.  A CUDA
 *    runtime error maps to BS_ECUDA.
 *  - All arithmetic on the ordering path is integer; results are bit-exact and
 *    do not depend on launch configuration, stream or batch composition.
 */
#ifndef BS_H
#define BS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BS_OK = 0,
    BS_EINVAL = 1,     /* argument out of range, non-finite vertex, zero extent */
    BS_ENOMEM = 2,     /* device scratch or admission budget exhausted */
    BS_EOVERFLOW = 3,  /* output capacity too small (the needed size is reported) */
    BS_ETIMEOUT = 4,   /* a bounded wait ran out (a server request past its timeout) */
    BS_EBUSY = 5,      /* server queue full; retry later */
    BS_ECUDA = 6,      /* CUDA runtime error */
    BS_ENOTREADY = 7,  /* server result not finished yet */
    BS_ECANCELED = 8   /* server request cancelled by bs_server_cancel */
} bs_status;

/* Largest quantised coordinate: positions are integers in [0, 2^21 - 1]. */
#define BS_QMAX 2097151
/* Maximum raster resolution per direction and maximum number of directions. */
#define BS_MAX_RES 4096
#define BS_MAX_DIRS 26
/* Largest part bs_order / bs_order_batched accept (points). */
#define BS_MAX_POINTS 6291456u

/* A triangle mesh of one scene node (Sec. 3: geometry in the node's subtree).
 * xyz: nverts*3 float32 positions; tri: ntris*3 vertex indices (< nverts);
 * face_rgb: ntris*3 bytes of per-face colour, or NULL (colour 0).
 * on_device: nonzero when the three arrays are device pointers; 0 when they are HOST
 * pointers, which the library copies to the device on the call's stream before use
 * (page-locked arrays directly; pageable ones through pinned staging the library owns,
 * reused once its previous copy has finished; arrays of consecutive meshes that lie
 * back to back in host memory move as one copy).  The caller keeps ownership. */
typedef struct {
    const float *xyz;
    uint32_t nverts;
    const uint32_t *tri;
    uint32_t ntris;
    const uint8_t *face_rgb;
    int32_t on_device;
} bs_mesh;

/* A view direction with integer components in {-1, 0, 1}, not all zero.  The
 * camera sits on the +d side of the node and looks along -d (Sec. 3.1 renders
 * from the bounding-box corners toward the centre; d = (+-1, +-1, +-1) are those
 * corners, the six axis directions are also allowed). */
typedef struct {
    int8_t x, y, z;
} bs_dir;

/* A surfel array in canonical order (ascending Morton code of the position).
 *  key : packed quantised position, x << 42 | y << 21 | z (21 bits each)
 *  nrm : unit normal as 3 x int16 (round-half-even of 32767 * n / |n|), facing
 *        the view it was sampled from; may be NULL for bs_order
 *  rgb : 3 bytes of face colour; may be NULL for bs_order
 *  src : emission index dir * res^2 + py * res + px of the kept pixel; may be NULL
 *  n   : number of surfels (output of bs_sample_visible, input of bs_order)
 *  cap : capacity of each array in rows (input of bs_sample_visible)
 *  bbox_min, scale : world position = bbox_min + q / scale (output of
 *        bs_sample_visible; bs_order reads scale to convert radii). */
typedef struct {
    uint64_t *key;
    int16_t *nrm;
    uint8_t *rgb;
    uint32_t *src;
    uint64_t n;
    uint64_t cap;
    float bbox_min[3];
    double scale;
} bs_surfels;

/* Ordering options.
 *  seed, part_id : the random starting surfel (Sec. 3.2) is
 *      s = (w0 * n) >> 32, w0 = word 0 of Philox4x32-10(ctr = {part_id, 0, 0, 0},
 *      key = {seed & 0xffffffff, seed >> 32}), unless start >= 0.
 *  start     : explicit starting index (< n), or -1 for the Philox start.
 *  max_count : order only the first max_count surfels (0 = all); the result is
 *      exactly the prefix of the full ordering (Sec. 3.2 stops at a target count).
 *  variant 1 (the paper's randomised progressive sampling, Sec. 3.2): the remaining
 *      set is an index array with swap-with-last removal; round t draws sample_size
 *      positions with replacement, position u = (w * |R|) >> 32 with w = word 0 of
 *      Philox4x32-10(ctr = {part_id, t, u, 1}, key = seed), and appends the
 *      1 + t / sample_step distinct sampled points farthest from the surfels chosen
 *      before the round (ties to the lowest index), removing them in that order.
 *      rad2[k] is then the squared distance of pick k to every earlier pick. */
typedef struct {
    uint64_t seed;
    uint32_t part_id;
    int64_t start;
    uint64_t max_count;
    int32_t variant;       /* 0: exact greedy permutation; 1: the randomised sampler of Sec. 3.2 */
    uint32_t sample_size;  /* variant 1: random subset size per round, 1..256 (paper: ~200) */
    uint32_t sample_step;  /* variant 1: one more pick per round after every sample_step rounds
                              (paper: k = 500); 0 = always one pick per round */
} bs_order_opts;

/* bs_sample_visible -- initial surfel set (Sec. 3.1).
 * Quantises the mesh to 21-bit integers over its bounding cube, rasterises it
 * orthographically from each of `ndirs` directions at res x res pixels with an
 * integer rasteriser (pixel-centre sampling, shared edges covered once, nearest
 * depth wins, equal depth to the lower triangle id), emits one surfel per
 * covered pixel, merges surfels with identical positions (keeping the smallest
 * emission index) and writes them in ascending Morton order.
 *  mesh  : geometry (see bs_mesh: device, or host arrays the library uploads);
 *          dirs: HOST array of ndirs directions.
 *  res   : pixels per side, 1..BS_MAX_RES; ndirs: 1..BS_MAX_DIRS.
 *  out   : caller-owned device arrays of out->cap rows (nrm, rgb, src may be NULL).
 * Returns BS_OK with out->n, out->bbox_min, out->scale set; BS_EOVERFLOW with
 * out->n set and nothing written when n > cap (n <= ndirs * res^2 always);
 * BS_EINVAL for bad arguments, a non-finite vertex or a zero-extent mesh.
 * Synchronises `cuda_stream` before returning (the count is read back). */
bs_status bs_sample_visible(const bs_mesh *mesh, const bs_dir *dirs, int ndirs, int res,
                            bs_surfels *out, void *cuda_stream);

/* bs_sample_visible_batched -- bs_sample_visible for many meshes in one set of
 * launches (the per-node sampling of Sec. 3.4 run for a whole scene).
 *  meshes : HOST array of nparts meshes (device or host, see bs_mesh; 1 <= nparts <= 65535)
 *  res    : HOST array of nparts resolutions; dirs: HOST array of ndirs directions
 *           shared by all parts; the total pixel count must stay below 2^32
 *  out    : HOST array of nparts descriptors of caller-owned device arrays
 * Every part's surfels are bit-identical to a bs_sample_visible call on that part.
 * On return out[p].n, bbox_min and scale are set for every part; a part whose n
 * exceeds its cap is not written and the call returns BS_EOVERFLOW (the other parts
 * are written).  BS_EINVAL names the first invalid part.  Synchronises the stream. */
bs_status bs_sample_visible_batched(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs,
                                    int ndirs, bs_surfels *out, void *cuda_stream);

/* One part's results of bs_sample_order_batched.  The caller owns every array (HOST
 * arrays, or DEVICE ones when the call's out_on_device is nonzero).
 *  key, nrm, rgb, src : the sampled surfel records in canonical order, as
 *         bs_sample_visible writes them (cap rows; each may be NULL: not returned)
 *  perm, rad2, radius : the ordering and per-prefix radii, as bs_order writes them
 *         (m = min(max_count or n, n) entries; rad2 and radius may be NULL)
 *  cap  : rows of the surfel arrays (and entries of perm/rad2/radius)
 *  n, bbox_min, scale : out, as in bs_surfels */
typedef struct {
    uint64_t *key;
    int16_t *nrm;
    uint8_t *rgb;
    uint32_t *src;
    uint32_t *perm;
    int64_t *rad2;
    float *radius;
    uint64_t cap;
    uint64_t n;
    float bbox_min[3];
    double scale;
} bs_part_result;

/* bs_sample_order_batched -- the whole path for many meshes in one call: each mesh is
 * sampled as bs_sample_visible_batched samples it (Sec. 3.1) and its surfels ordered as
 * bs_order_batched orders them (Sec. 3.2 greedy permutation, Sec. 4.1 radii), with the
 * results written to the caller's arrays -- host to host for a caller without device
 * buffers: host meshes (on_device = 0) are uploaded by the library, and with
 * out_on_device = 0 every output is a host array.  The surfel records are read back
 * while the ordering runs.  Results are bit-identical to the two calls.
 *  meshes, res, dirs : as bs_sample_visible_batched (meshes may be host or device)
 *  opts  : HOST array of nparts ordering options; out: HOST array of nparts results
 * BS_EOVERFLOW (every out[p].n set, nothing ordered) when a part has more than cap
 * surfels; the other errors as the two calls.  Synchronises the stream: host outputs
 * are complete on return. */
bs_status bs_sample_order_batched(const bs_mesh *meshes, const int *res, int nparts, const bs_dir *dirs, int ndirs,
                                  const bs_order_opts *opts, bs_part_result *out, int out_on_device,
                                  void *cuda_stream);

/* ---- Bottom-up generation from child surfels (Sec. 3.4), each surfel drawn as the
 * oriented disc of Sec. 4.2. ---- */

/* One child's surfels splatted into a parent node. */
typedef struct {
    const uint64_t *key;   /* DEVICE: positions in this set's own 21-bit frame (bs_surfels.key) */
    const int16_t *nrm;    /* DEVICE: snorm16 normals, 3 per surfel */
    const uint8_t *rgb;    /* DEVICE: RGB8, 3 per surfel, or NULL (black) */
    const uint32_t *perm;  /* DEVICE or NULL: splat i is surfel perm[i] (a prefix of an ordering) */
    uint64_t n;            /* splats used from this set */
    float bbox_min[3];     /* the set's frame, as bs_sample_visible reported it */
    double scale;
    int64_t r2;            /* squared disc radius in the set's quantised units, >= 0 */
    uint32_t node;         /* the parent node (index into nodes[]) it is drawn into */
} bs_splat_set;

/* A parent node: its quantisation frame, raster resolution and outputs. */
typedef struct {
    float frame_min[3];    /* the node's frame: q = floor((x - frame_min) * scale) */
    double scale;          /* > 0 */
    int32_t res;           /* 1..BS_MAX_RES */
} bs_splat_node;

/* bs_sample_splats -- the initial surfel set of parent nodes rendered from child surfels
 * instead of triangles (Sec. 3.4 bottom-up), each surfel an oriented disc (Sec. 4.2).
 * A splat's centre and radius move to its node's frame by IEEE double operations in a
 * fixed order (t = q / s_set; t = bbox_min + t; t = t - frame_min; t = t * s_node;
 * floor, clamped to [0, 2^21 - 1]; radius sqrt(r2) / s_set * s_node, R2 = ceil(r^2),
 * at most 3 (2^21 - 1)^2).  For every direction (axis directions only) a pixel is
 * covered by a disc when its centre's ray meets the disc's plane within the radius
 * (exact integer test; discs seen edge-on are skipped); the nearest hit wins (ties to
 * the lower global splat index, sets concatenated in order) and emits its hit point
 * (floor), the disc normal turned toward the camera and its colour.  Emission index,
 * merge of equal positions and Morton order are those of bs_sample_visible; src holds
 * the emission index.
 *  sets : HOST array of nsets descriptors (0 <= nsets); nodes : HOST array of nnodes
 *  dirs : HOST array of ndirs axis directions; out : HOST array of nnodes caller-owned
 *         device surfel arrays (out[i].bbox_min / scale are set to node i's frame)
 * BS_EINVAL for a non-axis direction, a set naming a missing node, a bad resolution or
 * scale, NULL arrays, or more than 2^32 - 1 splats; BS_EOVERFLOW as for
 * bs_sample_visible_batched.  Synchronises the stream. */
bs_status bs_sample_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *nodes, int nnodes,
                           const bs_dir *dirs, int ndirs, bs_surfels *out, void *cuda_stream);

/* bs_parent_frames -- the frames parent nodes are sampled in, and the child prefixes they
 * draw (Sec. 3.4 bottom-up generation with Sec. 4.1's prefix rule).  Parent k's children
 * are c in [child_ofs[k], child_ofs[k + 1]); child c's quantisation cube is
 * [child_min[3c + a], child_min[3c + a] + (2^21 - 1) / child_scale[c]] on axis a.
 *  - frame_min[3k + a] = the smallest child_min over parent k's children (float32);
 *  - frame_scale[k] = (2^21 - 1) / E, E = the largest (child_min + (2^21 - 1) /
 *    child_scale) - frame_min over the children and axes (IEEE double, in this order):
 *    the largest child cube maps onto 2^21 - 1;
 *  - child_r2[c] = (int64)(h * h), h = (2^21 / parent_res[k]) * (child_scale[c] /
 *    frame_scale[k]): one pixel step of the parent's raster in child units.  A child is
 *    drawn with the shortest prefix of its exact ordering reaching every child surfel
 *    within sqrt(child_r2) (bs_prefix_for_radius_batched).
 * All arrays are HOST arrays owned by the caller: child_min 3 * nchildren, child_scale
 * nchildren, child_ofs nparents + 1 (child_ofs[0] = 0, non-decreasing), parent_res
 * nparents, outputs frame_min 3 * nparents, frame_scale nparents, child_r2 nchildren
 * (nchildren = child_ofs[nparents]).  Host arithmetic only; no device work.
 * BS_EINVAL for NULL arrays, a parent without children, a non-positive or non-finite
 * scale, a non-finite corner or a resolution outside 1..BS_MAX_RES. */
bs_status bs_parent_frames(const float *child_min, const double *child_scale, const uint64_t *child_ofs, int nparents,
                           const int32_t *parent_res, float *frame_min, double *frame_scale, int64_t *child_r2);

/* ---- Headless renders for image-space coverage checks (Sec. 4.1's claim that the
 * prefix of length p(r), drawn as discs of radius r, covers every pixel of the object;
 * the discs of Sec. 4.2).  No window or graphics API: the image is a device buffer. ---- */

/* bs_render_mesh -- the depth pass of bs_sample_visible for one direction: image (DEVICE,
 * res x res uint64, row py at py * res) receives depth << 32 | triangle index of the
 * nearest triangle covering each pixel centre, all ones where none does, in the mesh's
 * own frame (the frame bs_sample_visible reports).  Errors as bs_sample_visible.
 * Synchronises the stream. */
bs_status bs_render_mesh(const bs_mesh *mesh, const bs_dir *dir, int res, unsigned long long *image,
                         void *cuda_stream);

/* bs_render_splats -- the depth pass of bs_sample_splats for one node and one axis
 * direction: image (DEVICE, node->res^2 uint64) receives depth << 32 | global splat index
 * of the nearest disc covering each pixel centre, all ones where none does.  sets' node
 * fields are ignored.  BS_EINVAL for a non-axis direction or a bad node.  Stream-ordered
 * (returns after enqueueing). */
bs_status bs_render_splats(const bs_splat_set *sets, int nsets, const bs_splat_node *node, const bs_dir *dir,
                           unsigned long long *image, void *cuda_stream);

/* bs_order -- progressive ordering of one part (Sec. 3.2 goal; Sec. 4.1 radius).
 * Computes the exact greedy permutation (farthest-first traversal) of the
 * points s->key[0..n): perm[0] is the start index; perm[k] (k >= 1) is the
 * unchosen point whose squared distance to the nearest chosen point is largest,
 * ties to the lowest index; rad2[k] is that squared distance (int64, exact) and
 * rad2[0] = INT64_MAX.  Every prefix of length k >= 2 is then an r-net with
 * r^2 = rad2[k-1] (separation) covering all points within r^2 = rad2[k].
 * radius[k] = (float)(sqrt((double)rad2[k]) / s->scale), +inf for k = 0: the
 * splat radius in world units of the prefix of length k+1's covering.
 *  s    : device keys, s->n points (1..BS_MAX_POINTS); s->scale > 0 if radius != NULL.
 *  perm, rad2, radius : device outputs of m = min(max_count or n, n) entries;
 *         rad2 and radius may be NULL.
 * Duplicate keys are allowed: the remaining copies get rad2 = 0 and come last.
 * Stream-ordered: returns after enqueueing (no host synchronisation). */
bs_status bs_order(const bs_surfels *s, const bs_order_opts *opts, uint32_t *perm, int64_t *rad2,
                   float *radius, void *cuda_stream);

/* ---- Prefix selection at render time (Sec. 4.1). ---- */

/* r_m^2: the median squared nearest-neighbour distance inside the first pm surfels
 * of an ordering (the lower median, i.e. the ceil(pm/2)-th smallest; 0 for pm < 2).
 * s->key and perm (at least pm entries) are device arrays; *rm2 is written on the
 * host.  O(pm^2) work; pm <= min(n, 65536).  Synchronises the stream. */
bs_status bs_prefix_median_nn(const bs_surfels *s, const uint32_t *perm, uint64_t pm, int64_t *rm2,
                              void *cuda_stream);

/* The shortest prefix of an exact ordering whose surfels, drawn with radius r,
 * reach every point of the part: the smallest p >= 1 with rad2[p] <= r2 (a prefix
 * of length p reaches every point within sqrt(rad2[p])), or m when no ordered entry
 * qualifies.  rad2: device output of bs_order (variant 0), m entries; *p on the
 * host.  Synchronises the stream. */
bs_status bs_prefix_for_radius(const int64_t *rad2, uint64_t m, int64_t r2, uint64_t *p, void *cuda_stream);

/* bs_prefix_for_radius for nparts orderings in one launch (the children of the parent
 * nodes of Sec. 3.4's bottom-up generation).  rad2: HOST array of device pointers; m, r2:
 * HOST arrays; p: HOST output.  r2_at (HOST, may be NULL) receives rad2[min(p, m - 1)]:
 * the squared distance within which the prefix of length p reaches every point (exact for
 * p < m, an upper bound when no ordered entry qualifies).  Synchronises the stream. */
bs_status bs_prefix_for_radius_batched(const int64_t *const *rad2, const uint64_t *m, const int64_t *r2, int nparts,
                                       uint64_t *p, int64_t *r2_at, void *cuda_stream);

/* The paper's estimate of that prefix length, p(r) = pm * (r_m / r)^2, from the
 * squared radii rm2 = r_m^2 and r2 = r^2 (same units); +inf for r2 <= 0. */
double bs_prefix_estimate(uint64_t pm, int64_t rm2, int64_t r2);

/* bs_order_batched -- bs_order for many independent parts in one persistent
 * launch (the per-node preprocessing of Sec. 3.4 run for a whole scene).
 *  parts : HOST array of nparts descriptors (device keys inside).
 *  opts  : HOST array of nparts options (one per part).
 *  perm, rad2, radius : HOST arrays of nparts DEVICE pointers (rad2/radius
 *          arrays, or their entries, may be NULL).
 * Results are bit-identical to calling bs_order on each part.  Stream-ordered. */
bs_status bs_order_batched(const bs_surfels *parts, int nparts, const bs_order_opts *opts,
                           uint32_t *const *perm, int64_t *const *rad2, float *const *radius,
                           void *cuda_stream);

/* bs_order_noalloc -- bs_order for callers that may not allocate device memory.
 * The paper has no counterpart: this entry point exists for library users.  A
 * plugin or render thread running inside a host application that owns the GPU
 * memory budget, or a real-time loop that cannot afford an allocation that may
 * block or fail, cannot let the library call cudaMalloc or grow a memory pool.
 * This call computes exactly what bs_order computes (same arguments, same
 * bit-identical outputs) but takes all of its scratch from one fixed array of
 * about 1.1 MB that the library reserves in device memory on every GPU where it
 * is loaded, held until the process exits.  It calls no allocating routine.
 *  - Parts of at most BS_NOALLOC_MAX_POINTS points; larger ones return
 *    BS_EOVERFLOW with a message and nothing is launched.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any stream
 *    capture.
 *  - Every call shares the one array: calls whose work can overlap on the GPU
 *    (different streams, or different host threads, without ordering between
 *    them) race on it and give wrong results.  Serialise them on one stream.
 * Stream-ordered like bs_order. */
#define BS_NOALLOC_MAX_POINTS 65536u
bs_status bs_order_noalloc(const bs_surfels *s, const bs_order_opts *opts, uint32_t *perm, int64_t *rad2,
                           float *radius, void *cuda_stream);

/* ---- Serving: continuous batching of ordering requests (Sec. 3.4 at scale). ---- */
typedef struct bs_server bs_server;

/* Creates a server on the current CUDA device that keeps request state on the
 * device, admitting requests while their scratch fits in device_budget_bytes.
 * max_inflight bounds requests resident on the device at once (0 = 4096).
 * Returns NULL and sets *st on failure. */
bs_server *bs_server_create(uint64_t device_budget_bytes, int max_inflight, bs_status *st);

/* Queues one ordering request.  key: HOST array of n packed positions (copied
 * before return); scale: as in bs_surfels (for radius).  *ticket receives an id
 * for bs_server_poll.  BS_EBUSY if the host queue is full; BS_ENOMEM if the
 * request alone exceeds the device budget. */
bs_status bs_server_submit(bs_server *srv, const uint64_t *key, uint64_t n, double scale,
                           const bs_order_opts *opts, uint64_t *ticket);

/* If the ticket's result is ready, copies it to the HOST arrays perm/rad2/radius
 * (m entries; rad2/radius may be NULL) and releases it.  With perm == NULL the
 * call only reports the status (BS_OK when ready) and keeps the result.
 * BS_ENOTREADY while the request is queued or running; BS_EINVAL for an
 * unknown or already collected ticket; BS_ECANCELED for a cancelled one; the
 * request's own error for a failed one (BS_ENOMEM when its launch could not get
 * device memory, BS_ETIMEOUT when it stayed on the device longer than the
 * server's timeout).  The server's own host thread admits, launches and retires
 * requests; polling does not drive it. */
bs_status bs_server_poll(bs_server *srv, uint64_t ticket, uint32_t *perm, int64_t *rad2, float *radius);

/* Per-ticket timestamps in seconds on the server's monotonic clock:
 * t[0] submit, t[1] admitted to the device, t[2] finished on the device.
 * Valid after bs_server_poll returned BS_OK for the ticket. */
bs_status bs_server_times(bs_server *srv, uint64_t ticket, double t[3]);

/* Cancels a request.  A queued one leaves the queue at once; one on the device is
 * dropped when its launch ends (the kernel is not interrupted), which then releases
 * its device memory and budget; a finished, uncollected result is dropped.  Polling
 * the ticket afterwards returns BS_ECANCELED.  BS_EINVAL for an unknown ticket or a
 * request that already failed or was collected. */
bs_status bs_server_cancel(bs_server *srv, uint64_t ticket);

/* Waits for all in-flight work, frees device memory and the server. */
void bs_server_destroy(bs_server *srv);

/* ---- Scene-scale workload (the production-line scene of Sec. 5). ---- */

/* Generates nparts CAD-like parts (nboxes boxes of 2x2-quad faces and ncyl 32-segment
 * cylinders each) on the device from a seed, concatenated in the given order into
 * one mesh: vertices xyz (nparts * (54 nboxes + 98 ncyl) * 3 float32), triangles
 * (nparts * (48 nboxes + 192 ncyl) * 3 uint32; indices into that mesh, or into each
 * part's own vertices when local_indices != 0), per-face RGB8 (all DEVICE, owned by the
 * caller).  part_ids, lines, slots: HOST arrays (the part's Philox counter, its line
 * and its slot in the line: placement + (slot * dx, line * dy, 0)).  size_table
 * (1024 log-uniform sizes), cos32 and sin32 (32-segment ring) are HOST tables.
 * Every parameter comes from Philox4x32-10(ctr = {part_lo, part_hi, primitive, k},
 * key = seed) and every vertex from single float32 operations in a fixed order, so a
 * host implementation reproduces the mesh bit for bit.  Stream-ordered.  BS_EINVAL for
 * NULL arrays, negative counts, nboxes == ncyl == 0 or 2^32 vertices or more. */
bs_status bs_scene_generate(uint64_t seed, const uint64_t *part_ids, const int32_t *lines, const int32_t *slots,
                            int nparts, int nboxes, int ncyl, const float *size_table, const float *cos32,
                            const float *sin32, float dx, float dy, int local_indices, float *xyz, uint32_t *tri,
                            uint8_t *rgb, void *cuda_stream);

/* Launch-shape knobs for the autotuner (results never depend on them):
 *  "order_threads"      threads per ordering CTA (64, 128, 256, 512, 1024; 0 = auto)
 *  "order_ctas_per_sm"  cap on resident ordering CTAs per SM (0 = occupancy limit)
 *  "order_quarters"     batched rounds launch in 1024-thread CTAs that order the largest
 *                       parts on the whole CTA, then split into four 256-thread quarters
 *                       taking one part each: 0 = when a cost model predicts a gain,
 *                       1 = never, 2 = always (parts over 524,288 points stay whole)
 *  "order_full_parts"   k > 0: the k largest parts run on whole CTAs before the quarters
 *                       (0 = the cost model decides)
 *  "order_slots"        parts a 1024-thread CTA orders at once after its whole-CTA parts:
 *                       2, 4 (the default; 0 restores it) or 8 slots of 512, 256 or 128
 *                       threads taking parts of at most 1M, 512k or 256k points (8 slots
 *                       only when no part of the launch uses the sampler, variant 1)
 *  "server_slots"       launches a server created afterwards keeps in flight (1..256,
 *                       16 by default; each holds 64 MB of pinned result staging)
 *  "server_timeout_ms"  a request of a server created afterwards that is still on the
 *                       device this long after its launch fails with BS_ETIMEOUT
 *                       (0 = no timeout, the default)
 *  "fail_next_allocs"   the library's next k device-scratch allocations fail as if the
 *                       device were out of memory (error-path tests; host-side only)
 *  "pool_keep_mb"       freed scratch the library's per-device memory pool keeps for the
 *                       next call, in MiB (65536 by default; lowering it trims the pool)
 *  "order_cluster"      parts of at least "order_cluster_min" points (exact ordering)
 *                       split over a thread-block cluster of this many CTAs, one SM each:
 *                       1 = never (default: measured slower on GB300 at every size),
 *                       0 = automatic size (up to 16, one CTA per 32,768 points at most),
 *                       2..16 = that size (capped by the part's size)
 *  "order_cluster_min"  smallest part ordered on a cluster (262,144 points by default)
 *  "order_algo"         2 = exact multi-pick rounds (default), 1 = one pick per step
 *  "kernel_timing"      1 = record CUDA events around internal kernels (bs_last_launch_ms)
 * Process-wide; BS_EINVAL for an unknown name or value. */
bs_status bs_set_tuning(const char *name, int value);

/* Device time in milliseconds of the most recent launch of an internal kernel,
 * measured with CUDA events recorded on the launch's own stream around that one
 * kernel.  Recording is off until bs_set_tuning("kernel_timing", 1).  kernel:
 * "order_init", "order_loop" or "order_radius".  Waits for the stop event.
 * BS_ENOTREADY if no timed launch happened yet; BS_EINVAL for an unknown name. */
bs_status bs_last_launch_ms(const char *kernel, double *ms);

/* Message of the last failure on the calling thread ("" if none). */
const char *bs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BS_H */
