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
//   k_order_rounds  persistent (parts taken from atomic counters): exact multi-pick
//                 rounds -- gather the candidates above a threshold, one warp runs
//                 the greedy on them, every pick of the round applied in one pruned
//                 sweep (super-group, group and bucket boxes).  The largest parts of a
//                 launch run on whole CTAs; with quarter mode a 1024-thread CTA then
//                 takes four more parts at once on 256-thread quarters.  Writes the
//                 radii and the part's completion flag at the end of each part.
//   k_order_loop  the same greedy with one pick per step (order_algo 1): per step a
//                 block argmax over the group records, a scan of group boxes against
//                 the new point, and a warp per touched group updating its buckets.
//   k_radius      radius[k] = sqrt(rad2[k]) / scale in IEEE double, as float (after
//                 k_order_loop).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "bs_internal.cuh"

namespace cg = cooperative_groups;

namespace bs {

constexpr uint32_t FULL = 0xffffffffu;

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
            if (P.variant == 1) {
                P.R[i] = i;
                P.pos[i] = i;
            }
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

// ---------------------------------------------------------------------------
// Exact multi-pick rounds.  A round takes a threshold tau <= D1 (the current
// maximum) and gathers every unchosen point i with D[i] > tau, or D[i] == tau and
// i < icut, into a candidate set C (at most CAP points).  Every point outside C is
// below (tau, icut) in the (D, lowest index) order, and D only decreases, so while
// the best candidate (D updated by this round's picks) is still above (tau, icut)
// it is exactly the greedy's next pick.  One warp runs that small greedy; then all
// picks are applied to the whole part at once.  A fourth level of super-groups
// (32 groups, 32768 points) prunes the apply sweep of large parts.
//   sgkey = (D+1) << 15 | (32767 - i_in_supergroup);   top = (D+1) << 8 | (255 - sg)
// ---------------------------------------------------------------------------
constexpr int CAP_BITS = 7;
constexpr int CAP = 1 << CAP_BITS;  // candidates per round (CAP / 32 per lane of the simulating warp)
constexpr int OFF_BITS = 32 - CAP_BITS;  // 32-bit simulation keys: (D - tau + 1) << CAP_BITS | slot
constexpr int CPL = CAP / 32;
constexpr int MAXP = 64;     // picks per round (pick sets are 64-bit masks)
constexpr int MAX_SG = 192;  // super-groups: BS_MAX_POINTS / 32768
constexpr int TIE_GROUPS = 8;  // groups a tie window may span
constexpr int SMAX = 256;      // variant 1: largest random subset per round
constexpr int SPL = SMAX / 32;
constexpr int NB_SMEM = 2048;  // parts with at most this many buckets keep bucket records in shared memory
constexpr size_t SMEM_LIMIT = 227 * 1024 - 128;  // dynamic shared memory per CTA: the opt-in limit less the static part
// Quarter mode: a 1024-thread CTA runs four parts at once, 256 threads each, so four
// independent latency chains share the SM (one part's single simulating warp overlaps
// the others' sweeps).  A quarter takes parts of at most Q_SG super-groups.
constexpr int QT = 256;
constexpr int LB = 4;          // buckets whose loads are issued together in the gather and apply sweeps
constexpr int Q_SG = 16;       // 524,288 points
constexpr int Q_NB = 1024;     // bucket records in shared memory up to 32,768 points
// Other slot counts per 1024-thread CTA (bs_set_tuning "order_slots"): the largest part a
// slot takes (super-groups) for 2, 4 and 8 slots.
__host__ __device__ constexpr int slot_sg(int slots) { return slots == 2 ? 32 : slots == 4 ? Q_SG : 8; }

// Per-part shared state of the rounds kernel (one per part slot).
template <int SG>
struct RoundsSm {
    uint64_t sgkey[SG], sglo[SG], sghi[SG], sgmask[SG];
    uint32_t sglist[SG], heavy[SG];
    uint64_t ck[CAP];
    int64_t cd[CAP];
    uint32_t ci[CAP];
    uint64_t pk[MAXP];
    int64_t pd[MAXP];
    uint32_t pi[MAXP];
    int32_t px[MAXP], py[MAXP], pz[MAXP];  // the picks' coordinates, unpacked
    uint32_t sc[SMAX];   // variant 1: the round's sample (index), sorted by index
    int64_t sd[SMAX];    //            its distance to the chosen set
    uint64_t sk[SMAX];   //            its position
    uint32_t ppos[MAXP], tail[MAXP];
    uint32_t part, ccnt, gcnt, sgcnt, npick, icut;  // gather counters (reset when the previous round applies)
    uint32_t agcnt, asgcnt, nheavy;                 // apply counters (reset when the round's picks are written)
    uint32_t gnext, anext;  // the next listed group a warp takes in the gather and in the bucket updates
    int shift;
    int64_t tieD;
    // cluster mode: this CTA's best (top key) and the leader's candidate counters, one
    // per gather attempt parity (an attempt's counter is reset while the other is in use)
    uint64_t ctop;
    uint32_t cc2[2];
};

// Bytes of one part slot: the state, then bucket (bkey, blo, bhi: nbcap each) and group
// (gkey, glo, ghi: ngcap each; glist: ngcap u32) records.
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
template <int SG>
__host__ __device__ constexpr size_t slot_bytes(int nbcap, int ngcap) {
    return align16(sizeof(RoundsSm<SG>)) + (size_t)nbcap * 24 + align16((size_t)ngcap * 28);
}

// full-mode bucket capacity for a launch whose largest part has ngmax groups; nbmin =
// buckets of its smallest whole-CTA part (0: unknown): when that part has more than
// NB_SMEM buckets no whole-CTA part keeps bucket records in shared memory, and the
// space is left to the candidate matrix and the L1 cache
static int rounds_nbsm(int ngmax, int nbmin = 0) {
    return nbmin <= NB_SMEM && slot_bytes<MAX_SG>(NB_SMEM, ngmax) <= SMEM_LIMIT ? NB_SMEM : 0;
}

// Candidate matrix of a whole 1024-thread CTA: row r holds, for every candidate c of the
// round, min(2^32 - 1, d(r, c) - tau + 1), or 0 when d(r, c) < tau or r == c -- the
// value the candidate greedy takes the minimum with when r is picked.  Rows of CAP
// entries after the part's records, as many as the shared memory holds (at most CAP);
// the matrix serves the rounds whose candidates fit it.
constexpr size_t MAT_ROW = (size_t)CAP * 4;
__host__ __device__ constexpr int mat_rows(int nbcap, int ngcap) {
    return slot_bytes<MAX_SG>(nbcap, ngcap) >= SMEM_LIMIT
               ? 0
               : ((SMEM_LIMIT - slot_bytes<MAX_SG>(nbcap, ngcap)) / MAT_ROW >= (size_t)CAP
                      ? CAP
                      : (int)((SMEM_LIMIT - slot_bytes<MAX_SG>(nbcap, ngcap)) / MAT_ROW));
}

__device__ __forceinline__ void part_sync(int bar, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}

// The next work item for the calling warp from a shared counter (lane 0 takes it).
__device__ __forceinline__ uint32_t take_next(uint32_t *ctr, int lane) {
    uint32_t v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1u);
    return __shfl_sync(0xffffffffu, v, 0);
}


// L2 eviction priority as a per-access cache hint (a policy operand of the load or store)
__device__ __forceinline__ uint64_t l2_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t ld_hint_u64(const void *a, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint_u64(void *a, uint64_t v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" :: "l"(a), "l"(v), "l"(pol));
}

// A box with its corners unpacked.
struct Box {
    int32_t lx, ly, lz, hx, hy, hz;
};
__device__ __forceinline__ Box unpack_box(uint64_t lo, uint64_t hi) {
    return Box{(int32_t)pos_x(lo), (int32_t)pos_y(lo), (int32_t)pos_z(lo),
               (int32_t)pos_x(hi), (int32_t)pos_y(hi), (int32_t)pos_z(hi)};
}
// squared distance from (x, y, z) to the box, 0 inside (the same value as box_dist2)
__device__ __forceinline__ int64_t box_dist2_xyz(const Box &b, int32_t x, int32_t y, int32_t z) {
    const int32_t dx = max(max(b.lx - x, x - b.hx), 0);
    const int32_t dy = max(max(b.ly - y, y - b.hy), 0);
    const int32_t dz = max(max(b.lz - z, z - b.hz), 0);
    return (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
}

// bit t set if pick t may lower a D inside the box (whose largest D is maxD) or lies
// inside the index range `own` at granularity own_shift; px/py/pz the picks' coordinates
__device__ __forceinline__ uint64_t pick_mask(uint32_t np, const uint32_t *pi, const int32_t *px, const int32_t *py,
                                              const int32_t *pz, uint64_t allow, uint32_t own_shift, uint32_t own,
                                              uint64_t lo, uint64_t hi, int64_t maxD) {
    const int lane = threadIdx.x & 31;
    const Box b = unpack_box(lo, hi);
    bool ra = false, rb = false;
    const uint32_t ta = lane, tb = lane + 32;
    if (ta < np && ((allow >> ta) & 1ull))
        ra = (pi[ta] >> own_shift) == own || box_dist2_xyz(b, px[ta], py[ta], pz[ta]) < maxD;
    if (tb < np && ((allow >> tb) & 1ull))
        rb = (pi[tb] >> own_shift) == own || box_dist2_xyz(b, px[tb], py[tb], pz[tb]) < maxD;
    return (uint64_t)__ballot_sync(0xffffffffu, ra) | ((uint64_t)__ballot_sync(0xffffffffu, rb) << 32);
}

// One part ordered by TP threads (thread tid of them, warp-aligned) that synchronise on
// named barrier `bar`; S and the record arrays are this part slot's shared memory.  Warp
// simw runs the serial steps (the candidate greedy, the tie window, the sampler's
// choice): the quarters of a CTA pass different warps so that their serial steps issue
// from different schedulers of the SM.
//
// Cluster mode (CL): the part is split over the csize CTAs of a thread-block cluster.
// CTA crank owns super-groups [sg0, sg1) -- their points, buckets and groups -- and
// applies every pick of a round to them; candidates are gathered into the leader's
// (rank 0) shared memory through distributed shared memory, the leader runs the
// candidate greedy and the others copy its picks.  Every control decision (threshold,
// retry, pick count, loop exit) is taken by every CTA from the same values read after
// the same cluster barrier, so all CTAs pass the same sequence of barriers.  Only the
// exact ordering (variant 0) runs in cluster mode, with bucket records in global memory.
template <int TP, int SG, bool CL = false>
__device__ __forceinline__ void rounds_part(const PartDesc &P, RoundsSm<SG> &Sm, unsigned char *slot, int nbsm,
                                            int ngcap, int tid, int bar, int simw, int crank = 0, int csize = 1,
                                            uint32_t *mat = nullptr, int matrows = 0) {
    static_assert(TP >= CAP, "the candidate sort needs one thread per candidate");
    // the candidate matrix: rows of MS entries, CAP on whole 1024-thread CTAs and 64 in
    // part slots (rounds of at most 64 candidates there: the slots share the CTA's memory)
    constexpr bool MATRIX = !CL;
    // parts on fewer than 1024 threads (part slots, and the CTAs of smaller parts) read
    // and write their distances and keys with an L2 evict-first hint: the many parts of
    // such launches stream through L2, and the hint leaves the lines of the large parts
    // on 1024-thread CTAs (the longest chains, often running alongside) in place longer
    constexpr bool STREAM = TP < 1024 && !CL;
    const uint64_t pol = STREAM ? l2_first_policy() : 0ull;
    constexpr int MS = TP == 1024 ? CAP : 64;
    constexpr int CPLM = MS / 32;
    // the sampler (variant 1) sorts its sample with one thread per entry: slots of fewer
    // than SMAX threads order exact parts only (the host routes sampler parts elsewhere)
    constexpr bool SAMPLER = TP >= SMAX;
    constexpr int NW = TP / 32;
    const int lane = tid & 31, warp = tid >> 5;
    uint64_t *s_bkey = (uint64_t *)(slot + align16(sizeof(RoundsSm<SG>)));
    uint64_t *s_blo = s_bkey + nbsm;
    uint64_t *s_bhi = s_bkey + 2 * nbsm;
    uint64_t *s_gkey = s_bkey + 3 * nbsm;
    uint64_t *s_glo = s_gkey + ngcap;
    uint64_t *s_ghi = s_gkey + 2 * ngcap;
    uint32_t *s_glist = (uint32_t *)(s_gkey + 3 * ngcap);
    const uint32_t ng = P.ng, ns = (ng + 31) / 32;
    const uint32_t n = P.n, nb = P.nb, m = P.m;
    const uint64_t *__restrict__ key = P.key;
    int64_t *__restrict__ Dg = P.D;
    // this CTA's super-groups (all of them outside cluster mode)
    const uint32_t sg0 = CL ? (uint32_t)(((uint64_t)crank * ns) / (uint32_t)csize) : 0u;
    const uint32_t sg1 = CL ? (uint32_t)(((uint64_t)(crank + 1) * ns) / (uint32_t)csize) : ns;
    const uint32_t og0 = sg0 * 32, og1 = min(ng, sg1 * 32);  // this CTA's groups
    const bool leader = !CL || crank == 0;
    cg::cluster_group cl = cg::this_cluster();
    // the leader's candidate state (this CTA's own outside cluster mode)
    RoundsSm<SG> &Ld = CL ? *cl.map_shared_rank(&Sm, 0) : Sm;
    uint32_t attempt = 0;  // gather attempts of this part (cluster mode: picks the leader's counter)
    // a part of one super-group (most parts of a batch) keeps no super-group key: every
    // warp takes it from the group keys when it looks for the round's maximum, so the
    // key update and its barrier at the end of the round are skipped
    const bool one_sg = !CL && ns == 1 && P.variant == 0;
    // bucket records: shared memory when they fit (generic pointers either way)
    const bool bsm = !CL && nb <= (uint32_t)nbsm;
    if constexpr (MATRIX && TP == 1024) {
        // a whole-CTA part whose bucket records stay in global memory: the candidate
        // matrix may take their shared-memory space when that holds more rows
        const int brows = (int)min((size_t)CAP, (size_t)nbsm * 24 / MAT_ROW);
        if (!bsm && brows > matrows) {
            mat = (uint32_t *)s_bkey;
            matrows = brows;
        }
    }
    uint64_t *bkey = bsm ? s_bkey : P.bkey;
    const uint64_t *blo_p = bsm ? s_blo : P.blo;
    const uint64_t *bhi_p = bsm ? s_bhi : P.bhi;
    for (uint32_t g = og0 + tid; g < og1; g += TP) {
        s_gkey[g] = P.gkey[g];
        s_glo[g] = P.glo[g];
        s_ghi[g] = P.ghi[g];
    }
    if (bsm) {
        for (uint32_t b = tid; b < nb; b += TP) {
            s_bkey[b] = P.bkey[b];
            s_blo[b] = P.blo[b];
            s_bhi[b] = P.bhi[b];
        }
    }
    if (tid == 0) {
        if (leader) {
            P.perm[0] = P.start;
            P.rad2[0] = INT64_MAX;
        }
        Sm.shift = 3;
        Sm.tieD = -2;
        Sm.ccnt = 0; Sm.gcnt = 0; Sm.sgcnt = 0; Sm.icut = 0xffffffffu;
        Sm.gnext = 0; Sm.anext = 0;
        Sm.cc2[0] = 0; Sm.cc2[1] = 0;
        if (SAMPLER && !CL && P.variant == 1) {  // remove the start from the remaining set (swap with the last)
            const uint32_t y = P.R[n - 1];
            P.R[P.start] = y;
            P.pos[y] = P.start;
        }
    }
    part_sync(bar, TP);
    uint32_t round_t = 0;
    for (uint32_t sg = sg0 + warp; sg < sg1; sg += NW) {
        const uint32_t g = sg * 32 + lane;
        const bool vg = g < ng;
        const uint64_t gk = vg ? s_gkey[g] : 0ull;
        const uint64_t cand = vg ? (((gk >> 10) << 15) | (uint64_t)(32767 - (lane * 1024 + (1023 - (int)(gk & 1023))))) : 0ull;
        const uint64_t sk = warp_max_u64(cand);
        const uint64_t lo = vg ? s_glo[g] : ~0ull, hi = vg ? s_ghi[g] : 0ull;
        const uint32_t lx = __reduce_min_sync(FULL, vg ? pos_x(lo) : 0xffffffffu);
        const uint32_t ly = __reduce_min_sync(FULL, vg ? pos_y(lo) : 0xffffffffu);
        const uint32_t lz = __reduce_min_sync(FULL, vg ? pos_z(lo) : 0xffffffffu);
        const uint32_t hx = __reduce_max_sync(FULL, vg ? pos_x(hi) : 0u);
        const uint32_t hy = __reduce_max_sync(FULL, vg ? pos_y(hi) : 0u);
        const uint32_t hz = __reduce_max_sync(FULL, vg ? pos_z(hi) : 0u);
        if (lane == 0) {
            Sm.sgkey[sg] = sk;
            Sm.sglo[sg] = pack_pos(lx, ly, lz);
            Sm.sghi[sg] = pack_pos(hx, hy, hz);
        }
    }
    part_sync(bar, TP);
    uint32_t k = 1;
    while (k < m) {
      if (SAMPLER && !CL && P.variant == 1) {
       if constexpr (SAMPLER) {
        // (S1) the round's random subset of the remaining set R[0, n - k)
        const uint32_t L = n - k, S = P.sample_size;
        uint32_t c = 0, slot = 0;
        int64_t cd = 0;
        uint64_t ck = 0;
        if (tid < S) {
            const uint32_t ctr[4] = {P.part_id, round_t, (uint32_t)tid, 1u};
            const uint32_t kk[2] = {(uint32_t)P.seed, (uint32_t)(P.seed >> 32)};
            uint32_t w[4];
            philox4x32_10(ctr, kk, w);
            c = P.R[(uint32_t)(((uint64_t)w[0] * L) >> 32)];
            Sm.sc[tid] = c;
            cd = Dg[c];
            ck = key[c];
        }
        part_sync(bar, TP);
        // (S2) sorted by index (equal entries adjacent): slot = #smaller + #equal before
        if (tid < S) {
            for (uint32_t u = 0; u < S; ++u) {
                const uint32_t o = Sm.sc[u];
                slot += (o < c || (o == c && u < tid)) ? 1u : 0u;
            }
        }
        part_sync(bar, TP);
        if (tid < S) {
            Sm.sc[slot] = c;
            Sm.sd[slot] = cd;
            Sm.sk[slot] = ck;
        }
        part_sync(bar, TP);
        // (S3) the m_t = 1 + t / step distinct samples farthest from the chosen set
        //      (distances as of the round start), ties to the lowest index
        if (warp == simw) {
            uint32_t cs[SPL];
            int64_t ds[SPL];
            bool live[SPL];
#pragma unroll
            for (int u = 0; u < SPL; ++u) {
                const uint32_t sl = lane + 32 * u;
                live[u] = sl < S;
                cs[u] = live[u] ? Sm.sc[sl] : 0u;
                ds[u] = live[u] ? Sm.sd[sl] : 0;
            }
            const uint32_t mt = 1u + (P.sample_step ? round_t / P.sample_step : 0u);
            const uint32_t budget = min(min(mt, (uint32_t)MAXP), m - k);
            uint32_t np = 0;
            while (np < budget) {
                uint64_t kmax = 0;
#pragma unroll
                for (int u = 0; u < SPL; ++u)
                    if (live[u]) kmax = max(kmax, ((uint64_t)(ds[u] + 1) << 8) | (uint64_t)(255 - (lane + 32 * u)));
                const uint64_t best = warp_max_u64(kmax);
                if (best == 0) break;
                const uint32_t sl = 255u - (uint32_t)(best & 255u);
                const uint32_t cb = Sm.sc[sl];
                if (lane == 0) {
                    Sm.pi[np] = cb;
                    Sm.pk[np] = Sm.sk[sl];
                    Sm.pd[np] = (int64_t)(best >> 8) - 1;
                }
                ++np;
#pragma unroll
                for (int u = 0; u < SPL; ++u)
                    if (cs[u] == cb) live[u] = false;
            }
            if (lane == 0) Sm.npick = np;
        }
        part_sync(bar, TP);
        const uint32_t npk = Sm.npick;
        // (S4) rad2 of a pick: its distance to every earlier pick; gather what the removal needs
        int64_t r2 = 0;
        if (tid < npk) {
            r2 = Sm.pd[tid];
            const uint64_t q = Sm.pk[tid];
            for (uint32_t u = 0; u < tid; ++u) r2 = min(r2, dist2(q, Sm.pk[u]));
            Sm.ppos[tid] = P.pos[Sm.pi[tid]];
            Sm.tail[tid] = P.R[L - npk + tid];
        }
        part_sync(bar, TP);
        if (tid < npk) Sm.pd[tid] = r2;
        // (S5) remove the picks in pick order, each swapped with the current last entry;
        //      the last entries all lie in the tail window [L - npk, L) held in Sm.tail
        if (tid == 0) {
            const uint32_t base = L - npk;
            for (uint32_t q = 0; q < npk; ++q) {
                const uint32_t pp = Sm.ppos[q];
                const uint32_t y = Sm.tail[L - q - 1 - base];
                if (pp >= base) {
                    Sm.tail[pp - base] = y;
                } else {
                    P.R[pp] = y;
                    P.pos[y] = pp;
                }
                for (uint32_t r = q + 1; r < npk; ++r)
                    if (Sm.pi[r] == y) Sm.ppos[r] = pp;
            }
        }
        ++round_t;
        part_sync(bar, TP);
       }
      } else {
        // (1) current maximum (every warp computes it; no barrier needed).  Cluster mode:
        //     each CTA's best over its own super-groups, combined after a cluster barrier
        //     (super-group indices are global, so the largest key is the global argmax)
        uint64_t top = 0, sk1 = 0;
        if (one_sg) {
            const uint64_t gk = lane < (int)ng ? s_gkey[lane] : 0ull;
            sk1 = warp_max_u64(lane < (int)ng ? (((gk >> 10) << 15) | (uint64_t)(32767 - (lane * 1024 + (1023 - (int)(gk & 1023)))))
                                              : 0ull);
            top = ((sk1 >> 15) << 8) | 255ull;
        } else {
            for (uint32_t sg = sg0 + lane; sg < sg1; sg += 32) top = max(top, ((Sm.sgkey[sg] >> 15) << 8) | (uint64_t)(255 - sg));
            top = warp_max_u64(top);
        }
        if constexpr (CL) {
            if (tid == 0) Sm.ctop = top;
            cl.sync();
            top = warp_max_u64(lane < csize ? cl.map_shared_rank(&Sm, lane)->ctop : 0ull);
        }
        const int64_t D1 = (int64_t)(top >> 8) - 1;
        const uint32_t sgj = 255u - (uint32_t)(top & 255u);
        // (2) threshold: tau = D1 (1 - 2^-shift); when more than CAP points tie at D1, a tie
        //     window instead: tau = D1 and an index cut (the lowest-index tied points fit)
        const int shift = Sm.shift;
        const bool tie = D1 == Sm.tieD;
        const int64_t tau = tie ? D1 : D1 - (D1 >> shift);
        // (3) gather the candidates (the gather counters were reset before the last barrier)
        if (tie) {
            // D1 points in index order from j on, over up to TIE_GROUPS groups holding D1
            // points, while they fit; icut = first index left out (no D1 point lies below j).
            // Cluster mode: the leader walks the groups of every CTA (group keys through
            // distributed shared memory, bucket keys and distances from L2)
            if (leader && warp == simw) {
                // owner of a super-group in cluster mode: the CTA whose range holds it
                auto owner = [&](uint32_t sg) {
                    int r = 0;
                    while (r + 1 < csize && sg >= (uint32_t)(((uint64_t)(r + 1) * ns) / (uint32_t)csize)) ++r;
                    return r;
                };
                const uint64_t sgkj = CL ? cl.map_shared_rank(&Sm, owner(sgj))->sgkey[sgj] : (one_sg ? sk1 : Sm.sgkey[sgj]);
                const uint32_t j = sgj * 32768u + (32767u - (uint32_t)(sgkj & 32767u));
                uint32_t cnt = 0, icut = n, used = 0;
                bool full = false;
                for (uint32_t g0 = j >> 10; g0 < ng && !full && used < TIE_GROUPS; ++g0) {
                    const uint64_t gk0 = CL ? cl.map_shared_rank(s_gkey, owner(g0 >> 5))[g0] : s_gkey[g0];
                    if ((int64_t)(gk0 >> 10) - 1 < tau) continue;
                    ++used;
                    const uint32_t b = g0 * 32 + lane;
                    const uint64_t bk = (b < nb && b >= (j >> 5)) ? (CL ? __ldcg(&bkey[b]) : bkey[b]) : 0ull;
                    uint32_t mask = __ballot_sync(FULL, (int64_t)(bk >> 5) - 1 >= tau);
                    while (mask) {
                        const int bb = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const uint32_t i = (g0 * 32 + bb) * 32 + lane;
                        const int64_t d = i < n ? (CL ? __ldcg(&Dg[i]) : Dg[i]) : -1;
                        const uint64_t ki = i < n ? key[i] : 0ull;
                        const bool c = d >= tau;
                        const uint32_t cm = __ballot_sync(FULL, c);
                        if (cnt + __popc(cm) > (uint32_t)CAP) {
                            icut = (g0 * 32 + bb) * 32;
                            full = true;
                            break;
                        }
                        if (c) {
                            const uint32_t slot = cnt + __popc(cm & ((1u << lane) - 1u));
                            Sm.ci[slot] = i;
                            Sm.cd[slot] = d;
                            Sm.ck[slot] = ki;
                        }
                        cnt += __popc(cm);
                    }
                    if (!full && used == TIE_GROUPS) icut = min(n, (g0 + 1) * 1024u);
                }
                if (lane == 0) {
                    if (CL) Sm.cc2[attempt & 1] = cnt; else Sm.ccnt = cnt;
                    Sm.icut = icut;
                }
            }
        } else {
            for (uint32_t sg = sg0 + tid; sg < sg1; sg += TP)
                if (one_sg || (int64_t)(Sm.sgkey[sg] >> 15) - 1 >= tau) Sm.sglist[atomicAdd(&Sm.sgcnt, 1u)] = sg;
            part_sync(bar, TP);
            const uint32_t nsgl = Sm.sgcnt;
            for (uint32_t li = warp; li < nsgl; li += NW) {
                const uint32_t g = Sm.sglist[li] * 32 + lane;
                if (g < ng && (int64_t)(s_gkey[g] >> 10) - 1 >= tau) s_glist[atomicAdd(&Sm.gcnt, 1u)] = g;
            }
            part_sync(bar, TP);
            const uint32_t ngl = Sm.gcnt;
            // each warp takes the next listed group when it is done with one (the groups'
            // costs differ widely; a fixed stride leaves the slot waiting for the busiest warp)
            for (uint32_t li = take_next(&Sm.gnext, lane); li < ngl; li = take_next(&Sm.gnext, lane)) {
                const uint32_t g = s_glist[li];
                const uint32_t b = g * 32 + lane;
                const uint64_t bk = b < nb ? bkey[b] : 0ull;
                uint32_t mask = __ballot_sync(FULL, (int64_t)(bk >> 5) - 1 >= tau);
                while (mask) {
                    // up to LB buckets per pass so their loads overlap
                    uint32_t bbs[LB];
                    int nb8 = 0;
                    while (mask && nb8 < LB) {
                        bbs[nb8++] = (uint32_t)(__ffs(mask) - 1);
                        mask &= mask - 1;
                    }
                    int64_t d[LB];
                    uint64_t ki[LB];
#pragma unroll
                    for (int u = 0; u < LB; ++u) {
                        const uint32_t i = (g * 32 + (u < nb8 ? bbs[u] : 0)) * 32 + lane;
                        const bool ok = u < nb8 && i < n;
                        d[u] = ok ? (STREAM ? (int64_t)ld_hint_u64(&Dg[i], pol) : Dg[i]) : -1;
                        ki[u] = ok ? (STREAM ? ld_hint_u64(&key[i], pol) : key[i]) : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < LB; ++u) {
                        if (u < nb8 && d[u] >= tau && d[u] >= 0) {
                            // cluster mode: staged in this CTA's (otherwise unused) sample
                            // arrays, then moved to the leader in one block per CTA
                            const uint32_t slot = atomicAdd(&Sm.ccnt, 1u);
                            if (CL ? slot < (uint32_t)SMAX : slot < (uint32_t)CAP) {
                                if (CL) {
                                    Sm.sc[slot] = (g * 32 + bbs[u]) * 32 + lane;
                                    Sm.sd[slot] = d[u];
                                    Sm.sk[slot] = ki[u];
                                } else {
                                    Sm.ci[slot] = (g * 32 + bbs[u]) * 32 + lane;
                                    Sm.cd[slot] = d[u];
                                    Sm.ck[slot] = ki[u];
                                }
                            }
                        }
                    }
                }
            }
        }
        uint32_t ccnt;
        if constexpr (CL) {
            if (!tie) {
                // this CTA's candidates into the leader's arrays: one remote atomic for the
                // block's slots (the full count, so the leader's total is exact), then the
                // entries that fall below CAP
                part_sync(bar, TP);
                const uint32_t mine = Sm.ccnt;
                if (tid == 0) Sm.icut = mine ? atomicAdd(&Ld.cc2[attempt & 1], mine) : 0u;  // icut: base, for now
                part_sync(bar, TP);
                const uint32_t base = Sm.icut;
                for (uint32_t t = tid; t < min(mine, (uint32_t)SMAX) && base + t < (uint32_t)CAP; t += TP) {
                    Ld.ci[base + t] = Sm.sc[t];
                    Ld.cd[base + t] = Sm.sd[t];
                    Ld.ck[base + t] = Sm.sk[t];
                }
                part_sync(bar, TP);
                if (tid == 0) Sm.icut = 0xffffffffu;
            }
            // every CTA reads the leader's count of this attempt; the leader clears the
            // other parity's counter for the next attempt (its readers, the previous
            // attempt's, all passed the barrier before this one)
            cl.sync();
            ccnt = Ld.cc2[attempt & 1];
            if (leader && tid == 0) Sm.cc2[(attempt + 1) & 1] = 0;
            ++attempt;
        } else {
            part_sync(bar, TP);
            ccnt = Sm.ccnt;
        }
        const uint32_t icut = Sm.icut;
        if (ccnt > CAP) {
            // too many candidates: move tau toward D1 by about log2(ccnt / CAP) halvings;
            // at tau == D1 switch to the tie window until D1 drops
            if (tid == 0) {
                if (tau == D1) {
                    Sm.tieD = D1;
                } else {
                    int inc = 1;
                    for (uint32_t c = ccnt / CAP; c > 1; c >>= 1) ++inc;
                    Sm.shift = min(shift + inc, 62);
                }
            }
            part_sync(bar, TP);  // every thread has read the counters
            if (tid == 0) { Sm.ccnt = 0; Sm.gcnt = 0; Sm.sgcnt = 0; Sm.icut = 0xffffffffu; Sm.gnext = 0; }
            part_sync(bar, TP);
            continue;
        }
        // (4) candidates in index order: slot order is the lowest-index tie-break (the
        //     leader's candidates in cluster mode; the other CTAs wait at the next barrier).
        //     With the candidate matrix (a round of 32-bit keys whose candidates fit it) the
        //     sorted candidates go to the sample arrays, which the exact variant leaves
        //     unused, and every thread then fills rows of the matrix
        const bool usemat = MATRIX && !tie && ccnt <= (uint32_t)min(matrows, MS) && D1 - tau < (int64_t)(1u << OFF_BITS) - 1;
        if (leader && !tie) {
            uint32_t ci = 0, rank = 0;
            int64_t cd = 0;
            uint64_t ck = 0;
            if (tid < ccnt) {
                ci = Sm.ci[tid];
                cd = Sm.cd[tid];
                ck = Sm.ck[tid];
                for (uint32_t u = 0; u < ccnt; ++u) rank += Sm.ci[u] < ci ? 1u : 0u;
                if (usemat) {
                    Sm.sc[rank] = ci;
                    Sm.sd[rank] = cd;
                    Sm.sk[rank] = ck;
                }
            }
            part_sync(bar, TP);
            if constexpr (MATRIX) {
                if (usemat) {
                    for (uint32_t r = warp; r < ccnt; r += NW) {
                        const uint64_t pr = Sm.sk[r];
                        const int32_t rx = (int32_t)pos_x(pr), ry = (int32_t)pos_y(pr), rz = (int32_t)pos_z(pr);
                        for (uint32_t c = lane; c < ccnt; c += 32) {
                            const uint64_t qc = Sm.sk[c];
                            const int32_t dx = (int32_t)pos_x(qc) - rx, dy = (int32_t)pos_y(qc) - ry,
                                          dz = (int32_t)pos_z(qc) - rz;
                            const int64_t t = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz - tau;
                            mat[r * MS + c] = (c == r || t < 0) ? 0u
                                                                 : (t >= (int64_t)0xfffffffeu ? 0xffffffffu : (uint32_t)t + 1u);
                        }
                    }
                }
            }
            if (!usemat && tid < ccnt) {
                Sm.ci[rank] = ci;
                Sm.cd[rank] = cd;
                Sm.ck[rank] = ck;
            }
            part_sync(bar, TP);
        }
        // (5) the greedy restricted to C, one warp, while the best stays above (tau, icut);
        //     slot lane + 32u lives in lane's register u.  The updates are branch-free (a
        //     branch per register keeps the four updates from overlapping); pick t is
        //     recorded in lane t & 31 and written out after the loop.
        if (leader && warp == simw && usemat) {
            // the matrix greedy: a pick lowers every candidate's key to its row's entry
            // (an entry of 0 leaves the round, the picked candidate's own entry among
            // them); 0 << CAP_BITS | slot marks a candidate out of the round
            const uint32_t budget = min((uint32_t)MAXP, m - k);
            uint32_t np = 0;
            uint32_t rp[CPLM];
            uint32_t rec[2] = {0u, 0u};  // slot << OFF_BITS | (D - tau)
#pragma unroll
            for (int u = 0; u < CPLM; ++u) {
                const uint32_t sl = lane + 32 * u;
                rp[u] = sl < ccnt ? (uint32_t)(Sm.sd[sl] - tau) + 1u : 0u;
            }
            const uint32_t *mcol = mat + lane;
            while (np < budget) {
                uint32_t kmax = 0;
#pragma unroll
                for (int u = 0; u < CPLM; ++u) kmax = max(kmax, (rp[u] << CAP_BITS) | (uint32_t)(CAP - 1 - (lane + 32 * u)));
                const uint32_t best = __reduce_max_sync(FULL, kmax);
                if (best < (uint32_t)CAP) break;
                const uint32_t slot = (uint32_t)(CAP - 1) - (best & (uint32_t)(CAP - 1));
                const uint32_t r = (slot << OFF_BITS) | ((best >> CAP_BITS) - 1u);
                rec[0] = (lane == (int)(np & 31) && np < 32) ? r : rec[0];
                rec[1] = (lane == (int)(np & 31) && np >= 32) ? r : rec[1];
                ++np;
                const uint32_t *row = mcol + slot * MS;
#pragma unroll
                for (int u = 0; u < CPLM; ++u) rp[u] = min(rp[u], row[32 * u]);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t t = lane + 32 * h;
                if (t < np) {
                    const uint32_t slot = rec[h] >> OFF_BITS;
                    Sm.pi[t] = Sm.sc[slot];
                    Sm.pk[t] = Sm.sk[slot];
                    Sm.pd[t] = tau + (int64_t)(rec[h] & ((1u << OFF_BITS) - 1u));
                }
            }
            if (lane == 0) Sm.npick = np;
        } else if (leader && warp == simw) {
            const uint32_t budget = min((uint32_t)MAXP, m - k);
            const bool tiecut = icut != 0xffffffffu;
            uint32_t np = 0;
            int32_t cx[CPL], cy[CPL], cz[CPL];
#pragma unroll
            for (int u = 0; u < CPL; ++u) {
                const uint32_t sl = lane + 32 * u;
                const uint64_t q = sl < ccnt ? Sm.ck[sl] : 0ull;
                cx[u] = (int32_t)pos_x(q);
                cy[u] = (int32_t)pos_y(q);
                cz[u] = (int32_t)pos_z(q);
            }
            if (D1 - tau < (int64_t)(1u << OFF_BITS) - 1) {
                // every candidate's D lies in [tau, D1] and stays there while it can be
                // picked, so rp = D - tau + 1 < 2^OFF_BITS (0 = out of the round) and a
                // 32-bit key rp << CAP_BITS | (CAP - 1 - slot) orders (D, lowest slot) in one
                // reduction
                uint32_t rp[CPL];
                uint32_t rec[2] = {0u, 0u};  // slot << OFF_BITS | (D - tau)
#pragma unroll
                for (int u = 0; u < CPL; ++u) {
                    const uint32_t sl = lane + 32 * u;
                    rp[u] = sl < ccnt ? (uint32_t)(Sm.cd[sl] - tau) + 1u : 0u;
                }
                while (np < budget) {
                    uint32_t kmax = 0;
#pragma unroll
                    for (int u = 0; u < CPL; ++u)
                        kmax = max(kmax, rp[u] ? (rp[u] << CAP_BITS) | (uint32_t)(CAP - 1 - (lane + 32 * u)) : 0u);
                    const uint32_t best = __reduce_max_sync(FULL, kmax);
                    if (best == 0) break;
                    const uint32_t slot = (uint32_t)(CAP - 1) - (best & (uint32_t)(CAP - 1));
                    const uint32_t off = (best >> CAP_BITS) - 1u;
                    if (off == 0 && tiecut && Sm.ci[slot] >= icut) break;  // a tied point past the cut
                    const uint32_t r = (slot << OFF_BITS) | off;
                    rec[0] = (lane == (int)(np & 31) && np < 32) ? r : rec[0];
                    rec[1] = (lane == (int)(np & 31) && np >= 32) ? r : rec[1];
                    ++np;
                    const int su = (int)(slot >> 5), so = (int)(slot & 31);
                    int32_t sx = cx[0], sy = cy[0], sz = cz[0];
#pragma unroll
                    for (int u = 1; u < CPL; ++u) {
                        sx = su == u ? cx[u] : sx;
                        sy = su == u ? cy[u] : sy;
                        sz = su == u ? cz[u] : sz;
                    }
                    const int32_t bx = __shfl_sync(FULL, sx, so), by = __shfl_sync(FULL, sy, so),
                                  bz = __shfl_sync(FULL, sz, so);
                    int64_t t[CPL];
#pragma unroll
                    for (int u = 0; u < CPL; ++u) {
                        const int32_t dx = cx[u] - bx, dy = cy[u] - by, dz = cz[u] - bz;
                        t[u] = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz - tau;
                    }
#pragma unroll
                    for (int u = 0; u < CPL; ++u) {
                        // the new D = min(D, d); below tau it cannot be picked in this round
                        const bool lower = t[u] < (int64_t)rp[u] - 1;
                        const uint32_t nv = t[u] < 0 ? 0u : (uint32_t)t[u] + 1u;
                        rp[u] = (lane + 32 * u == (int)slot) ? 0u : ((rp[u] != 0u && lower) ? nv : rp[u]);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t t = lane + 32 * h;
                    if (t < np) {
                        const uint32_t slot = rec[h] >> OFF_BITS;
                        Sm.pi[t] = Sm.ci[slot];
                        Sm.pk[t] = Sm.ck[slot];
                        Sm.pd[t] = tau + (int64_t)(rec[h] & ((1u << OFF_BITS) - 1u));
                    }
                }
            } else {
                int64_t Dc[CPL];  // -1 = out of the round
                int64_t recD[2] = {0, 0};
                uint32_t recS[2] = {0u, 0u};
#pragma unroll
                for (int u = 0; u < CPL; ++u) {
                    const uint32_t sl = lane + 32 * u;
                    Dc[u] = sl < ccnt ? Sm.cd[sl] : -1;
                }
                while (np < budget) {
                    uint64_t kmax = 0;
#pragma unroll
                    for (int u = 0; u < CPL; ++u)
                        kmax = max(kmax, Dc[u] >= 0 ? ((uint64_t)(Dc[u] + 1) << 8) | (uint64_t)(255 - (lane + 32 * u))
                                                    : (uint64_t)0);
                    const uint64_t best = warp_max_u64(kmax);
                    if (best == 0) break;
                    const uint32_t slot = 255u - (uint32_t)(best & 255u);
                    const int64_t Dbest = (int64_t)(best >> 8) - 1;
                    if (Dbest == tau && tiecut && Sm.ci[slot] >= icut) break;  // a tied point past the cut
                    const bool mine = lane == (int)(np & 31);
                    recD[0] = (mine && np < 32) ? Dbest : recD[0];
                    recS[0] = (mine && np < 32) ? slot : recS[0];
                    recD[1] = (mine && np >= 32) ? Dbest : recD[1];
                    recS[1] = (mine && np >= 32) ? slot : recS[1];
                    ++np;
                    const int su = (int)(slot >> 5), so = (int)(slot & 31);
                    int32_t sx = cx[0], sy = cy[0], sz = cz[0];
#pragma unroll
                    for (int u = 1; u < CPL; ++u) {
                        sx = su == u ? cx[u] : sx;
                        sy = su == u ? cy[u] : sy;
                        sz = su == u ? cz[u] : sz;
                    }
                    const int32_t bx = __shfl_sync(FULL, sx, so), by = __shfl_sync(FULL, sy, so),
                                  bz = __shfl_sync(FULL, sz, so);
                    int64_t t[CPL];
#pragma unroll
                    for (int u = 0; u < CPL; ++u) {
                        const int32_t dx = cx[u] - bx, dy = cy[u] - by, dz = cz[u] - bz;
                        t[u] = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
                    }
#pragma unroll
                    for (int u = 0; u < CPL; ++u) {
                        const int64_t nd = min(Dc[u], t[u]);
                        Dc[u] = (lane + 32 * u == (int)slot || Dc[u] < 0 || nd < tau) ? -1 : nd;
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t t = lane + 32 * h;
                    if (t < np) {
                        Sm.pi[t] = Sm.ci[recS[h]];
                        Sm.pk[t] = Sm.ck[recS[h]];
                        Sm.pd[t] = recD[h];
                    }
                }
            }
            if (lane == 0) Sm.npick = np;
        }
        if (tid == 0 && !tie && ccnt < CAP / 4 && shift > 1) Sm.shift = shift - 1;
        if constexpr (CL) cl.sync(); else part_sync(bar, TP);
      }
        const uint32_t np = CL ? Ld.npick : Sm.npick;
        // (6) apply the round's picks to the whole part (cluster mode: to this CTA's
        //     points; each CTA copies the leader's picks, marks those it owns chosen, and
        //     the leader writes the outputs)
        const uint32_t own_lo = sg0 * 32768u, own_hi = sg1 * 32768u;
        for (uint32_t t = tid; t < np; t += TP) {
            const uint32_t pit = Ld.pi[t];
            const uint64_t q = Ld.pk[t];
            if (CL && !leader) Sm.pi[t] = pit;
            if (!CL || (pit >= own_lo && pit < own_hi)) Dg[pit] = -1;
            if (leader) {
                P.perm[k + t] = pit;
                P.rad2[k + t] = Sm.pd[t];
            }
            Sm.px[t] = (int32_t)pos_x(q);
            Sm.py[t] = (int32_t)pos_y(q);
            Sm.pz[t] = (int32_t)pos_z(q);
        }
        if (tid == 0) {
            // the next round's gather counters (this round read them before the last
            // barrier) and this round's apply counters
            Sm.ccnt = 0; Sm.gcnt = 0; Sm.sgcnt = 0; Sm.icut = 0xffffffffu; Sm.gnext = 0;
            Sm.asgcnt = 0; Sm.agcnt = 0; Sm.nheavy = 0; Sm.anext = 0;
        }
        part_sync(bar, TP);
        const uint64_t all = np >= 64 ? ~0ull : ((1ull << np) - 1ull);
        for (uint32_t sg = sg0 + warp; sg < sg1; sg += NW) {
            const uint64_t mk = pick_mask(np, Sm.pi, Sm.px, Sm.py, Sm.pz, all, 15, sg, Sm.sglo[sg], Sm.sghi[sg],
                                          one_sg ? INT64_MAX : (int64_t)(Sm.sgkey[sg] >> 15) - 1);
            if (mk && lane == 0) {
                Sm.sgmask[sg] = mk;
                Sm.sglist[atomicAdd(&Sm.asgcnt, 1u)] = sg;
            }
        }
        part_sync(bar, TP);
        const uint32_t nsgl = Sm.asgcnt;
        // A super-group's groups are tested against its picks by one warp walking the picks
        // (lanes = groups) or, with more picks, by a warp per group (lanes = picks): the
        // second takes more instructions but spreads a super-group over more warps.
        constexpr int LIGHT_MAX = TP > QT ? 16 : 4;
        for (uint32_t li = warp; li < nsgl; li += NW) {
            const uint32_t sg = Sm.sglist[li];
            const uint64_t sgm = Sm.sgmask[sg];
            if (__popcll((long long)sgm) <= LIGHT_MAX) {
                // few picks: one lane per group walks them
                const uint32_t g = sg * 32 + lane;
                if (g < ng) {
                    const int64_t gD = (int64_t)(s_gkey[g] >> 10) - 1;
                    const Box gb = unpack_box(s_glo[g], s_ghi[g]);
                    uint64_t mm = sgm;
                    bool rel = false;
                    while (mm) {  // the same (at most four) picks on every lane: no divergence
                        const int t = __ffsll((long long)mm) - 1;
                        mm &= mm - 1;
                        rel |= (Sm.pi[t] >> 10) == g || box_dist2_xyz(gb, Sm.px[t], Sm.py[t], Sm.pz[t]) < gD;
                    }
                    if (rel) s_glist[atomicAdd(&Sm.agcnt, 1u)] = g;
                }
            } else if (lane == 0) {
                Sm.heavy[atomicAdd(&Sm.nheavy, 1u)] = sg;
            }
        }
        part_sync(bar, TP);
        {
            // many picks: one warp per (super-group, group), the lanes test the picks
            const uint32_t nh = Sm.nheavy;
            for (uint32_t it = warp; it < nh * 32; it += NW) {
                const uint32_t sg = Sm.heavy[it >> 5];
                const uint32_t g = sg * 32 + (it & 31);
                if (g >= ng) continue;
                const uint64_t gm = pick_mask(np, Sm.pi, Sm.px, Sm.py, Sm.pz, Sm.sgmask[sg], 10, g, s_glo[g], s_ghi[g],
                                              (int64_t)(s_gkey[g] >> 10) - 1);
                if (gm && lane == 0) s_glist[atomicAdd(&Sm.agcnt, 1u)] = g;
            }
        }
        part_sync(bar, TP);
        const uint32_t ngl = Sm.agcnt;
        for (uint32_t li = take_next(&Sm.anext, lane); li < ngl; li = take_next(&Sm.anext, lane)) {
            const uint32_t g = s_glist[li];
            const uint64_t gm = pick_mask(np, Sm.pi, Sm.px, Sm.py, Sm.pz, Sm.sgmask[g >> 5], 10, g, s_glo[g], s_ghi[g],
                                          (int64_t)(s_gkey[g] >> 10) - 1);
            const uint32_t b = g * 32 + lane;
            const bool vb = b < nb;
            uint64_t bk = vb ? bkey[b] : 0ull;
            const Box bb = unpack_box(vb ? blo_p[b] : 0ull, vb ? bhi_p[b] : 0ull);
            const int64_t bD = (int64_t)(bk >> 5) - 1;  // -1 past the end: no pick qualifies
            // picks that may lower a D in this lane's bucket (gm is the same on every lane)
            uint64_t bm = 0;
            {
                uint64_t mm = gm;
                while (mm) {
                    const int t = __ffsll((long long)mm) - 1;
                    mm &= mm - 1;
                    const bool r = (Sm.pi[t] >> 5) == b || box_dist2_xyz(bb, Sm.px[t], Sm.py[t], Sm.pz[t]) < bD;
                    bm |= r ? 1ull << t : 0ull;
                }
            }
            uint32_t amask = __ballot_sync(FULL, bm != 0);
            const bool aff = bm != 0;
            while (amask) {
                // up to LB affected buckets per pass so their loads overlap
                uint32_t bbs[LB];
                int nb8 = 0;
                while (amask && nb8 < LB) {
                    bbs[nb8++] = (uint32_t)(__ffs(amask) - 1);
                    amask &= amask - 1;
                }
                int64_t d[LB];
                uint64_t ki[LB];
#pragma unroll
                for (int u = 0; u < LB; ++u) {
                    const uint32_t i = (g * 32 + (u < nb8 ? bbs[u] : 0)) * 32 + lane;
                    const bool ok = u < nb8 && i < n;
                    d[u] = ok ? (STREAM ? (int64_t)ld_hint_u64(&Dg[i], pol) : Dg[i]) : -1;
                    ki[u] = ok ? (STREAM ? ld_hint_u64(&key[i], pol) : key[i]) : 0ull;
                }
#pragma unroll
                for (int u = 0; u < LB; ++u) {
                    if (u >= nb8) break;
                    const uint32_t i = (g * 32 + bbs[u]) * 32 + lane;
                    const uint64_t mu = __shfl_sync(FULL, bm, (int)bbs[u]);
                    int64_t dd = d[u];
                    {
                        // every lane walks the bucket's picks (mu is the same on every lane)
                        const int32_t x = (int32_t)pos_x(ki[u]), y = (int32_t)pos_y(ki[u]), z = (int32_t)pos_z(ki[u]);
                        int64_t nd = dd;
                        uint64_t mm = mu;
                        while (mm) {
                            const int t = __ffsll((long long)mm) - 1;
                            mm &= mm - 1;
                            const int32_t dx = x - Sm.px[t], dy = y - Sm.py[t], dz = z - Sm.pz[t];
                            nd = min(nd, (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz);
                        }
                        if (dd > 0 && nd < dd) {  // chosen points (-1) and duplicates (0) stay
                            dd = nd;
                            if (STREAM) st_hint_u64(&Dg[i], (uint64_t)nd, pol);
                            else Dg[i] = nd;
                        }
                    }
                    const uint64_t nk = i < n ? (((uint64_t)(dd + 1) << 5) | (uint64_t)(31 - lane)) : 0ull;
                    const uint64_t nbk = warp_max_u64(nk);
                    if (lane == (int)bbs[u]) bk = nbk;
                }
            }
            if (aff) bkey[b] = bk;
            const uint64_t cand = vb ? (((bk >> 5) << 10) | (uint64_t)(1023 - (lane * 32 + (31 - (int)(bk & 31))))) : 0ull;
            const uint64_t ngk = warp_max_u64(cand);
            if (lane == 0) s_gkey[g] = ngk;
        }
        part_sync(bar, TP);
        if (!one_sg) {
            for (uint32_t li = warp; li < nsgl; li += NW) {
                const uint32_t sg = Sm.sglist[li];
                const uint32_t g = sg * 32 + lane;
                const uint64_t gk = g < ng ? s_gkey[g] : 0ull;
                const uint64_t cand = g < ng ? (((gk >> 10) << 15) | (uint64_t)(32767 - (lane * 1024 + (1023 - (int)(gk & 1023))))) : 0ull;
                const uint64_t sk = warp_max_u64(cand);
                if (lane == 0) Sm.sgkey[sg] = sk;
            }
        }
        k += np;
        // the next round reads the super-group keys; one_sg parts read only group keys,
        // which the bucket updates wrote before the last barrier
        if (!one_sg) part_sync(bar, TP);
    }
    // the part's radii, then its completion flag (host-mapped memory, after a
    // system-scope fence so the host sees every output of the part first).  Cluster
    // mode: the CTAs share the radii, reading the leader's rad2 from L2 after a barrier
    if constexpr (CL) cl.sync();
    if (P.radius)
        for (uint32_t q = (uint32_t)crank * TP + tid; q < m; q += (uint32_t)csize * TP) {
            const int64_t r2 = CL ? __ldcg(&P.rad2[q]) : P.rad2[q];
            P.radius[q] = r2 == INT64_MAX ? __int_as_float(0x7f800000)
                                          : (float)__ddiv_rn(__dsqrt_rn((double)r2), P.scale);
        }
    if constexpr (CL) cl.sync(); else part_sync(bar, TP);
    if (tid == 0 && leader && P.done) {
        __threadfence_system();
        *(volatile uint32_t *)P.done = 1u;
    }
    part_sync(bar, TP);
}

// Persistent rounds kernel.  Parts [0, nfull) run one at a time on the whole CTA; with
// QUARTERS (CT = 1024) the CTA then splits into four 256-thread quarters that take the
// remaining parts [nfull, nparts) one each, on named barriers 1-4.  next[0] and next[1]
// are the two phases' work counters.
template <int CT, int SLOTS>
__global__ void __launch_bounds__(CT) k_order_rounds(const PartDesc *__restrict__ parts, int nparts, int nfull,
                                                     uint32_t *__restrict__ next, int ngmax, int nbsm, int ngq, int nbq,
                                                     int qmat) {
    extern __shared__ __align__(16) unsigned char smraw[];
    static_assert(SLOTS == 1 || SLOTS == 2 || SLOTS == 4 || SLOTS == 8, "1, 2, 4 or 8 part slots per CTA");
    __shared__ uint32_t s_part[8];  // one entry per slot
    for (;;) {
        if (threadIdx.x == 0) s_part[0] = atomicAdd(&next[0], 1u);
        __syncthreads();
        const uint32_t p = s_part[0];
        __syncthreads();
        if (p >= (uint32_t)nfull) break;
        const int mrows = CT == 1024 ? mat_rows(nbsm, ngmax) : 0;
        rounds_part<CT, MAX_SG>(parts[p], *(RoundsSm<MAX_SG> *)smraw, smraw, nbsm, ngmax, threadIdx.x, 0, 0, 0, 1,
                                (uint32_t *)(smraw + slot_bytes<MAX_SG>(nbsm, ngmax)), mrows);
    }
    if constexpr (SLOTS > 1) {
        constexpr int ST = CT / SLOTS, S_SG = slot_sg(SLOTS), SW = ST / 32;
        const int q = threadIdx.x / ST, tid = threadIdx.x % ST;
        // a slot: its records, then (qmat = 64) a 64 x 64 candidate matrix
        const size_t sb = slot_bytes<S_SG>(nbq, ngq);
        unsigned char *slot = smraw + (size_t)q * (sb + (size_t)qmat * 64 * 4);
        for (;;) {
            if (tid == 0) s_part[q] = (uint32_t)nfull + atomicAdd(&next[1], 1u);
            part_sync(1 + q, ST);
            const uint32_t p = s_part[q];
            part_sync(1 + q, ST);
            if (p >= (uint32_t)nparts) break;
            // the slots' serial warps sit on different schedulers (warp index modulo 4)
            rounds_part<ST, S_SG>(parts[p], *(RoundsSm<S_SG> *)slot, slot, nbq, ngq, tid, 1 + q, q % SW, 0, 1,
                                  (uint32_t *)(slot + sb), qmat);
        }
    }
}

// Persistent cluster kernel: each thread-block cluster orders one part at a time on all
// of its CTAs (the largest parts of a launch; next[0] is the work counter).
template <int CT>
__global__ void __launch_bounds__(CT) k_order_cluster(const PartDesc *__restrict__ parts, int nparts,
                                                      uint32_t *__restrict__ next, int ngmax) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint32_t s_part;
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) s_part = atomicAdd(&next[0], 1u);
        cl.sync();
        const uint32_t p = *cl.map_shared_rank(&s_part, 0);
        cl.sync();  // every CTA has its part index before the leader takes the next one
        if (p >= (uint32_t)nparts) break;
        rounds_part<CT, MAX_SG, true>(parts[p], *(RoundsSm<MAX_SG> *)smraw, smraw, 0, ngmax, threadIdx.x, 0, 0, crank,
                                      csize);
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
static int g_order_algo = 2;              // 1 = one pick per step, 2 = exact multi-pick rounds
static int g_ctas_per_sm_override = 0;    // set by bs_set_tuning("order_ctas_per_sm", v)
static int g_quarters = 0;                // set by bs_set_tuning("order_quarters", v): 0 auto, 1 off, 2 on
static int g_full_parts = 0;              // set by bs_set_tuning("order_full_parts", k); 0 = cost model
static int g_slots = 4;                   // set by bs_set_tuning("order_slots", v): parts per 1024-thread CTA
static int g_cluster = 1;                 // bs_set_tuning("order_cluster", c): 0 auto, 1 off, 2..16 CTAs
static uint32_t g_cluster_min = 262144;   // bs_set_tuning("order_cluster_min", n): smallest cluster part

void order_set_tuning(int threads, int ctas_per_sm) {
    g_loop_threads_override = threads;
    g_ctas_per_sm_override = ctas_per_sm;
}

void order_set_algo(int algo) { g_order_algo = algo; }

void order_set_quarters(int v) { g_quarters = v; }

void order_set_full_parts(int k) { g_full_parts = k; }

void order_set_slots(int v) { g_slots = v; }

void order_set_cluster(int c, int min_points) {
    if (c >= 0) g_cluster = c;
    if (min_points > 0) g_cluster_min = (uint32_t)min_points;
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

// Lets a kernel launch with up to the device's opt-in shared memory per block.  Every
// call sets the same value, so calls from several host threads (each launching with its
// own dynamic size) cannot lower the limit under another thread's launch.
template <typename K>
static cudaError_t allow_smem(K kern) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// whole-CTA shared memory: the part's records, then (1024-thread CTAs) the candidate matrix
static size_t rounds_smem_full(int ngmax, int ct, int nbmin = 0) {
    const int nbsm = rounds_nbsm(ngmax, nbmin);
    return slot_bytes<MAX_SG>(nbsm, ngmax) + (ct == 1024 ? (size_t)mat_rows(nbsm, ngmax) * MAT_ROW : 0);
}

// slot-mode bucket capacity: what is left of a slot's share of the shared memory
template <int SLOTS>
static int slot_nb(int ngq) {
    constexpr int S_SG = slot_sg(SLOTS);
    const long left = (long)(SMEM_LIMIT / SLOTS) - (long)align16(sizeof(RoundsSm<S_SG>)) - (long)align16((size_t)ngq * 28);
    return (int)std::max(0L, std::min((long)Q_NB, left / 24));
}

template <int CT, int SLOTS>
static cudaError_t launch_rounds(const PartDesc *d_parts, int nparts, int nfull, uint32_t *d_next, int ngmax, int ngq,
                                 int grid, cudaStream_t stream, int nbmin = 0) {
    int nbq = 0;
    int qmat = 0;
    size_t smem = rounds_smem_full(ngmax, CT, nbmin);
    if constexpr (SLOTS > 1) {
        nbq = slot_nb<SLOTS>(ngq);
        // a 64 x 64 candidate matrix per slot where the slots' records leave room for it
        const size_t sb = slot_bytes<slot_sg(SLOTS)>(nbq, ngq);
        qmat = SLOTS * (sb + 64 * 64 * 4) <= SMEM_LIMIT ? 64 : 0;
        smem = std::max(smem, SLOTS * (sb + (size_t)qmat * 64 * 4));
    }
    if (smem > SMEM_LIMIT) return cudaErrorInvalidConfiguration;
    cudaError_t e = allow_smem(k_order_rounds<CT, SLOTS>);
    if (e != cudaSuccess) return e;
    k_order_rounds<CT, SLOTS><<<grid, CT, smem, stream>>>(d_parts, nparts, nfull, d_next, ngmax,
                                                           rounds_nbsm(ngmax, nbmin), ngq, nbq, qmat);
    return cudaGetLastError();
}

template <int T>
static cudaError_t launch_loop(const PartDesc *d_parts, int nparts, uint32_t *d_next, int ngmax, int grid,
                               cudaStream_t stream, int algo, int nbmin = 0) {
    if (algo == 1) {
        const size_t smem = (size_t)ngmax * 36;
        cudaError_t e = allow_smem(k_order_loop<T>);
        if (e != cudaSuccess) return e;
        k_order_loop<T><<<grid, T, smem, stream>>>(d_parts, nparts, d_next, ngmax);
        return cudaGetLastError();
    } else if constexpr (T >= CAP && T >= SMAX) {
        return launch_rounds<T, 1>(d_parts, nparts, nparts, d_next, ngmax, 0, grid, stream, nbmin);
    } else {
        return cudaErrorInvalidConfiguration;  // the rounds kernel needs at least CAP threads
    }
}

template <int T>
static int occupancy(int ngmax, int algo, int nbmin = 0) {
    int blocks = 0;
    cudaError_t e = cudaSuccess;
    if (algo == 1) {
        const size_t smem = (size_t)ngmax * 36;
        allow_smem(k_order_loop<T>);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_order_loop<T>, T, smem);
    } else if constexpr (T >= CAP && T >= SMAX) {
        const size_t smem = rounds_smem_full(ngmax, T, nbmin);
        allow_smem(k_order_rounds<T, 1>);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_order_rounds<T, 1>, T, smem);
    } else {
        blocks = 1;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(blocks, 1);
}

static int pick_threads(int ngmax, bool batched, int algo) {
    if (g_loop_threads_override) return algo == 2 ? std::max(g_loop_threads_override, 256) : g_loop_threads_override;
    // measured: 16 warps per part beat more resident parts; parts of 64k points and more
    // order faster on 32 warps (a 442k-surfel part: 281 ms against 316 ms)
    if (algo == 2) return ngmax <= 8 ? 256 : (ngmax >= 64 ? 1024 : 512);
    if (batched) return ngmax > 256 ? 256 : 128;
    if (ngmax <= 32) return 128;
    if (ngmax <= 512) return 256;
    return 512;
}

// How many of the largest parts (sizes sorted descending) to run on whole 1024-thread
// CTAs before the CTAs split into quarters for the rest; -1 when plain whole-CTA launches
// are predicted faster.  Cost model (measured on GB300): a part costs n ln n; a whole CTA
// orders at speed 1, a quarter at 0.41 with four per SM.  kmin parts are too large for a
// quarter.
static int quarter_split(const std::vector<uint32_t> &ns, int sms, int kmin, int slots = 4) {
    const int P = (int)ns.size();
    if (kmin >= P) return -1;
    std::vector<double> w(P), tail(P + 1, 0.0);
    for (int i = 0; i < P; ++i) w[i] = (double)ns[i] * std::log((double)ns[i] + 2.0);
    for (int i = P - 1; i >= 0; --i) tail[i] = tail[i + 1] + w[i];
    // speed of one part slot relative to a whole CTA (measured for quarters; assumed for 2 and 8)
    const double RQ = slots == 2 ? 0.7 : slots == 8 ? 0.22 : 0.41;
    double best = std::max(tail[0] / sms, w[0]);  // whole CTAs only
    int pick = -1;
    for (int k = kmin; k <= std::min(P - 1, std::max(kmin, sms)); ++k) {
        const double tfull = k > 0 ? std::max(w[0], tail[0] - tail[k] > 0 ? (tail[0] - tail[k]) / sms : 0.0) : 0.0;
        const int free_sms = std::max(1, sms - std::min(k, sms / 2));
        const double tq = std::max(tail[k] / (slots * RQ * free_sms), w[k] / RQ);
        const double t = std::max(tfull, tq);
        if (t < best * 0.97) {  // a clear predicted gain only
            best = t;
            pick = k;
        }
    }
    return pick;
}

// one persistent rounds launch over parts[0..nparts) (sorted by size, largest first; ns
// their sizes, ngs their group counts); d_next holds two zeroed work counters
static cudaError_t launch_set(const PartDesc *d_parts, int nparts, uint32_t *d_next, int ngmax, int T, int sms,
                              cudaStream_t stream, int algo, const std::vector<uint32_t> &ns,
                              const std::vector<uint32_t> &ngs, bool throughput = false, bool any_sampler = false) {
    if (algo == 2 && g_quarters != 1 && !(g_loop_threads_override && g_loop_threads_override != 1024)) {
        // parts per CTA after the whole-CTA parts: order_slots (4 by default); eight 128-thread
        // slots cannot run the sampler variant
        const int slots = (g_slots == 8 && any_sampler) ? 4 : g_slots;
        int kmin = 0;
        while (kmin < nparts && ngs[kmin] > (uint32_t)(slot_sg(slots) * 32)) ++kmin;
        int nfull = -1;
        if (g_full_parts > 0) nfull = std::max(kmin, std::min(g_full_parts, nparts));
        else if (g_quarters == 2) nfull = kmin;
        else if (nparts >= 2 * sms) nfull = quarter_split(ns, sms, kmin, slots);
        else if (throughput && nparts - kmin >= 8) {
            // a server launch: parts of 64k points and more keep whole CTAs (a quarter
            // orders one at about 0.41 of a whole CTA's speed), the rest share SMs
            nfull = kmin;
            while (nfull < nparts && ns[nfull] >= 65536u) ++nfull;
        }
        if (nfull >= 0 && nfull < nparts) {
            const int ngq = (int)ngs[nfull];
            // a small launch takes only the CTAs its parts fill (other launches share the GPU)
            const int grid = throughput ? std::min(sms, nfull + (nparts - nfull + slots - 1) / slots) : sms;
            // buckets of the smallest whole-CTA part (none: no whole-CTA bucket records)
            const int nbmin = nfull > 0 ? (int)((ns[nfull - 1] + 31u) / 32u) : NB_SMEM + 1;
            switch (slots) {
                case 2: return launch_rounds<1024, 2>(d_parts, nparts, nfull, d_next, ngmax, ngq, grid, stream, nbmin);
                case 8: return launch_rounds<1024, 8>(d_parts, nparts, nfull, d_next, ngmax, ngq, grid, stream, nbmin);
                default: return launch_rounds<1024, 4>(d_parts, nparts, nfull, d_next, ngmax, ngq, grid, stream, nbmin);
            }
        }
    }
    // every part of this launch runs on a whole CTA: the smallest one's buckets
    const int nbmin = nparts > 0 ? (int)((ns[nparts - 1] + 31u) / 32u) : 0;
    int per_sm = 1;
    switch (T) {
        case 64: per_sm = occupancy<64>(ngmax, algo, nbmin); break;
        case 128: per_sm = occupancy<128>(ngmax, algo, nbmin); break;
        case 256: per_sm = occupancy<256>(ngmax, algo, nbmin); break;
        case 512: per_sm = occupancy<512>(ngmax, algo, nbmin); break;
        default: per_sm = occupancy<1024>(ngmax, algo, nbmin); break;
    }
    if (g_ctas_per_sm_override) per_sm = std::min(per_sm, g_ctas_per_sm_override);
    const int grid = std::max(1, std::min(nparts, sms * per_sm));
    switch (T) {
        case 64: return launch_loop<64>(d_parts, nparts, d_next, ngmax, grid, stream, algo, nbmin);
        case 128: return launch_loop<128>(d_parts, nparts, d_next, ngmax, grid, stream, algo, nbmin);
        case 256: return launch_loop<256>(d_parts, nparts, d_next, ngmax, grid, stream, algo, nbmin);
        case 512: return launch_loop<512>(d_parts, nparts, d_next, ngmax, grid, stream, algo, nbmin);
        default: return launch_loop<1024>(d_parts, nparts, d_next, ngmax, grid, stream, algo, nbmin);
    }
}

// Cluster launch over parts[0..nparts) (all of at least csize super-groups, exact
// ordering): csize CTAs of 1024 threads per part, at most nclusters clusters resident
// (persistent over the parts).  The cluster size shrinks until the device can hold one.
static cudaError_t launch_cluster(const PartDesc *d_parts, int nparts, uint32_t *d_next, int ngmax, int csize,
                                  int nclusters, cudaStream_t stream) {
    const size_t smem = slot_bytes<MAX_SG>(0, ngmax);
    auto kern = k_order_cluster<1024>;
    cudaError_t e = allow_smem(kern);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (; csize >= 2; --csize) {
        attr[0].val.clusterDim.x = (unsigned)csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)csize, 1, 1);
        int maxc = 0;
        if (cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            maxc = 0;
        }
        if (maxc >= 1) {
            const int nc = std::max(1, std::min(std::min(nclusters, maxc), nparts));
            cfg.gridDim = dim3((unsigned)(csize * nc), 1, 1);
            return cudaLaunchKernelEx(&cfg, kern, d_parts, nparts, d_next, ngmax);
        }
    }
    return cudaErrorInvalidConfiguration;
}

// The library's side stream of the current device (cluster launches beside the rest).
static cudaStream_t side_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

// Orders nparts parts.  host descriptors: keys, outputs, n, m, start, scale filled in.
bs_status order_parts(std::vector<PartDesc> &hp, cudaStream_t stream, bool batched, bool throughput) {
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
        if (p.variant == 1) total += 2 * align_up((size_t)p.n * 4);
        if (!p.rad2) total += align_up((size_t)p.m * 8);
    }
    const size_t desc_bytes = align_up((size_t)nparts * sizeof(PartDesc));
    const size_t gofs_bytes = align_up((size_t)nparts * 4);
    total += desc_bytes + gofs_bytes + 256;
    char *ws = nullptr;
    cudaError_t e = pool_malloc_async((void **)&ws, total, stream);
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
        if (p.variant == 1) {
            p.R = (uint32_t *)take((size_t)p.n * 4);
            p.pos = (uint32_t *)take((size_t)p.n * 4);
        }
        gofs[r] = total_groups;
        total_groups += p.ng;
        sorted[r] = p;
    }
    bs_status rc = BS_OK;
    do {
        if (cudaMemcpyAsync(d_parts, sorted.data(), (size_t)nparts * sizeof(PartDesc), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemcpyAsync(d_gofs, gofs.data(), (size_t)nparts * 4, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaMemsetAsync(d_next, 0, 32, stream) != cudaSuccess) {
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
        // the one-pick-per-step kernel only knows the exact greedy permutation
        // (and only the rounds kernel publishes per-part completion flags)
        bool sampled = false, any_variant1 = false;
        for (const auto &q : sorted) {
            sampled |= q.variant == 1 || q.done != nullptr;
            any_variant1 |= q.variant == 1;
        }
        const int algo = sampled ? 2 : g_order_algo;
        timing_mark(1, 0, stream);
        std::vector<uint32_t> ns(nparts), ngs(nparts);
        for (int r = 0; r < nparts; ++r) { ns[r] = sorted[r].n; ngs[r] = sorted[r].ng; }
        // the largest parts (exact ordering, at least order_cluster_min points) on thread-block
        // clusters, the rest as before; with both, the clusters run on the side stream
        int kc = 0, csize = 0;
        if (algo == 2 && g_cluster != 1) {
            while (kc < nparts && sorted[kc].variant == 0 && sorted[kc].n >= g_cluster_min) ++kc;
            if (kc > 0) {
                const int ns_min = (int)((sorted[kc - 1].ng + 31) / 32);
                if (g_cluster >= 2) {
                    csize = g_cluster;
                } else {
                    const int budget = kc == nparts ? sms : sms / 2;
                    csize = std::min(16, ns_min);
                    while (csize > 2 && kc * csize > budget) --csize;
                }
                csize = std::min(csize, ns_min);
                if (csize < 2) kc = 0;
            }
        }
        if (kc > 0) {
            const int nclusters = std::max(1, std::min(kc, sms / csize));
            uint32_t ngc = 1;
            for (int r = 0; r < kc; ++r) ngc = std::max(ngc, sorted[r].ng);
            if (kc == nparts) {
                e = launch_cluster(d_parts, kc, d_next + 4, (int)ngc, csize, nclusters, stream);
            } else {
                cudaStream_t side = side_stream();
                cudaEvent_t ev[2] = {nullptr, nullptr};
                e = side ? cudaSuccess : cudaErrorNotReady;
                for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(ev[0], stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev[0], 0);
                if (e == cudaSuccess) e = launch_cluster(d_parts, kc, d_next + 4, (int)ngc, csize, nclusters, side);
                if (e == cudaSuccess) {
                    std::vector<uint32_t> ns2(ns.begin() + kc, ns.end()), ngs2(ngs.begin() + kc, ngs.end());
                    uint32_t ngr = 1;
                    for (int r = kc; r < nparts; ++r) ngr = std::max(ngr, sorted[r].ng);
                    e = launch_set(d_parts + kc, nparts - kc, d_next, (int)ngr,
                                   pick_threads((int)ngr, batched, algo), sms, stream, algo, ns2, ngs2, throughput,
                                   any_variant1);
                }
                if (e == cudaSuccess) e = cudaEventRecord(ev[1], side);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev[1], 0);
                for (int i = 0; i < 2; ++i)
                    if (ev[i]) cudaEventDestroy(ev[i]);
            }
        } else {
            e = launch_set(d_parts, nparts, d_next, (int)ngmax, pick_threads((int)ngmax, batched, algo), sms, stream,
                           algo, ns, ngs, throughput, any_variant1);
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
        if (any_radius && algo == 1) {  // the rounds kernel writes radii at the end of each part
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

static_assert(sizeof(PartDesc) <= NA_NEXT - NA_DESC, "the descriptor must fit before the part counter");
static_assert(NA_D % 8 == 0 && NA_RAD2 % 8 == 0 && NA_BUCKETS % 8 == 0 && NA_GROUPS % 8 == 0,
              "scratch regions hold 8-byte words");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Writes the part descriptor (passed by value, so nothing is read from host memory
// once the launch is queued) into the scratch array and zeroes the part counter and
// the group offset that follow it.
__global__ void k_noalloc_setup(PartDesc p, PartDesc *d_desc, uint32_t *d_next) {
    if (threadIdx.x == 0) {
        *d_desc = p;
        d_next[0] = 0u;
        d_next[1] = 0u;
    }
}

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
    if (p.variant != 0) {
        set_error("bs_order_noalloc: only the exact ordering (variant 0) runs without allocation");
        return BS_EINVAL;
    }
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
    k_noalloc_setup<<<1, 32, 0, stream>>>(p, d_desc, d_next);  // d_next[0] counter, d_next[1] = gofs[0] = 0
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("bs_order_noalloc: descriptor setup failed: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    k_order_init<<<(p.ng + 7) / 8, 256, 0, stream>>>(d_desc, d_next + 1, 1, p.ng);
    const int T = pick_threads((int)p.ng, false, g_order_algo);
    switch (T) {
        case 64: e = launch_loop<64>(d_desc, 1, d_next, (int)p.ng, 1, stream, g_order_algo); break;
        case 128: e = launch_loop<128>(d_desc, 1, d_next, (int)p.ng, 1, stream, g_order_algo); break;
        case 256: e = launch_loop<256>(d_desc, 1, d_next, (int)p.ng, 1, stream, g_order_algo); break;
        case 512: e = launch_loop<512>(d_desc, 1, d_next, (int)p.ng, 1, stream, g_order_algo); break;
        default: e = launch_loop<1024>(d_desc, 1, d_next, (int)p.ng, 1, stream, g_order_algo); break;
    }
    if (e == cudaSuccess && p.radius && g_order_algo == 1) {  // the rounds kernel writes radii itself
        k_radius<<<dim3(std::min<uint32_t>((p.m + 255) / 256, 64), 1), 256, 0, stream>>>(d_desc, 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { set_error("bs_order_noalloc: launch failed: %s", cudaGetErrorString(e)); return BS_ECUDA; }
    return BS_OK;
}

}  // namespace bs
