// imin_dev.cuh -- device-side pieces of the sampled-dominator-tree estimator (Alg. 2 of
// arXiv 2302.13529) for sm_103a.
//
// One warp owns one sampled graph (Def. 4) at a time and runs, without ever materialising
// the sampled graph:
//   1. a level-synchronous BFS from the seeds (all at depth 0 under a virtual super-seed,
//      Sec. 4 "From Multiple Seeds to One Seed"). The out-edges of a frontier are flattened
//      into groups of 4 consecutive edge ids; each lane takes one group, loads its 4
//      thresholds with one 16-byte load, evaluates one Philox4x32-10 call whose 4 output words
//      decide the 4 edges, and loads the target id only for live edges. Live targets that are
//      neither seeds nor blocked go through a warp-shared open-addressing hash (global id ->
//      local id). A newly inserted vertex gets the next local id, so local ids follow BFS
//      discovery order and every level occupies a contiguous id range; the discovering vertex
//      becomes its initial dominator candidate. Live edges to already-known vertices are kept
//      as "non-tree" edges.
//   2. immediate dominators (Defs. 5-6) by the iterative intersection scheme of Cooper,
//      Harvey and Kennedy on BFS numbering: start from the BFS tree and, for every non-tree
//      edge (p, v), lower idom(v) to the nearest common ancestor of idom(v), p and v's BFS
//      parent in the current tree, until a pass changes nothing. A dominator of v lies on
//      every path to v, in particular on a shortest one, so it has a smaller BFS number and
//      the tree always satisfies idom(v) < v. Why the result is the dominator tree: the
//      ancestor sets X(v) start as BFS-tree paths, which contain every dominator, and each
//      update keeps them supersets of the dominator sets; at the end every in-edge (p, v)
//      -- the parent edge included, which is why it is folded in every pass -- has idom(v)
//      above p, so X is a post-fixed point of the dominance equations, hence contained in
//      their greatest fixed point, the dominator sets. Both inclusions give equality.
//   3. subtree sizes (Thm. 6) by one sweep over BFS levels from the deepest up (a dominator
//      is strictly shallower than what it dominates), adding each size into its idom.
//   4. Delta[u] += c[u] for every reached non-seed u (64-bit atomics into global memory).
//
// The warp's working set lives either in shared memory (tier 0) or in a per-warp global
// scratch slot (tiers 1 and 2, bigger capacities). A sample that exceeds its tier's capacity
// is abandoned (its hash entries are cleared) and handed to the next tier; nothing it
// computed has been published, so the retry is exact.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace imin {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kEmpty = 0xFFFFFFFFu;
// Tiers: 0-2 are warp-per-sample (0: shared-memory hash, 1: per-warp global hash for up to
// 16K vertices, 2: per-warp whole-graph scratch, the final fallback); 3 is block-per-sample with
// a shared-memory visited bitmap (graphs with n <= kCtaMaxVertices).
constexpr int kTiers = 4;
constexpr int kTierWhole = 2;
constexpr int kTierCta = 3;
constexpr int32_t kCtaMaxVertices = 1 << 18;
constexpr int kStageCap = 128;  // 32 lanes x 4 edges per group

enum : uint32_t { kErrCapacity = 1u, kErrInternal = 2u };

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3). Counter c, key (k0, k1).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

struct DevGraph {
    int32_t n;
    int32_t m;
    const int32_t* __restrict__ row_ptr;  // [n+1]
    const int32_t* __restrict__ col;      // [m], padded to a multiple of 4
    const uint4* __restrict__ thr4;       // [ceil(m/4)] IC: thresholds; LT: interval widths - 1
    const uint4* __restrict__ lo4;        // LT: start of each in-edge's interval; nullptr for IC
};

// The 32-bit word of vertex v's triggering draw in sample j of call `round` (linear-threshold
// model): word v & 3 of Philox4x32-10 at counter (v >> 2, j, round, 0x80000000). Edge words use
// the last counter word e >> 34 = 0, so the two never share a counter.
__device__ __forceinline__ uint32_t vertex_word(uint32_t v, uint32_t j, uint32_t round, uint32_t k0,
                                                uint32_t k1)
{
    const uint4 r = philox4x32_10(make_uint4(v >> 2, j, round, 0x80000000u), k0, k1);
    const uint32_t k = v & 3u;
    return k == 0 ? r.x : (k == 1 ? r.y : (k == 2 ? r.z : r.w));
}

// Propagation model of a kernel instantiation: IC or LT fixed at compile time, or taken from the
// graph at run time (batched kernels, whose queries may mix models).
enum : int { kModelIC = 0, kModelLT = 1, kModelAny = 2 };

// Live mask (bit k: edge 4q + k) of the edges 4q .. 4q+3 that lie in [beg, end), in sample j of
// call `round`; th = thr4[q].
//   IC (Def. 4): edge e is live iff its Philox word (counter (q, j, round, 0), word e & 3) <= thr.
//   LT (Sec. 4.5, linear-threshold triggering sets): edge e = (u, v) is live iff v's word lies in
//   e's interval [lo, lo + thr], i.e. (word - lo) mod 2^32 <= thr; the in-edges of v hold disjoint
//   intervals, so at most one of them is live.
template <int M = kModelAny>
__device__ __forceinline__ uint32_t group_live(const DevGraph& g, uint32_t q, const uint4& th, int32_t beg,
                                               int32_t end, uint32_t j, uint32_t round, uint32_t k0,
                                               uint32_t k1)
{
    const int32_t e0 = static_cast<int32_t>(q << 2);
    if (M == kModelIC || (M == kModelAny && g.lo4 == nullptr)) {
        const uint4 r = philox4x32_10(make_uint4(q, j, round, 0u), k0, k1);
        uint32_t m = 0;
        m |= (e0 + 0 >= beg && e0 + 0 < end && r.x <= th.x) ? 1u : 0u;
        m |= (e0 + 1 >= beg && e0 + 1 < end && r.y <= th.y) ? 2u : 0u;
        m |= (e0 + 2 >= beg && e0 + 2 < end && r.z <= th.z) ? 4u : 0u;
        m |= (e0 + 3 >= beg && e0 + 3 < end && r.w <= th.w) ? 8u : 0u;
        return m;
    }
    uint32_t in = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) in |= (e0 + k >= beg && e0 + k < end) ? (1u << k) : 0u;
    const int4 c = __ldg(reinterpret_cast<const int4*>(g.col) + q);
    const uint4 lo = __ldg(g.lo4 + q);
    uint32_t m = 0;
    if ((in & 1u) && vertex_word(static_cast<uint32_t>(c.x), j, round, k0, k1) - lo.x <= th.x) m |= 1u;
    if ((in & 2u) && vertex_word(static_cast<uint32_t>(c.y), j, round, k0, k1) - lo.y <= th.y) m |= 2u;
    if ((in & 4u) && vertex_word(static_cast<uint32_t>(c.z), j, round, k0, k1) - lo.z <= th.z) m |= 4u;
    if ((in & 8u) && vertex_word(static_cast<uint32_t>(c.w), j, round, k0, k1) - lo.w <= th.w) m |= 8u;
    return m;
}

// Control block of one Alg. 2 call (zeroed before it starts).
struct RoundCtl {
    uint32_t cursor[kTiers];  // next work item of each tier
    uint32_t count[kTiers];   // samples handed to tier t (t >= 1)
    uint32_t error;           // kErr* bits
    uint32_t pad;
};

// Stats slots (unsigned long long each), kStPerTier per tier: stats[tier * kStPerTier + slot].
enum { kStSamples = 0, kStReached, kStExamined, kStLive, kStNontree, kStPasses, kStPerTier,
       kStCount = kStPerTier * kTiers };

struct SampleParams {
    DevGraph g;
    const int32_t* seeds;          // [ns]
    uint32_t ns;
    const uint32_t* excl;          // n-bit mask: seeds and blocked vertices
    uint32_t key_lo, key_hi;
    uint32_t round;
    uint32_t theta;
    unsigned long long* delta;     // [n]
    RoundCtl* ctl;
    uint32_t* lists;               // [kTiers*theta]: input list of tier t at lists + t*theta
    const int32_t* done;           // optional stop flag (GreedyReplace phase 2)
    unsigned long long* stats;     // optional [kStCount] (per-tier slots)
};

// Vertices blocked in one sample on top of excl (the spread of blocker sets scores each set on
// the same samples); kept out of SampleParams, whose size the hot kernels are sensitive to.
struct ExtraBlocked {
    const int32_t* v;
    uint32_t n;
};

// Whether v is one of the sample's extra blocked vertices (a handful at most).
__device__ __forceinline__ bool extra_blocked(const ExtraBlocked& x, uint32_t v)
{
    for (uint32_t i = 0; i < x.n; ++i)
        if (static_cast<uint32_t>(x.v[i]) == v) return true;
    return false;
}

// Capacities of one tier's per-warp working set.
struct TierCfg {
    uint32_t rcap;   // local ids incl. the super-seed (0) and the seeds
    uint32_t hcap;   // hash slots, power of two, >= 2 * rcap
    uint32_t hbits;  // log2(hcap)
    uint32_t ecap;   // non-tree edges
    uint32_t dcap;   // BFS levels
    uint8_t* gscratch;      // tiers 1-2: per-warp slots
    uint64_t warp_bytes;    // bytes per slot (tier 0: shared memory per warp)
    uint32_t from_range;    // take samples [0, theta) directly (first tier that runs)
    uint32_t next_tier;     // tier that re-runs this tier's overflowing samples
};

// Hand-off snapshot of a sample the warp tier 0 gave up on, taken at the start of the BFS level
// it could not hold: kHandoffHeader header words (sample, lb, le, nlev, nE, offsets of gid, par
// and edges, query of a batch), the level offsets lvl[0..nlev], gid[0..le), par[0..le) and the
// non-tree edges recorded before that level, as (local source, global target). The block tier
// resumes the sample from it instead of running the first levels again. Sizes follow the warp
// tier's capacities (rcap, dcap, ecap).
constexpr uint32_t kHandoffHeader = 16;
struct Handoff {
    uint32_t off_gid, off_par, off_edges, stride;
};
__host__ __device__ inline Handoff handoff_layout(uint32_t rcap, uint32_t dcap, uint32_t ecap)
{
    Handoff h;
    h.off_gid = (4u * (kHandoffHeader + dcap + 1u) + 15u) & ~15u;
    h.off_par = h.off_gid + ((4u * rcap + 15u) & ~15u);
    h.off_edges = h.off_par + ((4u * rcap + 15u) & ~15u);
    h.stride = h.off_edges + ((8u * ecap + 15u) & ~15u);
    return h;
}

// Block-per-sample tier (sample_cta.cu): per-block slot layout and shared-memory sizes.
struct CtaCfg {
    uint32_t bm_words;    // visited bitmap words (>= n/32)
    uint32_t res_slots;   // resolution hash slots (power of two)
    uint32_t res_shift;   // 32 - log2(res_slots)
    uint32_t rcap;        // local ids per slot
    uint32_t ecap;        // non-tree edges per slot
    uint32_t global_bitmap;  // 1: the bitmap is in the slot (large n); 0: in shared memory,
                             // where it also holds the resolution hash
    uint32_t tree_words;     // shared words free after the BFS for the packed tree (one per vertex)
    uint32_t handoff_stride; // 0: none; else the bytes of one warp-tier hand-off snapshot, stored
                             // by list position after the grid's slots (Handoff below)
    uint64_t off_bm, off_gid, off_par, off_idom, off_rows, off_edges, slot_bytes;
    uint8_t* scratch;
    uint32_t from_list;   // 1: take the samples that tier 0 handed over; 0: all of [0, theta)
};

// One query of a batch (batch.cu): its graph, seed set, masks, counters and results.
struct BatchQuery {
    DevGraph g;
    const int32_t* seeds;
    uint32_t ns;
    uint32_t* excl;               // seeds and blocked vertices
    uint32_t* cb;                 // GreedyReplace phase-1 candidates (N_out(S) \ S)
    uint32_t key_lo, key_hi;
    uint32_t theta;
    unsigned long long* delta;    // [n]
    int32_t* blockers;            // [b]
    int32_t count;                // AdvancedGreedy: rounds; GreedyReplace: phase-1 rounds
    int32_t* flags;               // GreedyReplace: [0] stop flag, [1] vertex unblocked this step
    uint32_t start;               // step at which the query joined: its round is step - start
    int32_t gr;                   // 1: GreedyReplace schedule, 0: AdvancedGreedy
    uint8_t* done;                // [theta] 1: the warp tier finished the sample in this step;
                                  // NULL: the query's samples all go to the block tier
};

// Queries of a batch are grouped by visited-bitmap size (n <= 2^16, 2^17, 2^18 with the bitmap
// in shared memory; larger graphs with the bitmap in each block's global slot) so that each
// group's launch reserves only the shared memory its largest graph needs.
constexpr int kBatchClasses = 4;
constexpr int kBatchGlobalClass = 3;

__host__ __device__ inline int batch_class(int32_t n)
{
    return n <= (1 << 16) ? 0 : (n <= (1 << 17) ? 1 : (n <= kCtaMaxVertices ? 2 : kBatchGlobalClass));
}

struct BatchCtl {
    unsigned long long cursor[kBatchClasses];  // next (query, sample chunk) item of each class
    uint32_t over_count;          // samples handed to the whole-graph kernel
    uint32_t over_cursor;
    uint32_t error;
    uint32_t pad;
    unsigned long long warp_cursor;  // next (query, sample chunk) item of the warp tier
    uint32_t handoff_count[kBatchClasses];   // hand-off snapshots the warp tier left per class
    uint32_t handoff_cursor[kBatchClasses];  // next snapshot the class's block launch resumes
};

// One greedy step of a batch: round `step` of every query that is still active.
struct BatchStep {
    const BatchQuery* q;
    uint32_t nq;
    const unsigned long long* prefix;  // [nq+1] first item of each query in this launch's class
                                       // (queries of other classes and inactive ones: empty)
    uint32_t chunk;                    // samples per item
    uint32_t cls;                      // size class of this launch
    uint32_t step;
    uint32_t handoff_stride;           // 0: no hand-off; else the bytes of one snapshot (Handoff)
    BatchCtl* ctl;
    uint2* over;                       // (query, sample) overflow items, then (handoff_stride != 0)
                                       // handoff_cap snapshots per size class (batch_handoff_base)
    uint32_t over_cap;
    uint32_t handoff_cap;              // hand-off snapshots per size class
    unsigned long long* stats;
    uint32_t all_ic;                   // 1: every query's graph uses the IC model
};

// The hand-off snapshots of size class k in a batched step: after the overflow items.
__host__ __device__ inline uint64_t batch_handoff_offset(uint32_t over_cap)
{
    return (8ull * over_cap + 255) & ~255ull;
}

// Byte layout of one warp's working set (same for shared and global memory).
struct WarpLayout {
    uint64_t lvl, hkey, hval, gid, idom, par, hslot, edges, total;
};

__host__ __device__ inline uint64_t align16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

__host__ __device__ inline WarpLayout warp_layout(uint32_t rcap, uint32_t hcap, uint32_t ecap,
                                                 uint32_t dcap, bool with_hslot)
{
    WarpLayout L;
    uint64_t o = 0;
    L.lvl = o;   o = align16(o + 4ull * (dcap + 1));
    L.hkey = o;  o = align16(o + 4ull * hcap);
    L.hval = o;  o = align16(o + 4ull * (hcap > rcap ? hcap : rcap));  // doubles as c[]
    L.gid = o;   o = align16(o + 4ull * rcap);
    L.idom = o;  o = align16(o + 4ull * rcap);
    L.par = o;   o = align16(o + 4ull * rcap);
    L.hslot = o; o = align16(o + (with_hslot ? 4ull * rcap : 0));
    L.edges = o; o = align16(o + 8ull * ecap);
    L.total = o;
    return L;
}

template <bool G>
struct WarpSpace {
    uint32_t* lvl;
    uint32_t* hkey;
    uint32_t* hval;
    int32_t* gid;
    uint32_t* idom;
    uint32_t* par;   // BFS parent (idom before the dominator passes)
    uint32_t* hslot;
    uint2* edges;
    uint2* stage;  // always shared memory, kStageCap entries
    uint32_t rcap, hcap, hbits, ecap, dcap;
};

// Loads of words that other lanes update with atomics or stores during the same sample.
// Global scratch is read through L2 (.cg) so that no stale L1 line is ever used.

// One step of the two-finger NCA walk over immediate dominators: the finger with the larger local
// id (the deeper one; ids follow BFS discovery order, so a dominator's id is smaller) moves to its
// immediate dominator. Written with selects, so every lane of a warp issues exactly one load per
// step whichever finger it moves.
template <typename F>
__device__ __forceinline__ void nca_step(uint32_t& a, uint32_t& b, F idom_of)
{
    const bool up_a = a > b;
    const uint32_t nx = idom_of(up_a ? a : b);
    a = up_a ? nx : a;
    b = up_a ? b : nx;
}

template <bool G>
__device__ __forceinline__ uint32_t ld_shared_word(const uint32_t* p)
{
    if constexpr (G) {
        return __ldcg(p);
    } else {
        return *reinterpret_cast<const volatile uint32_t*>(p);
    }
}

struct SampleCounters {
    unsigned long long reached = 0, examined = 0, live = 0, nontree = 0, passes = 0, done = 0;
};

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, uint32_t lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += t;
    }
    return x;
}

__device__ __forceinline__ bool excluded(const uint32_t* excl, uint32_t v)
{
    return (__ldg(excl + (v >> 5)) >> (v & 31)) & 1u;
}

enum SampleResult { kSampleDone = 0, kSampleOverflow = 1, kSampleError = 2 };

// Runs sample j of call P.round in warp space w. kClearAll: reset the whole hash afterwards
// (small shared tables) instead of the slots recorded in hslot[].
template <bool G, bool kClearAll, int M = kModelAny>
__device__ __forceinline__ int run_sample(const SampleParams& P, const WarpSpace<G>& w,
                                          uint32_t j, uint32_t lane, SampleCounters& sc,
                                          uint32_t* level_state = nullptr)
{
    const uint32_t ns = P.ns;
    const uint32_t hmask = w.hcap - 1;
    const uint32_t hshift = 32 - w.hbits;

    for (uint32_t i = lane; i < ns; i += 32) {
        w.gid[1 + i] = P.seeds[i];
        w.idom[1 + i] = 0;
        w.par[1 + i] = 0;
    }
    if (lane == 0) {
        w.idom[0] = 0;
        w.lvl[0] = 1;
        w.lvl[1] = 1 + ns;
    }
    __syncwarp();

    uint32_t nR = 1 + ns;  // local ids in use (warp-uniform)
    uint32_t nE = 0;       // non-tree edges
    uint32_t nlev = 1;     // completed levels; level d = [lvl[d], lvl[d+1])
    bool over = false;
    unsigned long long examined = 0, live = 0;

    uint32_t lb = 1, le = 1 + ns;
    uint32_t nE_level = 0;  // non-tree edges recorded before the current level
    while (lb < le) {
        nE_level = nE;
        for (uint32_t base = lb; base < le && !over; base += 32) {
            // ---- the frontier vertices of this chunk and their edge groups
            const uint32_t idx = base + lane;
            int32_t beg = 0, end = 0;
            if (idx < le) {
                const int32_t u = w.gid[idx];
                beg = __ldg(P.g.row_ptr + u);
                end = __ldg(P.g.row_ptr + u + 1);
            }
            examined += static_cast<uint32_t>(end - beg);
            const uint32_t ng =
                end > beg ? (static_cast<uint32_t>(end - 1) >> 2) - (static_cast<uint32_t>(beg) >> 2) + 1
                          : 0u;
            const uint32_t incl = warp_incl_scan(ng, lane);
            const uint32_t total = __shfl_sync(kFull, incl, 31);

            for (uint32_t t0 = 0; t0 < total && !over; t0 += 32) {
                const uint32_t t = t0 + lane;
                // owner lane: the first lane whose inclusive group count exceeds t
                uint32_t pos = 0;
#pragma unroll
                for (uint32_t step = 16; step >= 1; step >>= 1) {
                    const uint32_t v = __shfl_sync(kFull, incl, pos + step - 1);
                    if (v <= t) pos += step;
                }
                const uint32_t o_incl = __shfl_sync(kFull, incl, pos);
                const uint32_t o_ng = __shfl_sync(kFull, ng, pos);
                const int32_t o_beg = __shfl_sync(kFull, beg, pos);
                const int32_t o_end = __shfl_sync(kFull, end, pos);

                bool ok0 = false, ok1 = false, ok2 = false, ok3 = false;
                uint32_t v0 = 0, v1 = 0, v2 = 0, v3 = 0;
                const uint32_t ul = base + pos;
                if (t < total) {
                    const uint32_t q = (static_cast<uint32_t>(o_beg) >> 2) + (t - (o_incl - o_ng));
                    const uint4 th = __ldg(P.g.thr4 + q);
                    const int32_t e0 = static_cast<int32_t>(q << 2);
                    // the IC decision of group_live written out as four flags (measured 2-5 %
                    // faster on the warp tiers than testing a materialised mask)
                    if (M == kModelIC || (M == kModelAny && P.g.lo4 == nullptr)) {
                        const uint4 r = philox4x32_10(make_uint4(q, j, P.round, 0u), P.key_lo, P.key_hi);
                        ok0 = (e0 + 0 >= o_beg) && (e0 + 0 < o_end) && (r.x <= th.x);
                        ok1 = (e0 + 1 >= o_beg) && (e0 + 1 < o_end) && (r.y <= th.y);
                        ok2 = (e0 + 2 >= o_beg) && (e0 + 2 < o_end) && (r.z <= th.z);
                        ok3 = (e0 + 3 >= o_beg) && (e0 + 3 < o_end) && (r.w <= th.w);
                    } else {
                        const uint32_t lm = group_live<M>(P.g, q, th, o_beg, o_end, j, P.round, P.key_lo, P.key_hi);
                        ok0 = (lm & 1u) != 0;
                        ok1 = (lm & 2u) != 0;
                        ok2 = (lm & 4u) != 0;
                        ok3 = (lm & 8u) != 0;
                    }
                    if (ok0) { v0 = static_cast<uint32_t>(__ldg(P.g.col + e0 + 0)); ok0 = !excluded(P.excl, v0); }
                    if (ok1) { v1 = static_cast<uint32_t>(__ldg(P.g.col + e0 + 1)); ok1 = !excluded(P.excl, v1); }
                    if (ok2) { v2 = static_cast<uint32_t>(__ldg(P.g.col + e0 + 2)); ok2 = !excluded(P.excl, v2); }
                    if (ok3) { v3 = static_cast<uint32_t>(__ldg(P.g.col + e0 + 3)); ok3 = !excluded(P.excl, v3); }
                }
                const uint32_t nc = (uint32_t)ok0 + (uint32_t)ok1 + (uint32_t)ok2 + (uint32_t)ok3;
                live += nc;
                const uint32_t cincl = warp_incl_scan(nc, lane);
                const uint32_t ctot = __shfl_sync(kFull, cincl, 31);
                if (ctot == 0) continue;
                {
                    uint32_t p = cincl - nc;
                    if (ok0) w.stage[p++] = make_uint2(ul, v0);
                    if (ok1) w.stage[p++] = make_uint2(ul, v1);
                    if (ok2) w.stage[p++] = make_uint2(ul, v2);
                    if (ok3) w.stage[p++] = make_uint2(ul, v3);
                }
                __syncwarp();

                // ---- insert the staged live targets, one per lane per step
                for (uint32_t s0 = 0; s0 < ctot; s0 += 32) {
                    const bool act = s0 + lane < ctot;
                    uint32_t st = 0, slot = 0, cu = 0, cv = 0;
                    if (act) {
                        const uint2 c = w.stage[s0 + lane];
                        cu = c.x;
                        cv = c.y;
                        slot = (cv * 0x9E3779B1u) >> hshift;
                        for (uint32_t probe = 0; probe < w.hcap; ++probe) {
                            const uint32_t k = ld_shared_word<G>(w.hkey + slot);
                            if (k == cv) { st = 2; break; }
                            if (k == kEmpty) {
                                const uint32_t prev = atomicCAS(w.hkey + slot, kEmpty, cv);
                                if (prev == kEmpty) { st = 1; break; }
                                if (prev == cv) { st = 2; break; }
                            }
                            slot = (slot + 1) & hmask;
                        }
                    }
                    const uint32_t won = __ballot_sync(kFull, st == 1);
                    const uint32_t lid = nR + __popc(won & lanemask_lt());
                    bool bad = act && st == 0;  // table full: cannot happen below capacity
                    if (st == 1) {
                        if (lid < w.rcap) {
                            w.hval[slot] = lid;
                            w.gid[lid] = static_cast<int32_t>(cv);
                            w.idom[lid] = cu;
                            w.par[lid] = cu;
                            if constexpr (!kClearAll) w.hslot[lid] = slot;
                        } else {
                            w.hkey[slot] = kEmpty;  // this lane owns the slot; undo it
                            bad = true;
                        }
                    }
                    nR += __popc(won);
                    __syncwarp();
                    bool nt = false;
                    uint32_t vl = 0;
                    if (st == 2) {
                        vl = ld_shared_word<G>(w.hval + slot);
                        nt = vl != cu;  // a self-loop never matters
                    }
                    const uint32_t ntm = __ballot_sync(kFull, nt);
                    const uint32_t epos = nE + __popc(ntm & lanemask_lt());
                    if (nt && epos < w.ecap) w.edges[epos] = make_uint2(cu, vl);
                    nE += __popc(ntm);
                    if (__any_sync(kFull, bad) || nE > w.ecap || nR > w.rcap) over = true;
                }
                __syncwarp();
            }
        }
        if (over) break;
        if (nR > le) {
            if (nlev + 1 > w.dcap) { over = true; break; }
            if (lane == 0) w.lvl[nlev + 1] = nR;
            ++nlev;
        }
        lb = le;
        le = nR;
        __syncwarp();
    }

    if (over) {
        if (level_state != nullptr) {  // where a hand-off would resume: the start of this level
            level_state[0] = lb;
            level_state[1] = le;
            level_state[2] = nlev;
            level_state[3] = nE_level;
        }
        // abandon: clear every hash slot this sample used
        if constexpr (kClearAll) {
            for (uint32_t i = lane; i < w.hcap; i += 32) w.hkey[i] = kEmpty;
        } else {
            const uint32_t lim = nR < w.rcap ? nR : w.rcap;
            for (uint32_t i = 1 + ns + lane; i < lim; i += 32) w.hkey[w.hslot[i]] = kEmpty;
        }
        __syncwarp();
        return kSampleOverflow;
    }

    // ---- immediate dominators: iterate NCA(idom(v), p) over non-tree edges to the fixed point
    uint32_t passes = 0;
    bool broken = false;
    if (nE > 0) {
        for (;;) {
            bool changed = false;
            for (uint32_t k = lane; k < nE; k += 32) {
                const uint2 e = w.edges[k];
                uint32_t a = ld_shared_word<G>(w.idom + e.y);
                uint32_t b = e.x;
                // both chains strictly decrease towards the super-seed (id 0)
                for (uint32_t guard = 0; a != b; ++guard) {
                    if (guard > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, [&](uint32_t x) { return ld_shared_word<G>(w.idom + x); });
                }
                b = w.par[e.y];
                for (uint32_t guard = 0; a != b; ++guard) {
                    if (guard > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, [&](uint32_t x) { return ld_shared_word<G>(w.idom + x); });
                }
                if (!broken && a < ld_shared_word<G>(w.idom + e.y)) {
                    const uint32_t old = atomicMin(w.idom + e.y, a);
                    changed |= a < old;
                }
            }
            ++passes;
            broken = __any_sync(kFull, broken);
            if (broken || !__any_sync(kFull, changed)) break;
            if (passes > nR + 1) { broken = true; break; }  // a monotone descent cannot take longer
        }
    }
    __syncwarp();

    // ---- subtree sizes, deepest level first
    uint32_t* c = w.hval;
    for (uint32_t i = lane; i < nR; i += 32) c[i] = 1;
    __syncwarp();
    for (uint32_t d = nlev - 1; d >= 1; --d) {
        const uint32_t b0 = w.lvl[d], b1 = w.lvl[d + 1];
        for (uint32_t i = b0 + lane; i < b1; i += 32)
            atomicAdd(c + ld_shared_word<G>(w.idom + i), ld_shared_word<G>(c + i));
        __syncwarp();
    }

    // ---- publish: Delta[u] += c[u] for reached non-seeds; then clear the hash
    for (uint32_t i = 1 + ns + lane; i < nR; i += 32)
        atomicAdd(P.delta + w.gid[i], static_cast<unsigned long long>(ld_shared_word<G>(c + i)));
    if constexpr (kClearAll) {
        for (uint32_t i = lane; i < w.hcap; i += 32) w.hkey[i] = kEmpty;
    } else {
        for (uint32_t i = 1 + ns + lane; i < nR; i += 32) w.hkey[w.hslot[i]] = kEmpty;
    }
    __syncwarp();

    sc.reached += nR - 1;
    sc.examined += examined;
    sc.live += live;
    sc.nontree += nE;
    sc.passes += passes;
    sc.done += 1;
    return broken ? kSampleError : kSampleDone;
}

// Writes the hand-off snapshot (Handoff, at hb) of the sample in warp space w that run_sample
// just gave up on, from the level state it reported (at: lb, le, nlev, nE at the start of the
// level it could not hold); q is the sample's query in a batch (0 otherwise). The warp's arrays
// still hold the sample: the abandon only cleared its hash keys.
template <bool G>
__device__ __forceinline__ void write_handoff(const WarpSpace<G>& w, uint32_t lane, uint8_t* hb, const Handoff& h,
                                              uint32_t j, uint32_t q, const uint32_t at[4])
{
    uint32_t* hdr = reinterpret_cast<uint32_t*>(hb);
    const uint32_t le = at[1], nlev = at[2], ne = at[3];
    if (lane == 0) {
        hdr[0] = j;
        hdr[1] = at[0];
        hdr[2] = le;
        hdr[3] = nlev;
        hdr[4] = ne;
        hdr[5] = h.off_gid;
        hdr[6] = h.off_par;
        hdr[7] = h.off_edges;
        hdr[8] = q;
    }
    for (uint32_t i = lane; i <= nlev; i += 32) hdr[kHandoffHeader + i] = w.lvl[i];
    int32_t* hg = reinterpret_cast<int32_t*>(hb + h.off_gid);
    uint32_t* hp = reinterpret_cast<uint32_t*>(hb + h.off_par);
    for (uint32_t i = lane; i < le; i += 32) {
        hg[i] = w.gid[i];
        hp[i] = w.par[i];
    }
    uint2* he = reinterpret_cast<uint2*>(hb + h.off_edges);
    for (uint32_t k = lane; k < ne; k += 32) {
        const uint2 e = w.edges[k];
        he[k] = make_uint2(e.x, static_cast<uint32_t>(w.gid[e.y]));
    }
    __syncwarp();
}


}  // namespace imin
