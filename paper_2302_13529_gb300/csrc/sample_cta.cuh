// sample_cta.cuh -- the block-per-sample routine of Alg. 2, shared by the single-query kernel
// (sample_cta.cu), the batched multi-query kernel (batch.cu) and the spread estimate (spread.cu).
// The visited bitmap is in shared memory for graphs of up to 2^18 vertices and in the block's
// global slot for larger ones.
//
// One block owns one sampled graph at a time (persistent over the samples of the call through
// an atomic cursor); it has 128 threads when the visited bitmap is in shared memory and 256 when
// it is in global memory (cta_threads below):
//   * visited set: an n-bit bitmap in shared memory; discovering a vertex is one shared-memory
//     atomicOr, so no cascade size ever overflows the visited structure;
//   * BFS level by level, 2 frontier vertices per thread per block-wide scan: their out-edges are
//     flattened into 4-edge groups; each thread takes one group per iteration (binary search
//     for the owner row), loads its 4 thresholds with one 16-byte load and decides them with
//     one Philox4x32-10 call;
//   * live edges (a few percent of the examined ones) accumulate in a per-warp stage across
//     iterations and are visited by the whole warp once the stage is half full (and at the end
//     of each chunk): target load, visited test-and-set, and one shared atomic per warp to hand
//     out local ids (ballot + popcount). Batching the visits keeps the dependent target loads
//     and ballots off the per-iteration path and all 32 lanes busy when they run;
//   * per-vertex arrays indexed by local id (BFS discovery order) -- global id, BFS parent,
//     immediate dominator -- live in a per-block slot of global memory that is written once
//     per discovery and read back densely, so it streams through L2;
//   * live edges to already-visited vertices ("non-tree" edges) are rare; their targets are
//     resolved from global to local ids afterwards through a small hash built in the (then
//     cleared) bitmap space, in chunks when there are many;
//   * dominators, subtree sizes and the counter update follow the same scheme as the warp
//     tiers (imin_dev.cuh): iterated NCA folding over non-tree edges plus each target's BFS
//     parent, a deepest-level-first subtree sweep, and 64-bit atomics into Delta.
// A sample that exceeds the non-tree edge capacity or the level capacity is abandoned and
// handed to the whole-graph warp tier (tier 2).
#pragma once

#include "imin_dev.cuh"

namespace imin {
namespace cta {

constexpr uint32_t kVpt = 2;        // frontier vertices per thread per chunk
constexpr uint32_t kStage = 192;    // live edges staged per warp (visited once another full
                                    // iteration might not fit)
constexpr uint32_t kCtaLevels = 512;

// Threads per block. With the visited bitmap in shared memory (n <= 2^18) a block has 128
// threads, and 8 blocks share an SM. With the bitmap in global memory (larger graphs, whose
// cascades are larger and bound by memory latency) a block has kCtaThreadsGlobal threads, so a
// cascade gets more threads and fewer cascades share an SM.
constexpr uint32_t kCtaThreadsSmem = 128;
constexpr uint32_t kCtaThreadsGlobal = 256;
template <bool kSmemBitmap>
__host__ __device__ constexpr uint32_t cta_threads()
{
    return kSmemBitmap ? kCtaThreadsSmem : kCtaThreadsGlobal;
}

template <uint32_t T>
struct CtaDims {
    static_assert(T % 32 == 0 && T <= 1024, "whole warps");
    static constexpr uint32_t kWarps = T / 32;
    static constexpr uint32_t kChunk = T * kVpt;  // frontier vertices per chunk
    // 16-bit tree entries that fit in the BFS arrays of CtaShared once the BFS is over
    static constexpr uint32_t kTree16 = (8 * kWarps * kStage + 12 * kChunk) / 2;
};

template <uint32_t T>
struct CtaShared {
    union {
        struct {
            uint2 stage[CtaDims<T>::kWarps][kStage];  // (local id of the source, edge id)
            uint32_t incl[CtaDims<T>::kChunk];        // inclusive group count of the chunk's vertices
            int32_t beg[CtaDims<T>::kChunk];          // their edge ranges
            int32_t end[CtaDims<T>::kChunk];
        } b;
        // the dominator passes of large trees: immediate dominators of local ids past the
        // resolution space, as 16-bit entries
        uint16_t tree16[CtaDims<T>::kTree16];
    };
    uint32_t lvl[kCtaLevels + 1];
    uint32_t wsum[CtaDims<T>::kWarps];
    uint32_t item, nR, nE, flag;
};

// Find-or-insert of a global id in the resolution hash (keys then values, h slots each).
__device__ __forceinline__ uint32_t res_slot(uint32_t* keys, uint32_t hmask, uint32_t hshift,
                                             uint32_t v, bool insert)
{
    uint32_t slot = (v * 0x9E3779B1u) >> hshift;
    for (uint32_t probe = 0; probe <= hmask; ++probe) {
        const uint32_t k = *reinterpret_cast<volatile uint32_t*>(keys + slot);
        if (k == v) return slot;
        if (k == kEmpty) {
            if (!insert) return kEmpty;
            const uint32_t prev = atomicCAS(keys + slot, kEmpty, v);
            if (prev == kEmpty || prev == v) return slot;
        }
        slot = (slot + 1) & hmask;
    }
    return kEmpty;
}

struct Slot {
    int32_t* gid;
    uint32_t* par;   // BFS parent; reused for subtree sizes after the dominator passes
    uint32_t* idom;
    int2* rows;      // [row_ptr[v], row_ptr[v+1]) of every reached vertex, read at its level
    uint2* edges;
};

// Visit the staged live edges of one warp: test-and-set the visited bit of each target; a new
// vertex gets the next local id (one shared atomic per warp), an old one yields a non-tree edge.
// kSpread: reachability only -- no parents, dominator seeds or non-tree edges are recorded.
template <bool kSpread, uint32_t T>
__device__ __forceinline__ void visit_staged(const SampleParams& P, const CtaCfg& C, uint32_t* bm,
                                             CtaShared<T>& sh, const Slot& S, const uint2* stage,
                                             uint32_t count, uint32_t lane,
                                             unsigned long long& lv, const ExtraBlocked& xb)
{
    for (uint32_t s0 = 0; s0 < count; s0 += 32) {
        const bool act = s0 + lane < count;
        bool disc = false, nt = false;
        uint32_t ul = 0, v = 0;
        int2 row = make_int2(0, 0);
        if (act) {
            const uint2 c = stage[s0 + lane];
            ul = c.x;
            v = static_cast<uint32_t>(__ldg(P.g.col + c.y));
            row = make_int2(__ldg(P.g.row_ptr + v), __ldg(P.g.row_ptr + v + 1));
            if (!excluded(P.excl, v) && !(kSpread && extra_blocked(xb, v))) {
                ++lv;
                const uint32_t bit = 1u << (v & 31);
                disc = (atomicOr(bm + (v >> 5), bit) & bit) == 0;
                nt = !disc;
            }
        }
        const uint32_t dm = __ballot_sync(kFull, disc);
        if (dm) {
            uint32_t b = 0;
            const uint32_t leader = __ffs(dm) - 1;
            if (lane == leader) b = atomicAdd(&sh.nR, __popc(dm));
            b = __shfl_sync(kFull, b, leader);
            if (disc) {
                const uint32_t lid = b + __popc(dm & lanemask_lt());
                if (lid < C.rcap) {
                    S.gid[lid] = static_cast<int32_t>(v);
                    if constexpr (!kSpread) {
                        S.par[lid] = ul;
                        S.idom[lid] = ul;
                    }
                    S.rows[lid] = row;
                } else {
                    sh.flag = 1;
                }
            }
        }
        if constexpr (kSpread) continue;
        const uint32_t nm = __ballot_sync(kFull, nt);
        if (nm) {
            uint32_t b = 0;
            const uint32_t leader = __ffs(nm) - 1;
            if (lane == leader) b = atomicAdd(&sh.nE, __popc(nm));
            b = __shfl_sync(kFull, b, leader);
            if (nt) {
                const uint32_t pe = b + __popc(nm & lanemask_lt());
                if (pe < C.ecap) S.edges[pe] = make_uint2(ul, v);
                else sh.flag = 1;
            }
        }
    }
}

// Loads of words that other threads update with atomics (idom, c): from L2.
__device__ __forceinline__ uint32_t ld_tree(const uint32_t* p) { return __ldcg(p); }

// Immediate dominators by folding NCA(idom(v), p, parent(v)) over the non-tree edges until a pass
// changes nothing, then subtree sizes (deepest level first) and Delta += c for reached
// non-seeds, on the slot arrays in global memory, for trees too large for shared memory (c
// reuses the parent array, which is dead once the passes end). Returns true when the iteration
// failed its bounds (cannot happen for a well-formed sample).
template <uint32_t T>
__device__ __forceinline__ bool finish_tree(const SampleParams& P, CtaShared<T>& sh, const Slot& S,
                                            uint32_t* idom, uint32_t* c, uint32_t nR, uint32_t nE,
                                            uint32_t nlev, uint32_t ns, uint32_t tid, uint32_t* passes_out)
{
    constexpr uint32_t kCtaThreads = T;
    bool broken = false;
    uint32_t passes = 0;
    if (nE > 0) {
        for (;;) {
            int changed = 0;
            for (uint32_t k = tid; k < nE; k += kCtaThreads) {
                const uint2 e = S.edges[k];
                uint32_t a = ld_tree(idom + e.y), b = e.x;
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, [&](uint32_t x) { return ld_tree(idom + x); });
                }
                b = S.par[e.y];
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, [&](uint32_t x) { return ld_tree(idom + x); });
                }
                if (!broken && a < ld_tree(idom + e.y)) {
                    const uint32_t old = atomicMin(idom + e.y, a);
                    changed |= a < old;
                }
            }
            ++passes;
            broken = __syncthreads_or(broken);
            if (broken || !__syncthreads_or(changed)) break;
            if (passes > nR + 1) { broken = true; break; }
        }
    }
    *passes_out = passes;
    for (uint32_t i = tid; i < nR; i += kCtaThreads) c[i] = 1;
    __syncthreads();
    for (uint32_t d = nlev - 1; d >= 1; --d) {
        const uint32_t b0 = sh.lvl[d], b1 = sh.lvl[d + 1];
        for (uint32_t i = b0 + tid; i < b1; i += kCtaThreads) atomicAdd(c + ld_tree(idom + i), ld_tree(c + i));
        __syncthreads();
    }
    for (uint32_t i = 1 + ns + tid; i < nR; i += kCtaThreads)
        atomicAdd(P.delta + S.gid[i], static_cast<unsigned long long>(ld_tree(c + i)));
    __syncthreads();
    return broken;
}

// The dominator passes of finish_tree on packed shared-memory words, one per local id,
// (idom << 16) | c with c = 0 (every id fits: nR <= K), so atomicMin on the word is atomicMin on
// idom.
template <uint32_t T>
__device__ __forceinline__ bool tree_passes_packed(const Slot& S, uint32_t* w, uint32_t nR, uint32_t nE,
                                                   uint32_t tid, uint32_t* passes_out)
{
    constexpr uint32_t kCtaThreads = T;
    volatile uint32_t* vw = w;
    bool broken = false;
    uint32_t passes = 0;
    if (nE > 0) {
        for (;;) {
            int changed = 0;
            for (uint32_t k = tid; k < nE; k += kCtaThreads) {
                const uint2 e = S.edges[k];
                uint32_t a = vw[e.y] >> 16, b = e.x;
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, [&](uint32_t x) { return vw[x] >> 16; });
                }
                b = S.par[e.y];
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, [&](uint32_t x) { return vw[x] >> 16; });
                }
                if (!broken && a < (vw[e.y] >> 16)) {
                    const uint32_t old = atomicMin(w + e.y, a << 16);
                    changed |= (a << 16) < old;
                }
            }
            ++passes;
            broken = __syncthreads_or(broken);
            if (broken || !__syncthreads_or(changed)) break;
            if (passes > nR + 1) { broken = true; break; }
        }
    }
    *passes_out = passes;
    return broken;
}

// Volatile 16-bit shared-memory load at a shared-space byte address.
__device__ __forceinline__ uint32_t lds_u16(uint32_t addr)
{
    unsigned short v;
    asm volatile("ld.volatile.shared.u16 %0, [%1];" : "=h"(v) : "r"(addr) : "memory");
    return v;
}

// Lower a 16-bit shared entry to min(entry, a) (compare-and-swap on its 32-bit word); 1 if it
// fell, 0 if not, -1 if the swap kept failing (cannot happen: each failure means another thread
// lowered a neighbouring or the same entry, and entries only fall).
__device__ __forceinline__ int lower16(uint16_t* p, uint32_t a)
{
    uint32_t* w = reinterpret_cast<uint32_t*>(reinterpret_cast<uintptr_t>(p) & ~static_cast<uintptr_t>(3));
    const uint32_t sh = (reinterpret_cast<uintptr_t>(p) & 2) ? 16u : 0u;
    uint32_t old = *reinterpret_cast<volatile uint32_t*>(w);
    for (uint32_t it = 0; it < (1u << 20); ++it) {
        if (a >= ((old >> sh) & 0xFFFFu)) return 0;
        const uint32_t prev = atomicCAS(w, old, (old & ~(0xFFFFu << sh)) | (a << sh));
        if (prev == old) return 1;
        old = prev;
    }
    return -1;
}

// The dominator passes of finish_tree for trees of fewer than 2^16 vertices that outgrow the
// packed words: idom as 16-bit shared entries for local ids below KA (the resolution space, 16
// bits per id) and KA .. KA + kTree16 - 1 (the BFS arrays, free once the BFS is over), the
// deepest ids in S.idom. Every NCA walk climbs to smaller ids, so almost all of its steps are
// shared-memory loads. On return S.idom holds the final immediate dominators of all ids.
template <uint32_t T>
__device__ __forceinline__ bool tree_passes16(CtaShared<T>& sh, const Slot& S, uint16_t* a16, uint32_t KA,
                                              uint32_t nR, uint32_t nE, uint32_t tid, uint32_t* passes_out)
{
    constexpr uint32_t kCtaThreads = T, kTree16 = CtaDims<T>::kTree16;
    uint16_t* b16 = sh.tree16;
    const uint32_t na = min(nR, KA), nb = min(nR, KA + kTree16);
    for (uint32_t i = tid; i < na; i += kCtaThreads) a16[i] = static_cast<uint16_t>(ld_tree(S.idom + i));
    for (uint32_t i = KA + tid; i < nb; i += kCtaThreads) b16[i - KA] = static_cast<uint16_t>(ld_tree(S.idom + i));
    __syncthreads();
    // one shared-memory load for either region (an address select, no branch)
    const uint32_t base_a = static_cast<uint32_t>(__cvta_generic_to_shared(a16));
    const uint32_t base_b = static_cast<uint32_t>(__cvta_generic_to_shared(b16));
    auto idom_of = [&](uint32_t x) -> uint32_t {
        if (x < KA + kTree16) return lds_u16(x < KA ? base_a + 2 * x : base_b + 2 * (x - KA));
        return ld_tree(S.idom + x);
    };
    bool broken = false;
    uint32_t passes = 0;
    if (nE > 0) {
        for (;;) {
            int changed = 0;
            for (uint32_t k = tid; k < nE; k += kCtaThreads) {
                const uint2 e = S.edges[k];
                uint32_t a = idom_of(e.y), b = e.x;
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, idom_of);
                }
                b = S.par[e.y];
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    nca_step(a, b, idom_of);
                }
                if (!broken && a < idom_of(e.y)) {
                    int fell;
                    if (e.y < KA) fell = lower16(a16 + e.y, a);
                    else if (e.y < KA + kTree16) fell = lower16(b16 + (e.y - KA), a);
                    else fell = a < atomicMin(S.idom + e.y, a) ? 1 : 0;
                    if (fell < 0) broken = true;
                    changed |= fell > 0;
                }
            }
            ++passes;
            broken = __syncthreads_or(broken);
            if (broken || !__syncthreads_or(changed)) break;
            if (passes > nR + 1) { broken = true; break; }
        }
    }
    *passes_out = passes;
    for (uint32_t i = tid; i < na; i += kCtaThreads) S.idom[i] = a16[i];
    for (uint32_t i = KA + tid; i < nb; i += kCtaThreads) S.idom[i] = b16[i - KA];
    __syncthreads();
    return broken;
}

// Subtree sizes (deepest level first) and Delta += c for reached non-seeds, once the immediate
// dominators are final, with the first K local ids -- the shallowest BFS levels -- as packed
// shared-memory words (idom << 16) | c and ids K..nR-1 (kSplit) on the slot arrays (idom in
// S.idom; c in S.par, which is dead once the passes end). For trees of fewer than 2^16
// vertices: c < 2^16 never carries into idom. On entry w[i] = idom(i) << 16 for i < K.
template <bool kSplit, uint32_t T>
__device__ __forceinline__ void tree_sweep_packed(const SampleParams& P, CtaShared<T>& sh, const Slot& S,
                                                  uint32_t* w, uint32_t K, uint32_t nR, uint32_t nlev,
                                                  uint32_t ns, uint32_t tid)
{
    constexpr uint32_t kCtaThreads = T;
    volatile uint32_t* vw = w;
    auto idom_of = [&](uint32_t x) -> uint32_t {
        if (!kSplit || x < K) return vw[x] >> 16;
        return __ldcg(S.idom + x);
    };
    auto c_of = [&](uint32_t x) -> uint32_t {
        if (!kSplit || x < K) return vw[x] & 0xFFFFu;
        return __ldcg(S.par + x);
    };
    for (uint32_t i = tid; i < K; i += kCtaThreads) w[i] = (vw[i] & 0xFFFF0000u) | 1u;
    if constexpr (kSplit) {
        for (uint32_t i = K + tid; i < nR; i += kCtaThreads) S.par[i] = 1;
    }
    __syncthreads();
    for (uint32_t d = nlev - 1; d >= 1; --d) {
        const uint32_t b0 = sh.lvl[d], b1 = sh.lvl[d + 1];
        for (uint32_t i = b0 + tid; i < b1; i += kCtaThreads) {
            const uint32_t x = idom_of(i), ci = c_of(i);
            if (!kSplit || x < K) atomicAdd(w + x, ci);
            else atomicAdd(S.par + x, ci);
        }
        __syncthreads();
    }
    for (uint32_t i = 1 + ns + tid; i < nR; i += kCtaThreads)
        atomicAdd(P.delta + S.gid[i], static_cast<unsigned long long>(c_of(i)));
    __syncthreads();
}

// Restores a warp-tier hand-off snapshot (Handoff, at hb) into the block's slot and visited
// bitmap and into sh, and sets from = (lb, le, nlev) for run_sample_cta: the sample continues
// at the start of the level the warp tier could not hold, with the ids, parents, level offsets
// and non-tree edges the warp tier had found before it. Ids are in the warp tier's discovery
// order, which is a BFS order like the block tier's own.
template <uint32_t T>
__device__ __forceinline__ void restore_handoff(const SampleParams& P, const uint8_t* hb, const Slot& S,
                                                uint32_t* bm, CtaShared<T>& sh, uint32_t tid, uint32_t from[3])
{
    const uint32_t* hdr = reinterpret_cast<const uint32_t*>(hb);
    const uint32_t lb = hdr[1], le = hdr[2], nlev = min(hdr[3], kCtaLevels), ne = hdr[4];
    const int32_t* hg = reinterpret_cast<const int32_t*>(hb + hdr[5]);
    const uint32_t* hp = reinterpret_cast<const uint32_t*>(hb + hdr[6]);
    const uint2* he = reinterpret_cast<const uint2*>(hb + hdr[7]);
    const uint32_t ns = P.ns;
    for (uint32_t i = tid; i < le; i += T) {
        if (i == 0) {
            S.par[0] = 0;
            S.idom[0] = 0;
            continue;
        }
        const int32_t v = hg[i];
        const uint32_t p = hp[i];
        S.gid[i] = v;
        S.par[i] = p;
        S.idom[i] = p;
        if (i >= lb) S.rows[i] = make_int2(__ldg(P.g.row_ptr + v), __ldg(P.g.row_ptr + v + 1));
        if (i >= 1 + ns) atomicOr(bm + (static_cast<uint32_t>(v) >> 5), 1u << (v & 31));
    }
    for (uint32_t k = tid; k < ne; k += T) S.edges[k] = he[k];
    for (uint32_t i = tid; i <= nlev; i += T) sh.lvl[i] = hdr[kHandoffHeader + i];
    if (tid == 0) {
        sh.nR = le;
        sh.nE = ne;
        sh.flag = 0;
    }
    from[0] = lb;
    from[1] = le;
    from[2] = nlev;
    __syncthreads();
}

// bm: visited bitmap (shared or global memory); res: 2 * C.res_slots words of shared memory for
// the non-tree target resolution -- the bitmap itself when kResInBitmap (it is cleared first).
// kSpread: only the BFS; |R| (seeds included) is added to sc.reached and the dominator step is
// skipped (the Monte-Carlo spread estimate of Def. 3); xb lists vertices blocked in this sample
// only (reachability mode). `from` (lb, le, nlev) resumes a sample at the start of a level whose
// state the caller restored (restore_handoff).
template <bool kResInBitmap, bool kSpread = false, int M = kModelAny, uint32_t T>
__device__ __forceinline__ int run_sample_cta(const SampleParams& P, const CtaCfg& C, uint32_t* bm,
                                              uint32_t* res, CtaShared<T>& sh, const Slot& S, uint32_t j,
                                              uint32_t tid, SampleCounters& sc,
                                              unsigned long long& examined, unsigned long long& live,
                                              ExtraBlocked xb = ExtraBlocked{nullptr, 0u},
                                              const uint32_t* from = nullptr)
{
    constexpr uint32_t kCtaThreads = T, kCtaWarps = CtaDims<T>::kWarps, kChunk = CtaDims<T>::kChunk;
    const uint32_t ns = P.ns;
    const uint32_t lane = tid & 31, wid = tid >> 5;
    uint32_t lb = 1, le = 1 + ns, nlev = 1;
    if (from == nullptr) {
        for (uint32_t i = tid; i < ns; i += kCtaThreads) {
            const int32_t u = P.seeds[i];
            S.gid[1 + i] = u;
            S.idom[1 + i] = 0;
            S.par[1 + i] = 0;
            S.rows[1 + i] = make_int2(__ldg(P.g.row_ptr + u), __ldg(P.g.row_ptr + u + 1));
        }
        if (tid == 0) {
            S.idom[0] = 0;
            S.par[0] = 0;
            sh.lvl[0] = 1;
            sh.lvl[1] = 1 + ns;
            sh.nR = 1 + ns;
            sh.nE = 0;
            sh.flag = 0;
        }
        __syncthreads();
    } else {
        // resumed at the start of a level: the caller restored the slot arrays of ids below le,
        // the rows of the level's vertices, the visited bits, sh.lvl, sh.nR and sh.nE
        lb = from[0];
        le = from[1];
        nlev = from[2];
    }

    unsigned long long ex = 0, lv = 0;
    bool over = false;
    while (lb < le) {
        for (uint32_t base = lb; base < le; base += kChunk) {
            // ---- the chunk's vertices (kVpt consecutive per thread) and their 4-edge groups
            int32_t beg[kVpt], end[kVpt];
            uint32_t ng[kVpt], sum = 0;
#pragma unroll
            for (uint32_t k = 0; k < kVpt; ++k) {
                const uint32_t idx = base + tid * kVpt + k;
                beg[k] = 0;
                end[k] = 0;
                if (idx < le) {
                    const int2 row = S.rows[idx];
                    beg[k] = row.x;
                    end[k] = row.y;
                }
                ex += static_cast<uint32_t>(end[k] - beg[k]);
                ng[k] = end[k] > beg[k]
                            ? (static_cast<uint32_t>(end[k] - 1) >> 2) - (static_cast<uint32_t>(beg[k]) >> 2) + 1
                            : 0u;
                sum += ng[k];
            }
            // warp-local inclusive group counts; the warps' totals locate a group's warp first,
            // so one barrier serves the whole chunk
            const uint32_t wincl = warp_incl_scan(sum, lane);
            uint32_t run = wincl - sum;
#pragma unroll
            for (uint32_t k = 0; k < kVpt; ++k) {
                run += ng[k];
                sh.b.incl[tid * kVpt + k] = run;
                sh.b.beg[tid * kVpt + k] = beg[k];
                sh.b.end[tid * kVpt + k] = end[k];
            }
            if (lane == 31) sh.wsum[wid] = wincl;
            __syncthreads();
            uint32_t woff[kCtaWarps];  // inclusive warp totals
            {
                uint32_t run = 0;
#pragma unroll
                for (uint32_t k = 0; k < kCtaWarps; ++k) {
                    run += sh.wsum[k];
                    woff[k] = run;
                }
            }
            const uint32_t total = woff[kCtaWarps - 1];

            // ---- groups: one per thread per iteration; live edges accumulate in the warp's
            // stage, which is visited by the full warp whenever it is at least half full and
            // once more at the end of the chunk
            uint32_t staged = 0;  // warp-uniform
            // the owner row and thresholds of the thread's next group are fetched while the
            // current group's Philox runs
            uint32_t nq = 0, nul = 0;
            int32_t nob = 0, noe = 0;
            uint4 nth = make_uint4(0, 0, 0, 0);
            auto fetch = [&](uint32_t t) {
                nob = 0;
                noe = 0;
                if (t < total) {
                    // the owner's warp, then the owner within the warp's kVpt * 32 entries
                    uint32_t w = 0, wb = 0;
#pragma unroll
                    for (uint32_t k = 0; k + 1 < kCtaWarps; ++k) {
                        const bool past = t >= woff[k];
                        w = past ? k + 1 : w;
                        wb = past ? woff[k] : wb;
                    }
                    const uint32_t tl = t - wb;
                    uint32_t p = w * (kVpt * 32);
#pragma unroll
                    for (uint32_t step = kVpt * 16; step >= 1; step >>= 1)
                        if (sh.b.incl[p + step - 1] <= tl) p += step;
                    nob = sh.b.beg[p];
                    noe = sh.b.end[p];
                    const uint32_t first = (p & (kVpt * 32 - 1)) ? sh.b.incl[p - 1] : 0u;
                    nq = (static_cast<uint32_t>(nob) >> 2) + (tl - first);
                    nul = base + p;
                    nth = __ldg(P.g.thr4 + nq);
                }
            };
            fetch(tid);
            for (uint32_t t0 = 0; t0 < total; t0 += kCtaThreads) {
                const uint32_t q = nq, ul = nul;
                const int32_t ob = nob, oe = noe;
                const uint4 th = nth;
                fetch(t0 + kCtaThreads + tid);
                uint32_t m = 0;
                if (oe > ob) m = group_live<M>(P.g, q, th, ob, oe, j, P.round, P.key_lo, P.key_hi);
                const uint32_t nc = __popc(m);
                const uint32_t cincl = warp_incl_scan(nc, lane);
                uint32_t w = staged + cincl - nc;
                while (m) {
                    const uint32_t i = __ffs(m) - 1;
                    m &= m - 1;
                    sh.b.stage[wid][w++] = make_uint2(ul, (q << 2) + i);
                }
                staged += __shfl_sync(kFull, cincl, 31);
                if (staged > kStage - 32 * 4) {  // the next iteration could overflow the stage
                    __syncwarp();
                    visit_staged<kSpread>(P, C, bm, sh, S, sh.b.stage[wid], staged, lane, lv, xb);
                    __syncwarp();
                    staged = 0;
                }
            }
            if (staged > 0) {
                __syncwarp();
                visit_staged<kSpread>(P, C, bm, sh, S, sh.b.stage[wid], staged, lane, lv, xb);
                __syncwarp();
            }
            __syncthreads();
        }
        const uint32_t nR = *reinterpret_cast<volatile uint32_t*>(&sh.nR);
        if (*reinterpret_cast<volatile uint32_t*>(&sh.flag)) { over = true; break; }
        if (nR > le && !kSpread) {  // level offsets feed the subtree sweep only
            if (nlev + 1 > kCtaLevels) { over = true; break; }
            if (tid == 0) sh.lvl[nlev + 1] = nR;
            ++nlev;
        }
        lb = le;
        le = nR;
    }
    __syncthreads();

    if (over) {
        for (uint32_t i = tid; i < C.bm_words; i += kCtaThreads) bm[i] = 0;
        __syncthreads();
        return kSampleOverflow;
    }
    examined += ex;
    live += lv;
    const uint32_t nR = sh.nR, nE = sh.nE;
    bool broken = false;

    // clear the visited bits (seeds were never marked)
    for (uint32_t i = 1 + ns + tid; i < nR; i += kCtaThreads) bm[S.gid[i] >> 5] = 0;
    __syncthreads();
    if constexpr (kSpread) {
        if (tid == 0) {
            sc.reached += nR - 1;
            sc.done += 1;
        }
        return kSampleDone;
    }

    // non-tree edge targets: global id -> local id through a hash in the bitmap space, in
    // chunks of at most half the hash's slots
    if (nE > 0) {
        uint32_t* keys = res;
        uint32_t* vals = res + C.res_slots;
        const uint32_t hmask = C.res_slots - 1;
        for (uint32_t c0 = 0; c0 < nE; c0 += C.res_slots / 2) {
            const uint32_t c1 = min(nE, c0 + C.res_slots / 2);
            for (uint32_t i = tid; i < C.res_slots; i += kCtaThreads) keys[i] = kEmpty;
            __syncthreads();
            for (uint32_t k = c0 + tid; k < c1; k += kCtaThreads)
                res_slot(keys, hmask, C.res_shift, S.edges[k].y, true);
            __syncthreads();
            for (uint32_t i = 1 + ns + tid; i < nR; i += kCtaThreads) {
                const uint32_t s = res_slot(keys, hmask, C.res_shift, static_cast<uint32_t>(S.gid[i]), false);
                if (s != kEmpty) vals[s] = i;
            }
            __syncthreads();
            for (uint32_t k = c0 + tid; k < c1; k += kCtaThreads) {
                const uint32_t s = res_slot(keys, hmask, C.res_shift, S.edges[k].y, false);
                if (s == kEmpty) broken = true;  // every target was reached: cannot happen
                else S.edges[k].y = vals[s];
            }
            __syncthreads();
        }
        if constexpr (kResInBitmap) {
            for (uint32_t i = tid; i < 2 * C.res_slots; i += kCtaThreads) bm[i] = 0;
        }
        broken = __syncthreads_or(broken);
        if (broken) return kSampleError;
    }

    // dominators, subtree sizes and counter update: trees that fit the (now free) resolution
    // space as packed shared-memory words entirely there; larger trees of fewer than 2^16
    // vertices with 16-bit immediate dominators in shared memory for the passes and the
    // shallowest ids packed for the sweep, the rest on the slot arrays; trees of 2^16 vertices
    // or more entirely on the slot arrays
    uint32_t passes = 0;
    if (nR < (1u << 16)) {
        const uint32_t K = min(nR, C.tree_words);
        if (K == nR) {
            for (uint32_t i = tid; i < K; i += kCtaThreads) res[i] = S.idom[i] << 16;
            __syncthreads();
            broken = tree_passes_packed<T>(S, res, nR, nE, tid, &passes);
            tree_sweep_packed<false>(P, sh, S, res, K, nR, nlev, ns, tid);
        } else {
            broken = tree_passes16(sh, S, reinterpret_cast<uint16_t*>(res), 2 * C.tree_words, nR, nE, tid,
                                   &passes);
            for (uint32_t i = tid; i < K; i += kCtaThreads) res[i] = ld_tree(S.idom + i) << 16;
            __syncthreads();
            tree_sweep_packed<true>(P, sh, S, res, K, nR, nlev, ns, tid);
        }
        if constexpr (kResInBitmap) {
            for (uint32_t i = tid; i < K; i += kCtaThreads) res[i] = 0;  // it is the bitmap
            __syncthreads();
        }
    } else {
        broken = finish_tree(P, sh, S, S.idom, S.par, nR, nE, nlev, ns, tid, &passes);
    }

    if (tid == 0) {
        sc.reached += nR - 1;
        sc.nontree += nE;
        sc.passes += passes;
        sc.done += 1;
    }
    return broken ? kSampleError : kSampleDone;
}

}  // namespace cta
}  // namespace imin
