// sample_cta.cu -- CTA-per-sample tier of Alg. 2 for graphs whose visited bitmap fits in
// shared memory (n <= 2^18).
//
// One 128-thread block owns one sampled graph at a time (persistent over the samples of the
// call through an atomic cursor):
//   * visited set: an n-bit bitmap in shared memory; discovering a vertex is one shared-memory
//     atomicOr, so no cascade size ever overflows the visited structure;
//   * BFS level by level: the frontier's out-edges are flattened into 4-edge groups over the
//     block (block-wide scan, binary search for the owner row); each thread loads 4 thresholds
//     with one 16-byte load and decides them with one Philox4x32-10 call; targets are loaded
//     only for live edges;
//   * per-vertex arrays indexed by local id (BFS discovery order) -- global id, BFS parent,
//     immediate dominator -- live in a per-block slot of global memory that is written once
//     per discovery and read back densely, so it streams through L2;
//   * live edges to already-visited vertices ("non-tree" edges) are rare; their targets are
//     resolved from global to local ids afterwards through a small hash built in the (then
//     cleared) bitmap space;
//   * dominators, subtree sizes and the counter update follow the same scheme as the warp
//     tiers (imin_dev.cuh): iterated NCA folding over non-tree edges plus each target's BFS
//     parent, a deepest-level-first subtree sweep, and 64-bit atomics into Delta.
// A sample that exceeds the non-tree edge capacity or the level capacity is abandoned and
// handed to the whole-graph warp tier (tier 2).
#include <algorithm>
#include <cstdlib>

#include "internal.h"

namespace imin {

namespace {

constexpr uint32_t kCtaThreads = 128;
constexpr uint32_t kCtaWarps = kCtaThreads / 32;
constexpr uint32_t kCtaLevels = 256;

struct CtaShared {
    uint32_t incl[kCtaThreads];
    int32_t beg[kCtaThreads];
    int32_t end[kCtaThreads];
    uint32_t lvl[kCtaLevels + 1];
    uint32_t wsum[kCtaWarps];
    uint32_t item, nR, nE, flag;
};

__device__ __forceinline__ uint32_t block_incl_scan(uint32_t x, uint32_t tid, CtaShared& sh,
                                                    uint32_t* total)
{
    const uint32_t lane = tid & 31, wid = tid >> 5;
    uint32_t incl = warp_incl_scan(x, lane);
    if (lane == 31) sh.wsum[wid] = incl;
    __syncthreads();
    uint32_t off = 0, tot = 0;
#pragma unroll
    for (uint32_t w = 0; w < kCtaWarps; ++w) {
        const uint32_t s = sh.wsum[w];
        if (w < wid) off += s;
        tot += s;
    }
    *total = tot;
    return incl + off;
}

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
    uint2* edges;
};

__device__ __forceinline__ int run_sample_cta(const SampleParams& P, const CtaCfg& C, uint32_t* bm,
                                              CtaShared& sh, const Slot& S, uint32_t j,
                                              uint32_t tid, SampleCounters& sc,
                                              unsigned long long& examined, unsigned long long& live)
{
    const uint32_t ns = P.ns;
    for (uint32_t i = tid; i < ns; i += kCtaThreads) {
        S.gid[1 + i] = P.seeds[i];
        S.idom[1 + i] = 0;
        S.par[1 + i] = 0;
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

    uint32_t lb = 1, le = 1 + ns, nlev = 1;
    unsigned long long ex = 0, lv = 0;
    bool over = false;
    while (lb < le) {
        for (uint32_t base = lb; base < le; base += kCtaThreads) {
            const uint32_t idx = base + tid;
            int32_t beg = 0, end = 0;
            if (idx < le) {
                const int32_t u = S.gid[idx];
                beg = __ldg(P.g.row_ptr + u);
                end = __ldg(P.g.row_ptr + u + 1);
            }
            ex += static_cast<uint32_t>(end - beg);
            const uint32_t ng =
                end > beg ? (static_cast<uint32_t>(end - 1) >> 2) - (static_cast<uint32_t>(beg) >> 2) + 1
                          : 0u;
            uint32_t total;
            const uint32_t incl = block_incl_scan(ng, tid, sh, &total);
            sh.incl[tid] = incl;
            sh.beg[tid] = beg;
            sh.end[tid] = end;
            __syncthreads();
            for (uint32_t t = tid; t < total; t += kCtaThreads) {
                uint32_t pos = 0;
#pragma unroll
                for (uint32_t step = kCtaThreads / 2; step >= 1; step >>= 1)
                    if (sh.incl[pos + step - 1] <= t) pos += step;
                const int32_t ob = sh.beg[pos], oe = sh.end[pos];
                const uint32_t first = pos ? sh.incl[pos - 1] : 0u;
                const uint32_t q = (static_cast<uint32_t>(ob) >> 2) + (t - first);
                const uint4 th = __ldg(P.g.thr4 + q);
                const uint4 r = philox4x32_10(make_uint4(q, j, P.round, 0u), P.key_lo, P.key_hi);
                const int32_t e0 = static_cast<int32_t>(q << 2);
                const uint32_t ul = base + pos;
                const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
                const uint32_t tw[4] = {th.x, th.y, th.z, th.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int32_t e = e0 + i;
                    if (e < ob || e >= oe || rw[i] > tw[i]) continue;
                    const uint32_t v = static_cast<uint32_t>(__ldg(P.g.col + e));
                    if (excluded(P.excl, v)) continue;
                    ++lv;
                    const uint32_t bit = 1u << (v & 31);
                    const uint32_t old = atomicOr(bm + (v >> 5), bit);
                    if ((old & bit) == 0) {
                        const uint32_t lid = atomicAdd(&sh.nR, 1u);
                        if (lid < C.rcap) {
                            S.gid[lid] = static_cast<int32_t>(v);
                            S.par[lid] = ul;
                            S.idom[lid] = ul;
                        } else {
                            sh.flag = 1;
                        }
                    } else {
                        const uint32_t pe = atomicAdd(&sh.nE, 1u);
                        if (pe < C.ecap) S.edges[pe] = make_uint2(ul, v);
                        else sh.flag = 1;
                    }
                }
            }
            __syncthreads();
        }
        const uint32_t nR = *reinterpret_cast<volatile uint32_t*>(&sh.nR);
        if (*reinterpret_cast<volatile uint32_t*>(&sh.flag)) { over = true; break; }
        if (nR > le) {
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

    // non-tree edge targets: global id -> local id through a hash in the bitmap space
    if (nE > 0) {
        uint32_t* keys = bm;
        uint32_t* vals = bm + C.res_slots;
        const uint32_t hmask = C.res_slots - 1;
        for (uint32_t i = tid; i < C.res_slots; i += kCtaThreads) keys[i] = kEmpty;
        __syncthreads();
        for (uint32_t k = tid; k < nE; k += kCtaThreads)
            res_slot(keys, hmask, C.res_shift, S.edges[k].y, true);
        __syncthreads();
        for (uint32_t i = 1 + ns + tid; i < nR; i += kCtaThreads) {
            const uint32_t s = res_slot(keys, hmask, C.res_shift, static_cast<uint32_t>(S.gid[i]), false);
            if (s != kEmpty) vals[s] = i;
        }
        __syncthreads();
        for (uint32_t k = tid; k < nE; k += kCtaThreads) {
            const uint32_t s = res_slot(keys, hmask, C.res_shift, S.edges[k].y, false);
            if (s == kEmpty) broken = true;  // every target was reached: cannot happen
            else S.edges[k].y = vals[s];
        }
        __syncthreads();
        for (uint32_t i = tid; i < 2 * C.res_slots; i += kCtaThreads) bm[i] = 0;
        broken = __syncthreads_or(broken);
        if (broken) return kSampleError;
    }

    // immediate dominators: fold NCA(idom(v), p, parent(v)) over the non-tree edges
    uint32_t passes = 0;
    if (nE > 0) {
        for (;;) {
            int changed = 0;
            for (uint32_t k = tid; k < nE; k += kCtaThreads) {
                const uint2 e = S.edges[k];
                uint32_t a = __ldcg(S.idom + e.y), b = e.x;
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    if (a > b) a = __ldcg(S.idom + a);
                    else b = __ldcg(S.idom + b);
                }
                b = S.par[e.y];
                for (uint32_t g = 0; a != b; ++g) {
                    if (g > 2 * nR) { broken = true; a = 0; break; }
                    if (a > b) a = __ldcg(S.idom + a);
                    else b = __ldcg(S.idom + b);
                }
                if (!broken && a < __ldcg(S.idom + e.y)) {
                    const uint32_t old = atomicMin(S.idom + e.y, a);
                    changed |= a < old;
                }
            }
            ++passes;
            broken = __syncthreads_or(broken);
            if (broken || !__syncthreads_or(changed)) break;
            if (passes > nR + 1) { broken = true; break; }
        }
    }

    // subtree sizes, deepest level first (c reuses the parent array)
    uint32_t* c = S.par;
    for (uint32_t i = tid; i < nR; i += kCtaThreads) c[i] = 1;
    __syncthreads();
    for (uint32_t d = nlev - 1; d >= 1; --d) {
        const uint32_t b0 = sh.lvl[d], b1 = sh.lvl[d + 1];
        for (uint32_t i = b0 + tid; i < b1; i += kCtaThreads)
            atomicAdd(c + __ldcg(S.idom + i), __ldcg(c + i));
        __syncthreads();
    }
    for (uint32_t i = 1 + ns + tid; i < nR; i += kCtaThreads)
        atomicAdd(P.delta + S.gid[i], static_cast<unsigned long long>(__ldcg(c + i)));
    __syncthreads();

    if (tid == 0) {
        sc.reached += nR - 1;
        sc.nontree += nE;
        sc.passes += passes;
        sc.done += 1;
    }
    return broken ? kSampleError : kSampleDone;
}

__global__ void __launch_bounds__(kCtaThreads, 8) k_sample_cta(SampleParams P, CtaCfg C)
{
    extern __shared__ __align__(16) uint32_t bm[];
    __shared__ CtaShared sh;
    const uint32_t tid = threadIdx.x;
    if (P.done != nullptr && *reinterpret_cast<const volatile int32_t*>(P.done) != 0) return;

    uint8_t* base = C.scratch + static_cast<uint64_t>(blockIdx.x) * C.slot_bytes;
    Slot S;
    S.gid = reinterpret_cast<int32_t*>(base + C.off_gid);
    S.par = reinterpret_cast<uint32_t*>(base + C.off_par);
    S.idom = reinterpret_cast<uint32_t*>(base + C.off_idom);
    S.edges = reinterpret_cast<uint2*>(base + C.off_edges);

    for (uint32_t i = tid; i < C.bm_words; i += kCtaThreads) bm[i] = 0;
    SampleCounters sc;
    unsigned long long examined = 0, live = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) sh.item = atomicAdd(&P.ctl->cursor[kTierCta], 1u);
        __syncthreads();
        const uint32_t j = sh.item;
        if (j >= P.theta) break;
        const int rc = run_sample_cta(P, C, bm, sh, S, j, tid, sc, examined, live);
        if (tid == 0) {
            if (rc == kSampleOverflow) {
                const uint32_t pos = atomicAdd(&P.ctl->count[kTierWhole], 1u);
                P.lists[kTierWhole * P.theta + pos] = j;
            } else if (rc == kSampleError) {
                atomicOr(&P.ctl->error, kErrInternal);
            }
        }
    }

    if (P.stats != nullptr) {
        // examined/live were counted per thread; everything else by thread 0
        const uint32_t lane = tid & 31;
        unsigned long long ex = examined, lv = live;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            ex += __shfl_down_sync(kFull, ex, o);
            lv += __shfl_down_sync(kFull, lv, o);
        }
        unsigned long long* st = P.stats + kTierCta * kStPerTier;
        if (lane == 0) {
            if (ex) atomicAdd(st + kStExamined, ex);
            if (lv) atomicAdd(st + kStLive, lv);
        }
        if (tid == 0 && sc.done > 0) {
            atomicAdd(st + kStSamples, sc.done);
            atomicAdd(st + kStReached, sc.reached);
            atomicAdd(st + kStNontree, sc.nontree);
            atomicAdd(st + kStPasses, sc.passes);
        }
    }
}

}  // namespace

bool plan_cta_tier(const DeviceInfo& dev, int32_t n, CtaCfg* c, uint32_t* blocks, uint64_t* smem,
                   uint64_t* scratch_bytes)
{
    if (n > kCtaMaxVertices) return false;
    const uint32_t words = std::max<uint32_t>((static_cast<uint32_t>(n) + 31) / 32, 2048);
    uint32_t slots = 1;
    while (2 * slots * 2 <= words) slots <<= 1;  // keys + values fit in the bitmap space
    c->bm_words = words;
    c->res_slots = slots;
    uint32_t bits = 0;
    while ((1u << bits) < slots) ++bits;
    c->res_shift = 32 - bits;
    c->rcap = static_cast<uint32_t>(n) + 1;
    c->ecap = slots / 2;
    if (const char* cap = std::getenv("IMIN_CTA_EDGE_CAP")) {  // test hook: force overflows
        const uint32_t v = static_cast<uint32_t>(std::strtoul(cap, nullptr, 10));
        if (v > 0) c->ecap = std::min(c->ecap, v);
    }
    uint64_t o = 0;
    c->off_gid = o;   o = align16(o + 4ull * c->rcap);
    c->off_par = o;   o = align16(o + 4ull * c->rcap);
    c->off_idom = o;  o = align16(o + 4ull * c->rcap);
    c->off_edges = o; o = align16(o + 8ull * c->ecap);
    c->slot_bytes = (o + 255) & ~255ull;
    *smem = 4ull * words;
    if (*smem > dev.smem_optin) return false;
    cudaFuncSetAttribute(k_sample_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(*smem));
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_cta, kCtaThreads, *smem);
    if (occ <= 0) return false;
    *blocks = static_cast<uint32_t>(occ) * dev.sms;
    *scratch_bytes = c->slot_bytes * *blocks;
    return true;
}

cudaError_t launch_cta_tier(const SampleParams& P, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                            uint8_t* scratch, cudaStream_t s)
{
    CtaCfg cfg = c;
    cfg.scratch = scratch;
    k_sample_cta<<<blocks, kCtaThreads, smem, s>>>(P, cfg);
    return cudaGetLastError();
}

}  // namespace imin
