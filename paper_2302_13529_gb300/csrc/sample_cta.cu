// sample_cta.cu -- single-query launch of the block-per-sample tier of Alg. 2 (the routine is
// in sample_cta.cuh): a persistent grid of blocks takes samples from an atomic cursor
// -- all of [0, theta), or the samples the warp tier 0 handed over when it ran first -- and a
// sample the block tier cannot hold is handed to the whole-graph warp tier.
#include <algorithm>
#include <cstdlib>

#include "internal.h"

#include "sample_cta.cuh"

namespace imin {

namespace {

using namespace cta;

// kSmemBitmap: the visited bitmap lives in shared memory (n <= 2^18) and doubles as the
// resolution hash; otherwise it lives in the block's global slot and the dynamic shared memory
// holds only the resolution hash.
template <bool kSmemBitmap, int M>
__global__ void __launch_bounds__(cta_threads<kSmemBitmap>(), 1024 / cta_threads<kSmemBitmap>()) k_sample_cta(SampleParams P, CtaCfg C)
{
    constexpr uint32_t kCtaThreads = cta_threads<kSmemBitmap>();
    extern __shared__ __align__(16) uint32_t dsm[];
    __shared__ CtaShared<kCtaThreads> sh;
    const uint32_t tid = threadIdx.x;
    if (P.done != nullptr && *reinterpret_cast<const volatile int32_t*>(P.done) != 0) return;

    uint8_t* base = C.scratch + static_cast<uint64_t>(blockIdx.x) * C.slot_bytes;
    Slot S;
    S.gid = reinterpret_cast<int32_t*>(base + C.off_gid);
    S.par = reinterpret_cast<uint32_t*>(base + C.off_par);
    S.idom = reinterpret_cast<uint32_t*>(base + C.off_idom);
    S.rows = reinterpret_cast<int2*>(base + C.off_rows);
    S.edges = reinterpret_cast<uint2*>(base + C.off_edges);
    uint32_t* bm = kSmemBitmap ? dsm : reinterpret_cast<uint32_t*>(base + C.off_bm);

    // a shared bitmap starts dirty; a global one is zeroed by the host and kept clean
    if constexpr (kSmemBitmap) {
        for (uint32_t i = tid; i < C.bm_words; i += kCtaThreads) bm[i] = 0;
    }
    SampleCounters sc;
    unsigned long long examined = 0, live = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) sh.item = atomicAdd(&P.ctl->cursor[kTierCta], 1u);
        __syncthreads();
        const uint32_t total =
            C.from_list ? *reinterpret_cast<const volatile uint32_t*>(&P.ctl->count[kTierCta]) : P.theta;
        if (sh.item >= total) break;
        const uint32_t j = C.from_list ? P.lists[kTierCta * P.theta + sh.item] : sh.item;
        int rc;
        if (C.handoff_stride != 0) {
            // the warp tier left this sample's state at the level it could not hold: resume there
            const uint8_t* hb = C.scratch + static_cast<uint64_t>(gridDim.x) * C.slot_bytes +
                                static_cast<uint64_t>(sh.item) * C.handoff_stride;
            uint32_t from[3];
            restore_handoff<kCtaThreads>(P, hb, S, bm, sh, tid, from);
            rc = run_sample_cta<kSmemBitmap, false, M>(P, C, bm, dsm, sh, S, j, tid, sc, examined, live,
                                                       ExtraBlocked{nullptr, 0u}, from);
        } else {
            rc = run_sample_cta<kSmemBitmap, false, M>(P, C, bm, dsm, sh, S, j, tid, sc, examined, live);
        }
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

bool plan_cta_tier(const DeviceInfo& dev, int32_t n, int32_t m, CtaCfg* c, uint32_t* blocks, uint64_t* smem,
                   uint64_t* scratch_bytes)
{
    const bool smem_bitmap = n <= kCtaMaxVertices;
    const uint32_t nwords = (static_cast<uint32_t>(n) + 31) / 32;
    uint32_t slots = 1;
    if (smem_bitmap) {
        c->bm_words = std::max<uint32_t>(nwords, 2048);
        while (2 * slots * 2 <= c->bm_words) slots <<= 1;  // keys + values fit in the bitmap space
    } else {
        c->bm_words = nwords;
        slots = 2048;  // 16 KB of shared memory for the resolution hash
    }
    c->global_bitmap = smem_bitmap ? 0u : 1u;
    c->handoff_stride = 0;  // set per query when the warp tier runs in front (api.cu)
    c->tree_words = smem_bitmap ? c->bm_words : 2 * slots;
    c->res_slots = slots;
    uint32_t bits = 0;
    while ((1u << bits) < slots) ++bits;
    c->res_shift = 32 - bits;
    // every reached vertex fits when the bitmap is shared; large graphs cap the slot arrays and
    // hand bigger cascades to the whole-graph tier
    c->rcap = smem_bitmap ? static_cast<uint32_t>(n) + 1
                          : static_cast<uint32_t>(std::min<int64_t>(static_cast<int64_t>(n) + 1, 1 << 18));
    c->ecap = static_cast<uint32_t>(std::min<int64_t>(16384, std::max<int64_t>(m, 1)));
    if (const char* cap = std::getenv("IMIN_CTA_EDGE_CAP")) {  // test hook: force overflows
        const uint32_t v = static_cast<uint32_t>(std::strtoul(cap, nullptr, 10));
        if (v > 0) c->ecap = std::min(c->ecap, v);
    }
    // test and profiling hook: fewer local ids per slot on large graphs (smaller scratch; bigger
    // cascades go to the whole-graph tier)
    if (const char* cap = std::getenv("IMIN_CTA_VERTEX_CAP"); cap && !smem_bitmap) {
        const uint32_t v = static_cast<uint32_t>(std::strtoul(cap, nullptr, 10));
        if (v > 0) c->rcap = std::max<uint32_t>(std::min(c->rcap, v), 2u);
    }
    uint64_t o = 0;
    c->off_bm = o;    o = align16(o + (smem_bitmap ? 0ull : 4ull * c->bm_words));
    c->off_gid = o;   o = align16(o + 4ull * c->rcap);
    c->off_par = o;   o = align16(o + 4ull * c->rcap);
    c->off_idom = o;  o = align16(o + 4ull * c->rcap);
    c->off_rows = o;  o = align16(o + 8ull * c->rcap);
    c->off_edges = o; o = align16(o + 8ull * c->ecap);
    c->slot_bytes = (o + 255) & ~255ull;
    *smem = smem_bitmap ? 4ull * c->bm_words : 8ull * slots;
    if (*smem > dev.smem_optin) return false;
    int occ = 0;
    if (smem_bitmap) {
        allow_max_dynamic_smem(k_sample_cta<true, kModelLT>, dev);
        allow_max_dynamic_smem(k_sample_cta<true, kModelIC>, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_cta<true, kModelIC>, cta_threads<true>(), *smem);
    } else {
        allow_max_dynamic_smem(k_sample_cta<false, kModelLT>, dev);
        allow_max_dynamic_smem(k_sample_cta<false, kModelIC>, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_cta<false, kModelIC>, cta_threads<false>(), *smem);
    }
    if (occ <= 0) return false;
    *blocks = static_cast<uint32_t>(occ) * dev.sms;
    *scratch_bytes = c->slot_bytes * *blocks;
    return true;
}

cudaError_t prepare_cta_scratch(const CtaCfg& c, uint32_t blocks, uint8_t* scratch, cudaStream_t s)
{
    if (!c.global_bitmap) return cudaSuccess;
    // zero every slot's bitmap (the kernel keeps them zero afterwards)
    return cudaMemset2DAsync(scratch + c.off_bm, c.slot_bytes, 0, 4ull * c.bm_words, blocks, s);
}

cudaError_t launch_cta_tier(const SampleParams& P, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                            uint8_t* scratch, cudaStream_t s)
{
    CtaCfg cfg = c;
    cfg.scratch = scratch;
    const bool lt = P.g.lo4 != nullptr;
    if (c.global_bitmap) {
        if (lt) k_sample_cta<false, kModelLT><<<blocks, cta_threads<false>(), smem, s>>>(P, cfg);
        else k_sample_cta<false, kModelIC><<<blocks, cta_threads<false>(), smem, s>>>(P, cfg);
    } else {
        if (lt) k_sample_cta<true, kModelLT><<<blocks, cta_threads<true>(), smem, s>>>(P, cfg);
        else k_sample_cta<true, kModelIC><<<blocks, cta_threads<true>(), smem, s>>>(P, cfg);
    }
    return cudaGetLastError();
}

}  // namespace imin
