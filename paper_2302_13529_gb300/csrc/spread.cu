// spread.cu -- the Monte-Carlo estimate of the expected spread E(S, G[V \ B]) (Def. 3; the
// paper evaluates the spread of every blocker set it reports by simulating the cascade on
// sampled graphs): the sum over theta sampled graphs of the number of vertices reachable from the
// seeds, seeds included. It runs the block-per-sample BFS of sample_cta.cuh without the
// dominator step, on the same Philox stream as Alg. 2 (sample j of call `round` under `key`).
#include "internal.h"

#include "sample_cta.cuh"

namespace imin {

namespace {

using namespace cta;

template <bool kSmemBitmap>
__global__ void __launch_bounds__(cta_threads<kSmemBitmap>(), 1024 / cta_threads<kSmemBitmap>()) k_spread_cta(SampleParams P, CtaCfg C,
                                                               unsigned long long* sum)
{
    constexpr uint32_t kCtaThreads = cta_threads<kSmemBitmap>();
    extern __shared__ __align__(16) uint32_t dsm[];
    __shared__ CtaShared<kCtaThreads> sh;
    const uint32_t tid = threadIdx.x;
    uint8_t* base = C.scratch + static_cast<uint64_t>(blockIdx.x) * C.slot_bytes;
    Slot S;
    S.gid = reinterpret_cast<int32_t*>(base + C.off_gid);
    S.par = reinterpret_cast<uint32_t*>(base + C.off_par);
    S.idom = reinterpret_cast<uint32_t*>(base + C.off_idom);
    S.rows = reinterpret_cast<int2*>(base + C.off_rows);
    S.edges = reinterpret_cast<uint2*>(base + C.off_edges);
    uint32_t* bm = kSmemBitmap ? dsm : reinterpret_cast<uint32_t*>(base + C.off_bm);
    if constexpr (kSmemBitmap) {
        for (uint32_t i = tid; i < C.bm_words; i += kCtaThreads) bm[i] = 0;
    }
    SampleCounters sc;
    unsigned long long examined = 0, live = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) sh.item = atomicAdd(&P.ctl->cursor[kTierCta], 1u);
        __syncthreads();
        const uint32_t j = sh.item;
        if (j >= P.theta) break;
        const int rc = run_sample_cta<kSmemBitmap, true>(P, C, bm, dsm, sh, S, j, tid, sc, examined, live);
        if (tid == 0 && rc != kSampleDone)  // only a cascade beyond the slot capacity can fail
            atomicOr(&P.ctl->error, rc == kSampleOverflow ? kErrCapacity : kErrInternal);
    }
    if (tid == 0 && sc.reached > 0) atomicAdd(sum, sc.reached);

    if (P.stats != nullptr) {
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
        }
    }
}

// The simulated spread of many blocker sets (the comparison algorithms of Sec. 5 -- BaselineGreedy,
// Exact -- score candidate sets this way): work item i is (set i / theta, sample i % theta); the
// sample runs with the set's k vertices blocked on top of excl, and its |R| (seeds included) is
// added to sums[set]. Every set sees the same samples (common random numbers).
template <bool kSmemBitmap>
__global__ void __launch_bounds__(cta_threads<kSmemBitmap>(), 1024 / cta_threads<kSmemBitmap>()) k_spread_sets(SampleParams P, CtaCfg C, const int32_t* sets,
                                                                uint32_t k, unsigned long long items,
                                                                unsigned long long* cursor,
                                                                unsigned long long* sums)
{
    constexpr uint32_t kCtaThreads = cta_threads<kSmemBitmap>();
    extern __shared__ __align__(16) uint32_t dsm[];
    __shared__ CtaShared<kCtaThreads> sh;
    __shared__ unsigned long long s_item;
    const uint32_t tid = threadIdx.x;
    uint8_t* base = C.scratch + static_cast<uint64_t>(blockIdx.x) * C.slot_bytes;
    Slot S;
    S.gid = reinterpret_cast<int32_t*>(base + C.off_gid);
    S.par = reinterpret_cast<uint32_t*>(base + C.off_par);
    S.idom = reinterpret_cast<uint32_t*>(base + C.off_idom);
    S.rows = reinterpret_cast<int2*>(base + C.off_rows);
    S.edges = reinterpret_cast<uint2*>(base + C.off_edges);
    uint32_t* bm = kSmemBitmap ? dsm : reinterpret_cast<uint32_t*>(base + C.off_bm);
    if constexpr (kSmemBitmap) {
        for (uint32_t i = tid; i < C.bm_words; i += kCtaThreads) bm[i] = 0;
    }
    SampleCounters sc;
    unsigned long long examined = 0, live = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(cursor, 1ull);
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= items) break;
        const uint32_t set = static_cast<uint32_t>(item / P.theta);
        const uint32_t j = static_cast<uint32_t>(item % P.theta);
        const unsigned long long before = sc.reached;
        const int rc = run_sample_cta<kSmemBitmap, true>(P, C, bm, dsm, sh, S, j, tid, sc, examined, live,
                                                         ExtraBlocked{sets + static_cast<uint64_t>(set) * k, k});
        if (tid == 0) {
            if (rc != kSampleDone) atomicOr(&P.ctl->error, rc == kSampleOverflow ? kErrCapacity : kErrInternal);
            else atomicAdd(sums + set, sc.reached - before);
        }
    }
}

}  // namespace

cudaError_t launch_spread_sets(const SampleParams& P, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                               uint8_t* scratch, const int32_t* sets, uint32_t k, unsigned long long items,
                               unsigned long long* cursor, unsigned long long* sums, cudaStream_t s)
{
    CtaCfg cfg = c;
    cfg.scratch = scratch;
    cfg.from_list = 0;
    const DeviceInfo dev = device_info();
    if (c.global_bitmap) {
        allow_max_dynamic_smem(k_spread_sets<false>, dev);
        k_spread_sets<false><<<blocks, cta_threads<false>(), smem, s>>>(P, cfg, sets, k, items, cursor, sums);
    } else {
        allow_max_dynamic_smem(k_spread_sets<true>, dev);
        k_spread_sets<true><<<blocks, cta_threads<true>(), smem, s>>>(P, cfg, sets, k, items, cursor, sums);
    }
    return cudaGetLastError();
}

cudaError_t launch_spread(const SampleParams& P, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                          uint8_t* scratch, unsigned long long* sum, cudaStream_t s)
{
    CtaCfg cfg = c;
    cfg.scratch = scratch;
    cfg.from_list = 0;
    const DeviceInfo dev = device_info();
    if (c.global_bitmap) {
        allow_max_dynamic_smem(k_spread_cta<false>, dev);
        k_spread_cta<false><<<blocks, cta_threads<false>(), smem, s>>>(P, cfg, sum);
    } else {
        allow_max_dynamic_smem(k_spread_cta<true>, dev);
        k_spread_cta<true><<<blocks, cta_threads<true>(), smem, s>>>(P, cfg, sum);
    }
    return cudaGetLastError();
}

}  // namespace imin
