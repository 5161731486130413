// batch.cu -- many independent queries (each with its own graph, seeds, budget, theta and key)
// advanced together, one greedy round per step: every step is one launch of the warp-per-sample
// kernel over the samples of all active queries (each finishes the samples whose cascade stays
// within the warp/block cutoff), one launch of the block-per-sample kernel per graph-size class
// for the rest, a launch of the whole-graph warp kernel for the rare samples the block tier could
// not hold, and one selection launch with a block per query. Work items are (query, chunk of
// samples) pairs handed out by an atomic cursor per launch, so uneven graphs and cascades are
// load-balanced across the whole GPU. Every query's Philox stream and round numbering are those
// of the single-query drivers, so each query's result is identical to running it alone.
#include <cstdlib>

#include "internal.h"
#include "sample_cta.cuh"
#include "select_dev.cuh"

namespace imin {

namespace {

using namespace cta;
using namespace sel;

constexpr uint32_t kWholeWarps = 8;  // warps per block of the batched whole-graph kernel
constexpr uint32_t kBatchWarps = 8;  // warps per block of the batched warp-tier kernel
constexpr uint64_t kWarpStageBytes = kStageCap * sizeof(uint2);

// Largest q with prefix[q] <= item (prefix[0] = 0, item < prefix[nq]).
__device__ __forceinline__ uint32_t find_query(const unsigned long long* prefix, uint32_t nq,
                                               unsigned long long item)
{
    uint32_t lo = 0, hi = nq;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Whether query q takes part in this step, and the blocker position the step fills. With
// c = step - start (the query's own round): AdvancedGreedy rounds 0 .. count-1 fill position c;
// GreedyReplace phase 1 (rounds 0 .. count-1) fills position c, phase 2 (rounds count ..
// 2*count-1) refills position 2*count-1-c until its stop flag is set.
__device__ __forceinline__ bool step_active(const BatchQuery& Q, const BatchStep& B, int32_t* pos,
                                            bool* phase2)
{
    if (B.step < Q.start) return false;
    const uint32_t cu = B.step - Q.start;
    if (cu > 0x7FFFFFFFu) return false;
    const int32_t c = static_cast<int32_t>(cu);
    *phase2 = false;
    if (!Q.gr) {
        *pos = c;
        return c < Q.count;
    }
    if (c < Q.count) {
        *pos = c;
        return true;
    }
    if (c >= 2 * Q.count) return false;
    if (*reinterpret_cast<const volatile int32_t*>(Q.flags) != 0) return false;
    *phase2 = true;
    *pos = 2 * Q.count - 1 - c;
    return true;
}

__device__ __forceinline__ SampleParams params_of(const BatchQuery& Q, uint32_t round)
{
    SampleParams P{};
    P.g = Q.g;
    P.seeds = Q.seeds;
    P.ns = Q.ns;
    P.excl = Q.excl;
    P.key_lo = Q.key_lo;
    P.key_hi = Q.key_hi;
    P.round = round;
    P.theta = Q.theta;
    P.delta = Q.delta;
    return P;
}

template <bool kSmemBitmap, int M>
__global__ void __launch_bounds__(cta_threads<kSmemBitmap>(), 1024 / cta_threads<kSmemBitmap>()) k_batch_cta(BatchStep B, CtaCfg C)
{
    constexpr uint32_t kCtaThreads = cta_threads<kSmemBitmap>();
    extern __shared__ __align__(16) uint32_t dsm[];
    __shared__ CtaShared<kCtaThreads> sh;
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_q;
    __shared__ int s_skip;
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

    const unsigned long long total = B.prefix[B.nq];
    SampleCounters sc;
    unsigned long long examined = 0, live = 0;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const unsigned long long item = atomicAdd(&B.ctl->cursor[B.cls], 1ull);
            s_item = item;
            if (item < total) {
                const uint32_t q = find_query(B.prefix, B.nq, item);
                int32_t pos;
                bool ph2;
                s_q = q;
                s_skip = !step_active(B.q[q], B, &pos, &ph2);
            }
        }
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= total) break;
        if (s_skip) continue;
        const uint32_t q = s_q;
        const BatchQuery& Q = B.q[q];
        const SampleParams P = params_of(Q, B.step - Q.start);
        const unsigned long long j0 = (item - B.prefix[q]) * B.chunk;
        const unsigned long long j1 = min(j0 + B.chunk, static_cast<unsigned long long>(Q.theta));
        for (unsigned long long j = j0; j < j1; ++j) {
            if (Q.done != nullptr && Q.done[j] != 0) continue;  // finished or handed over by the warp tier
            const int rc = run_sample_cta<kSmemBitmap, false, M>(P, C, bm, dsm, sh, S, static_cast<uint32_t>(j), tid,
                                                       sc, examined, live);
            if (tid == 0) {
                if (rc == kSampleOverflow) {
                    const uint32_t p = atomicAdd(&B.ctl->over_count, 1u);
                    if (p < B.over_cap) B.over[p] = make_uint2(q, static_cast<uint32_t>(j));
                    else atomicOr(&B.ctl->error, kErrCapacity);
                } else if (rc == kSampleError) {
                    atomicOr(&B.ctl->error, kErrInternal);
                }
            }
        }
    }
    // the samples of this class the warp tier handed over: resume each at the level it stopped
    if (B.handoff_stride != 0) {
        const uint32_t count =
            min(*reinterpret_cast<const volatile uint32_t*>(&B.ctl->handoff_count[B.cls]), B.handoff_cap);
        const uint8_t* list = reinterpret_cast<const uint8_t*>(B.over) + batch_handoff_offset(B.over_cap) +
                              static_cast<uint64_t>(B.cls) * B.handoff_cap * B.handoff_stride;
        for (;;) {
            __syncthreads();
            if (tid == 0) s_item = atomicAdd(&B.ctl->handoff_cursor[B.cls], 1u);
            __syncthreads();
            const unsigned long long h = s_item;
            if (h >= count) break;
            const uint8_t* hb = list + h * B.handoff_stride;
            const uint32_t* hdr = reinterpret_cast<const uint32_t*>(hb);
            const uint32_t j = hdr[0], q = hdr[8];
            const SampleParams P = params_of(B.q[q], B.step - B.q[q].start);
            uint32_t from[3];
            restore_handoff<kCtaThreads>(P, hb, S, bm, sh, tid, from);
            const int rc = run_sample_cta<kSmemBitmap, false, M>(P, C, bm, dsm, sh, S, j, tid, sc, examined, live,
                                                                 ExtraBlocked{nullptr, 0u}, from);
            if (tid == 0) {
                if (rc == kSampleOverflow) {
                    const uint32_t p = atomicAdd(&B.ctl->over_count, 1u);
                    if (p < B.over_cap) B.over[p] = make_uint2(q, j);
                    else atomicOr(&B.ctl->error, kErrCapacity);
                } else if (rc == kSampleError) {
                    atomicOr(&B.ctl->error, kErrInternal);
                }
            }
        }
    }
    if (B.stats != nullptr) {
        const uint32_t lane = tid & 31;
        unsigned long long ex = examined, lv = live;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            ex += __shfl_down_sync(kFull, ex, o);
            lv += __shfl_down_sync(kFull, lv, o);
        }
        unsigned long long* st = B.stats + kTierCta * kStPerTier;
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

// The warp tier of a step: one warp per sample, working set in shared memory with the
// warp/block cutoff as capacity, over the active queries that have a `done` array. Each
// sample's outcome is stored in done[j]: 1, counted here; 2, given up on and left as a hand-off
// snapshot in its size class's list (B.handoff_stride != 0, while the list has room), which the
// class's block launch resumes; 0, left to the block tier to run from the start.
template <int M>
__global__ void __launch_bounds__(kBatchWarps * 32, 4) k_batch_warp(BatchStep B, TierCfg T)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint8_t* mine = smem + wib * (kWarpStageBytes + T.warp_bytes);
    uint8_t* base = mine + kWarpStageBytes;
    const WarpLayout L = warp_layout(T.rcap, T.hcap, T.ecap, T.dcap, false);
    WarpSpace<false> w;
    w.stage = reinterpret_cast<uint2*>(mine);
    w.lvl = reinterpret_cast<uint32_t*>(base + L.lvl);
    w.hkey = reinterpret_cast<uint32_t*>(base + L.hkey);
    w.hval = reinterpret_cast<uint32_t*>(base + L.hval);
    w.gid = reinterpret_cast<int32_t*>(base + L.gid);
    w.idom = reinterpret_cast<uint32_t*>(base + L.idom);
    w.par = reinterpret_cast<uint32_t*>(base + L.par);
    w.hslot = reinterpret_cast<uint32_t*>(base + L.hslot);
    w.edges = reinterpret_cast<uint2*>(base + L.edges);
    w.rcap = T.rcap;
    w.hcap = T.hcap;
    w.hbits = T.hbits;
    w.ecap = T.ecap;
    w.dcap = T.dcap;
    for (uint32_t i = lane; i < w.hcap; i += 32) w.hkey[i] = kEmpty;
    __syncwarp();

    const unsigned long long total = B.prefix[B.nq];
    SampleCounters sc;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(&B.ctl->warp_cursor, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        const uint32_t q = find_query(B.prefix, B.nq, item);
        const BatchQuery& Q = B.q[q];
        int32_t pos;
        bool ph2;
        if (!step_active(Q, B, &pos, &ph2)) continue;
        const SampleParams P = params_of(Q, B.step - Q.start);
        const unsigned long long j0 = (item - B.prefix[q]) * B.chunk;
        const unsigned long long j1 = min(j0 + B.chunk, static_cast<unsigned long long>(Q.theta));
        for (unsigned long long j = j0; j < j1; ++j) {
            uint32_t at[4];
            const int rc = run_sample<false, true, M>(P, w, static_cast<uint32_t>(j), lane, sc, at);
            uint8_t outcome = rc == kSampleDone ? 1 : 0;
            if (rc == kSampleOverflow && B.handoff_stride != 0) {
                const uint32_t k = static_cast<uint32_t>(batch_class(Q.g.n));
                uint32_t pos = 0;
                if (lane == 0) pos = atomicAdd(&B.ctl->handoff_count[k], 1u);
                pos = __shfl_sync(kFull, pos, 0);
                if (pos < B.handoff_cap) {
                    const Handoff h = handoff_layout(T.rcap, T.dcap, T.ecap);
                    uint8_t* hb = reinterpret_cast<uint8_t*>(B.over) + batch_handoff_offset(B.over_cap) +
                                  (static_cast<uint64_t>(k) * B.handoff_cap + pos) * B.handoff_stride;
                    write_handoff(w, lane, hb, h, static_cast<uint32_t>(j), q, at);
                    outcome = 2;
                }
            }
            if (lane == 0) {
                Q.done[j] = outcome;
                if (rc == kSampleError) atomicOr(&B.ctl->error, kErrInternal);
            }
        }
    }
    if (B.stats != nullptr) {
        unsigned long long ex = sc.examined, lv = sc.live;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            ex += __shfl_down_sync(kFull, ex, o);
            lv += __shfl_down_sync(kFull, lv, o);
        }
        if (lane == 0 && sc.done > 0) {
            unsigned long long* st = B.stats;  // tier 0 slots
            atomicAdd(st + kStSamples, sc.done);
            atomicAdd(st + kStReached, sc.reached);
            atomicAdd(st + kStExamined, ex);
            atomicAdd(st + kStLive, lv);
            atomicAdd(st + kStNontree, sc.nontree);
            atomicAdd(st + kStPasses, sc.passes);
        }
    }
}

// The samples the block tier handed over, one warp each, with whole-graph capacity.
__global__ void __launch_bounds__(kWholeWarps * 32) k_batch_whole(BatchStep B, TierCfg T)
{
    __shared__ __align__(16) uint2 stage[kWholeWarps][kStageCap];
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * kWholeWarps + wib;
    uint8_t* base = T.gscratch + gw * T.warp_bytes;
    const WarpLayout L = warp_layout(T.rcap, T.hcap, T.ecap, T.dcap, true);
    WarpSpace<true> w;
    w.stage = stage[wib];
    w.lvl = reinterpret_cast<uint32_t*>(base + L.lvl);
    w.hkey = reinterpret_cast<uint32_t*>(base + L.hkey);
    w.hval = reinterpret_cast<uint32_t*>(base + L.hval);
    w.gid = reinterpret_cast<int32_t*>(base + L.gid);
    w.idom = reinterpret_cast<uint32_t*>(base + L.idom);
    w.par = reinterpret_cast<uint32_t*>(base + L.par);
    w.hslot = reinterpret_cast<uint32_t*>(base + L.hslot);
    w.edges = reinterpret_cast<uint2*>(base + L.edges);
    w.rcap = T.rcap;
    w.hcap = T.hcap;
    w.hbits = T.hbits;
    w.ecap = T.ecap;
    w.dcap = T.dcap;

    const uint32_t count = min(*reinterpret_cast<const volatile uint32_t*>(&B.ctl->over_count), B.over_cap);
    SampleCounters sc;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&B.ctl->over_cursor, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= count) break;
        const uint2 qj = B.over[item];
        const SampleParams P = params_of(B.q[qj.x], B.step - B.q[qj.x].start);
        const int rc = run_sample<true, false>(P, w, qj.y, lane, sc);
        if (lane == 0 && rc != kSampleDone)
            atomicOr(&B.ctl->error, rc == kSampleOverflow ? kErrCapacity : kErrInternal);
    }
}

// GreedyReplace phase 2, "B <- B \ {u}" for every query in phase 2 at this step.
__global__ void k_batch_unblock(BatchStep B)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B.nq) return;
    const BatchQuery& Q = B.q[q];
    int32_t pos;
    bool ph2;
    if (!step_active(Q, B, &pos, &ph2) || !ph2) return;
    const int32_t u = Q.blockers[pos];
    Q.flags[1] = u;
    atomicAnd(Q.excl + (u >> 5), ~(1u << (u & 31)));
}

// One block per query: the strict-max selection of the step (phase-1 candidates are CB).
__global__ void __launch_bounds__(kSelThreads) k_batch_select(BatchStep B)
{
    const BatchQuery& Q = B.q[blockIdx.x];
    int32_t pos;
    bool ph2;
    if (!step_active(Q, B, &pos, &ph2)) return;
    const bool use_cb = Q.gr && !ph2;
    unsigned long long bd = 0;
    int32_t bi = kNone;
    for (int32_t v = threadIdx.x; v < Q.g.n; v += blockDim.x) {
        const unsigned long long d = Q.delta[v];
        if (d != 0) Q.delta[v] = 0;
        const uint32_t bit = 1u << (v & 31);
        const bool cand = use_cb ? (Q.cb[v >> 5] & bit) != 0 : (Q.excl[v >> 5] & bit) == 0;
        if (cand && better(d, v, bd, bi)) {
            bd = d;
            bi = v;
        }
    }
    block_best<kSelThreads>(bd, bi);
    if (threadIdx.x == 0 && bi != kNone) {
        Q.blockers[pos] = bi;
        Q.excl[bi >> 5] |= 1u << (bi & 31);
        if (use_cb) Q.cb[bi >> 5] &= ~(1u << (bi & 31));
        if (ph2 && Q.flags[1] == bi) Q.flags[0] = 1;
    }
}

}  // namespace

bool plan_batch_cta(const DeviceInfo& dev, int32_t max_n, int32_t max_m, CtaCfg* c, uint32_t* blocks,
                    uint64_t* smem, uint64_t* scratch_bytes)
{
    uint32_t b0 = 0;
    uint64_t s0 = 0;
    if (!plan_cta_tier(dev, max_n, max_m, c, &b0, smem, &s0)) return false;
    int occ = 0;
    if (c->global_bitmap) {
        if (allow_max_dynamic_smem(k_batch_cta<false, kModelIC>, dev) != cudaSuccess ||
            allow_max_dynamic_smem(k_batch_cta<false, kModelAny>, dev) != cudaSuccess)
            return false;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_cta<false, kModelIC>, cta_threads<false>(), *smem);
    } else {
        if (allow_max_dynamic_smem(k_batch_cta<true, kModelIC>, dev) != cudaSuccess ||
            allow_max_dynamic_smem(k_batch_cta<true, kModelAny>, dev) != cudaSuccess)
            return false;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_cta<true, kModelIC>, cta_threads<true>(), *smem);
    }
    if (occ <= 0) return false;
    *blocks = static_cast<uint32_t>(occ) * dev.sms;
    *scratch_bytes = c->slot_bytes * *blocks;
    return true;
}

bool plan_batch_warp(const DeviceInfo& dev, uint32_t max_ns, uint32_t cutoff, TierCfg* c, uint32_t* blocks,
                     uint64_t* smem)
{
    if (cutoff == 0 || max_ns == 0 || max_ns > kBatchWarpMaxSeeds) return false;
    tier0_cfg(max_ns, cutoff, c);
    *smem = kBatchWarps * (kWarpStageBytes + c->warp_bytes);
    if (*smem > dev.smem_optin) return false;
    if (allow_max_dynamic_smem(k_batch_warp<kModelIC>, dev) != cudaSuccess ||
        allow_max_dynamic_smem(k_batch_warp<kModelAny>, dev) != cudaSuccess)
        return false;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_warp<kModelIC>, kBatchWarps * 32, *smem);
    if (occ <= 0) return false;
    *blocks = static_cast<uint32_t>(occ) * dev.sms;
    return true;
}

cudaError_t launch_batch_warp(const BatchStep& B, const TierCfg& c, uint32_t blocks, uint64_t smem,
                              cudaStream_t s)
{
    if (B.all_ic) k_batch_warp<kModelIC><<<blocks, kBatchWarps * 32, smem, s>>>(B, c);
    else k_batch_warp<kModelAny><<<blocks, kBatchWarps * 32, smem, s>>>(B, c);
    return cudaGetLastError();
}

cudaError_t launch_batch_unblock(const BatchStep& B, cudaStream_t s)
{
    k_batch_unblock<<<(B.nq + 127) / 128, 128, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_batch_cta(const BatchStep& B, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                             uint8_t* scratch, cudaStream_t s)
{
    CtaCfg cfg = c;
    cfg.scratch = scratch;
    if (c.global_bitmap) {
        if (B.all_ic) k_batch_cta<false, kModelIC><<<blocks, cta_threads<false>(), smem, s>>>(B, cfg);
        else k_batch_cta<false, kModelAny><<<blocks, cta_threads<false>(), smem, s>>>(B, cfg);
    } else {
        if (B.all_ic) k_batch_cta<true, kModelIC><<<blocks, cta_threads<true>(), smem, s>>>(B, cfg);
        else k_batch_cta<true, kModelAny><<<blocks, cta_threads<true>(), smem, s>>>(B, cfg);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_whole(const BatchStep& B, const TierCfg& whole, uint32_t blocks,
                               uint8_t* scratch, cudaStream_t s)
{
    TierCfg t = whole;
    t.gscratch = scratch;
    k_batch_whole<<<blocks, kWholeWarps * 32, 0, s>>>(B, t);
    return cudaGetLastError();
}

cudaError_t launch_batch_select(const BatchStep& B, cudaStream_t s)
{
    k_batch_select<<<B.nq, kSelThreads, 0, s>>>(B);
    return cudaGetLastError();
}

uint32_t whole_warps_per_block() { return kWholeWarps; }

}  // namespace imin
