// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "imin_dev.cuh"

namespace imin {

struct DeviceInfo {
    int device = 0;
    int sms = 0;
    uint64_t smem_optin = 0;
};

DeviceInfo device_info();

// Let `func` launch with up to the device's opt-in shared memory (minus its static shared
// memory). Raising the limit once means that plans made for different graph sizes never lower
// it under a launch that needs more; occupancy still follows each launch's actual size.
template <typename F>
cudaError_t allow_max_dynamic_smem(F func, const DeviceInfo& dev)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, func);
    if (e != cudaSuccess) return e;
    const int avail = static_cast<int>(dev.smem_optin) - static_cast<int>(a.sharedSizeBytes);
    return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, avail > 0 ? avail : 0);
}

// Record `msg` as the calling thread's last error (fixed buffer, no allocation); returns code.
int fail_msg(int code, const char* msg);

}  // namespace imin

// A graph resident in device memory (the opaque handle of include/imin.h).
struct imin_graph {
    int32_t n = 0;
    int32_t m = 0;
    int device = 0;
    imin::DeviceInfo dev;
    int32_t* row_ptr = nullptr;  // [n+1]
    int32_t* col = nullptr;      // [m] padded to a multiple of 4 (+4)
    uint4* thr4 = nullptr;       // thresholds (LT: interval widths - 1), same padding
    uint4* lo4 = nullptr;        // LT model: start of each in-edge's interval, same padding
    int32_t model = 0;           // 0: independent cascade (Def. 4); 1: linear threshold (Sec. 4.5)
    // sampled hash of the CSR: handles of the same graph share tuning results
    uint64_t fingerprint = 0;
    // warp/block cutoff picked by the autotuner, per seed-set size class (ceil(log2 |S|));
    // -1: not tuned yet
    mutable std::mutex tune_mu;
    mutable int32_t cutoff[32] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
                                  -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
};

namespace imin {

inline DevGraph dev_graph(const imin_graph* g)
{
    return DevGraph{g->n, g->m, g->row_ptr, g->col, g->thr4, g->lo4};
}

// Launch shape and capacities of the sample tiers for one graph / seed-set size.
struct TierPlan {
    TierCfg cfg[kTiers];
    uint32_t warps_per_block[kTiers];
    uint32_t blocks[kTiers];
    uint64_t smem_bytes[kTiers];  // dynamic shared memory per block
    uint64_t scratch_bytes[kTiers];
    bool use_cta = false;         // tier 3 replaces tiers 0 and 1
    CtaCfg cta{};
};

// Tier capacities for a graph with n vertices and m edges and a seed set of size ns.
// Capacities and per-warp shared-memory bytes of the warp tier 0 (working set in shared memory)
// for seed sets of up to ns vertices and r0 non-seed vertices.
void tier0_cfg(uint32_t ns, uint32_t r0, TierCfg* c);
// cutoff: non-seed capacity of the warp tier 0 run in front of the block tier (0: none).
TierPlan plan_tiers(const DeviceInfo& dev, int32_t n, int32_t m, uint32_t ns, uint32_t cutoff);

// Enqueue tier `tier` of one Alg. 2 call (tier 0 takes samples [0, theta); tiers 1 and 2 take
// the samples the previous tier could not hold). P.ctl must be zeroed and P.delta cleared
// before tier 0; `scratch` must point at plan.scratch_bytes[tier] bytes whose hash words are
// all 0xFF (tiers 1-2). Returns cudaSuccess without launching when the tier has no blocks.
// *launched is set to whether a kernel was enqueued.
cudaError_t launch_sample_tier(int tier, const SampleParams& P, const TierPlan& plan,
                               uint8_t* scratch, cudaStream_t s, bool* launched);

// Block-per-sample tier: layout, grid and shared memory. Graphs with n <= kCtaMaxVertices keep
// the visited bitmap in shared memory; larger ones keep it in each block's global slot.
bool plan_cta_tier(const DeviceInfo& dev, int32_t n, int32_t m, CtaCfg* c, uint32_t* blocks, uint64_t* smem,
                   uint64_t* scratch_bytes);
cudaError_t launch_cta_tier(const SampleParams& P, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                            uint8_t* scratch, cudaStream_t s);
// Zero the per-slot visited bitmaps of a large-graph block tier (no-op for the shared variant).
cudaError_t prepare_cta_scratch(const CtaCfg& c, uint32_t blocks, uint8_t* scratch, cudaStream_t s);

// Monte-Carlo spread (spread.cu): adds sum over samples [0, P.theta) of |R| (seeds included) to
// *sum, with the block tier's layout `c` and `blocks` slots of `scratch`.
cudaError_t launch_spread(const SampleParams& P, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                          uint8_t* scratch, unsigned long long* sum, cudaStream_t s);

// Spread of many blocker sets (spread.cu): for item i < items, adds |R| of sample i % P.theta with
// set i / P.theta (k vertices of `sets`) blocked on top of P.excl into sums[i / P.theta].
// *cursor must start at 0.
cudaError_t launch_spread_sets(const SampleParams& P, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                               uint8_t* scratch, const int32_t* sets, uint32_t k, unsigned long long items,
                               unsigned long long* cursor, unsigned long long* sums, cudaStream_t s);

// Batched multi-query steps (batch.cu).
bool plan_batch_cta(const DeviceInfo& dev, int32_t max_n, int32_t max_m, CtaCfg* c, uint32_t* blocks,
                    uint64_t* smem, uint64_t* scratch_bytes);
cudaError_t launch_batch_unblock(const BatchStep& B, cudaStream_t s);
cudaError_t launch_batch_cta(const BatchStep& B, const CtaCfg& c, uint32_t blocks, uint64_t smem,
                             uint8_t* scratch, cudaStream_t s);
cudaError_t launch_batch_whole(const BatchStep& B, const TierCfg& whole, uint32_t blocks,
                               uint8_t* scratch, cudaStream_t s);
cudaError_t launch_batch_select(const BatchStep& B, cudaStream_t s);
uint32_t whole_warps_per_block();
// The warp tier of a batch step (queries with at most kBatchWarpMaxSeeds seeds): capacities for
// seed sets of up to max_ns vertices and `cutoff` non-seed vertices; false if it cannot run.
constexpr uint32_t kBatchWarpMaxSeeds = 256;
constexpr uint32_t kDefaultCutoff = 96;
bool plan_batch_warp(const DeviceInfo& dev, uint32_t max_ns, uint32_t cutoff, TierCfg* c, uint32_t* blocks,
                     uint64_t* smem);
cudaError_t launch_batch_warp(const BatchStep& B, const TierCfg& c, uint32_t blocks, uint64_t smem,
                              cudaStream_t s);
// The warp/block cutoff of one query (api.cu): IMIN_TIER0_VERTICES when set; kDefaultCutoff with
// IMIN_AUTOTUNE=0 or on a capturing stream; otherwise the autotuner's value for the graph and the
// seed-set size class, tuned on `s` on first use and cached.
int tuned_cutoff(const imin_graph* g, const std::vector<int32_t>& seeds, uint64_t key, uint32_t theta_hint,
                 cudaStream_t s, uint32_t* out);

// Selection (Alg. 3/4 argmax) -----------------------------------------------------------------
struct SelectParams {
    unsigned long long* delta;     // [n]; cleared as it is read
    int32_t n;
    uint32_t* excl;                // n-bit mask; the winner is added
    uint32_t* cand;                // optional n-bit candidate mask (GreedyReplace phase 1);
                                   // when null the candidates are the vertices not in excl.
                                   // The winner is removed from it.
    int32_t* blockers;             // the winner is written to blockers[pos]
    int32_t pos;
    int32_t* done;                 // optional stop flag
    const int32_t* cur;            // optional: vertex unblocked for this round; winner == *cur
                                   // sets *done
    unsigned long long* part_d;    // [blocks] scratch
    int32_t* part_id;              // [blocks] scratch
    uint32_t* ticket;              // zero-initialised counter
};

int select_blocks();
cudaError_t launch_select(const SelectParams& p, cudaStream_t s);
cudaError_t launch_unblock(uint32_t* excl, const int32_t* blockers, int32_t pos, const int32_t* done,
                           int32_t* cur, cudaStream_t s);
cudaError_t launch_build_excl(uint32_t* excl, const int32_t* ids, int32_t count, cudaStream_t s);
cudaError_t launch_build_cb(const DevGraph& g, const int32_t* seeds, int32_t ns,
                            const uint32_t* excl, uint32_t* cb, uint32_t* cb_count,
                            cudaStream_t s);

}  // namespace imin
