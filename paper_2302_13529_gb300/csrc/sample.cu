// sample.cu -- the warp-per-sample tiers of Alg. 2 (DecreaseESComputation) and the planning of
// all tiers.
//
// Tier 0 keeps each warp's working set in shared memory and takes every sample first. In front
// of the block-per-sample tier 3 its capacity is the warp/block cutoff (a few dozen to a few
// hundred reached vertices, picked by the autotuner in api.cu) and a sample that outgrows it is
// re-run by tier 3; without tier 3, it holds 256 vertices and hands over to tier 1, a per-warp
// slot of global scratch with capacity for 16K reached vertices. Tier 2 holds any cascade
// (|R| <= n) and is launched with few warps, because its slots scale with n. Work is handed out
// by an atomic cursor per tier, so warps that draw small cascades keep pulling new samples.
#include <algorithm>
#include <cstdlib>

#include "internal.h"

namespace imin {

namespace {

constexpr uint32_t kWarpsPerBlock = 8;
constexpr uint32_t kStageBytes = kStageCap * sizeof(uint2);

uint32_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return static_cast<uint32_t>(p);
}

uint32_t log2u(uint32_t p)
{
    uint32_t b = 0;
    while ((1u << b) < p) ++b;
    return b;
}

uint32_t env_u32(const char* name, uint32_t dflt)
{
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    return static_cast<uint32_t>(std::strtoul(v, nullptr, 10));
}

template <int kTier, int M>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_sample_tier(SampleParams P, TierCfg T)
{
    constexpr bool G = kTier > 0;
    constexpr bool kClearAll = kTier == 0;
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wib = threadIdx.x >> 5;
    const uint64_t gw = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;

    if (P.done != nullptr && *reinterpret_cast<const volatile int32_t*>(P.done) != 0) return;

    const uint64_t smem_per_warp = kStageBytes + (G ? 0 : T.warp_bytes);
    uint8_t* my_smem = smem + wib * smem_per_warp;
    uint8_t* base = G ? T.gscratch + gw * T.warp_bytes : my_smem + kStageBytes;
    const WarpLayout L = warp_layout(T.rcap, T.hcap, T.ecap, T.dcap, !kClearAll);

    WarpSpace<G> w;
    w.stage = reinterpret_cast<uint2*>(my_smem);
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

    if constexpr (!G) {
        for (uint32_t i = lane; i < w.hcap; i += 32) w.hkey[i] = kEmpty;
        __syncwarp();
    }

    SampleCounters sc;
    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&P.ctl->cursor[kTier], 1u);
        item = __shfl_sync(kFull, item, 0);
        const bool from_range = kTier == 0 || T.from_range != 0;
        const uint32_t total =
            from_range ? P.theta : *reinterpret_cast<const volatile uint32_t*>(&P.ctl->count[kTier]);
        if (item >= total) break;
        const uint32_t j = from_range ? item : P.lists[kTier * P.theta + item];
        uint32_t at[4];
        const int rc = run_sample<G, kClearAll, M>(P, w, j, lane, sc, at);
        if (rc == kSampleOverflow) {
            uint32_t pos = 0;
            if (lane == 0) {
                if (kTier < kTierWhole) {
                    const uint32_t nt = T.next_tier;
                    pos = atomicAdd(&P.ctl->count[nt], 1u);
                    P.lists[nt * P.theta + pos] = j;
                } else {
                    atomicOr(&P.ctl->error, kErrCapacity);
                }
            }
            if constexpr (kTier == 0) {
                // tier 0 in front of the block tier: leave the sample's state at the start of
                // the level it could not hold, for the block tier to resume from
                if (T.gscratch != nullptr) {
                    pos = __shfl_sync(kFull, pos, 0);
                    const Handoff h = handoff_layout(T.rcap, T.dcap, T.ecap);
                    write_handoff(w, lane, T.gscratch + static_cast<uint64_t>(pos) * h.stride, h, j, 0u, at);
                }
            }
        } else if (rc == kSampleError) {
            if (lane == 0) atomicOr(&P.ctl->error, kErrInternal);
        }
    }

    if (P.stats != nullptr) {
        unsigned long long ex = sc.examined, lv = sc.live;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            ex += __shfl_down_sync(kFull, ex, o);
            lv += __shfl_down_sync(kFull, lv, o);
        }
        if (lane == 0 && sc.done > 0) {
            unsigned long long* st = P.stats + kTier * kStPerTier;
            atomicAdd(st + kStSamples, sc.done);
            atomicAdd(st + kStReached, sc.reached);
            atomicAdd(st + kStExamined, ex);
            atomicAdd(st + kStLive, lv);
            atomicAdd(st + kStNontree, sc.nontree);
            atomicAdd(st + kStPasses, sc.passes);
        }
    }
}

}  // namespace

DeviceInfo device_info()
{
    DeviceInfo d;
    cudaGetDevice(&d.device);
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, d.device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d.device);
    d.smem_optin = static_cast<uint64_t>(optin);
    return d;
}

void tier0_cfg(uint32_t ns, uint32_t r0, TierCfg* c)
{
    c->rcap = 1 + ns + r0;
    c->hcap = next_pow2(2ull * std::max<uint32_t>(r0, 32));  // load <= 1/2 + 32 in flight
    c->hbits = log2u(c->hcap);
    c->ecap = std::max<uint32_t>(r0 / 4, 32);  // a cascade with more goes to the next tier
    c->dcap = 32;
    c->warp_bytes = warp_layout(c->rcap, c->hcap, c->ecap, c->dcap, false).total;
    c->gscratch = nullptr;
    c->from_range = 1;
    c->next_tier = kTierCta;
}

TierPlan plan_tiers(const DeviceInfo& dev, int32_t n, int32_t m, uint32_t ns, uint32_t cutoff)
{
    TierPlan p{};
    // non-seed capacity of tier 0: in front of the block tier it is the warp/block cutoff (0: no
    // tier 0); behind the warp tiers alone it is 256
    uint32_t r0 = env_u32("IMIN_TIER0_VERTICES", 256);
    const uint32_t r1 = env_u32("IMIN_TIER1_VERTICES", 16384);  // non-seed capacity, tier 1
    const uint32_t b1 = env_u32("IMIN_TIER1_BLOCKS_PER_SM", 2);
    const bool allow_cta = env_u32("IMIN_DISABLE_CTA_TIER", 0) == 0;
    uint64_t t2_budget = static_cast<uint64_t>(env_u32("IMIN_TIER2_MIB", 4096)) << 20;

    // tier 3: block per sample with a shared-memory visited bitmap, whenever n allows
    if (allow_cta && plan_cta_tier(dev, n, m, &p.cta, &p.blocks[kTierCta], &p.smem_bytes[kTierCta],
                                   &p.scratch_bytes[kTierCta])) {
        p.use_cta = true;
        p.warps_per_block[kTierCta] = p.cta.global_bitmap ? 8u : 4u;  // 256- or 128-thread blocks
        // tier 2 only catches the rare samples with too many non-tree edges or levels
        t2_budget = std::min<uint64_t>(t2_budget, 1ull << 30);
        r0 = cutoff;
    }

    // tier 0: shared memory
    if (r0 > 0) {
        TierCfg& c = p.cfg[0];
        tier0_cfg(ns, r0, &c);
        p.warps_per_block[0] = kWarpsPerBlock;
        p.smem_bytes[0] = kWarpsPerBlock * (kStageBytes + c.warp_bytes);
        p.scratch_bytes[0] = 0;
        int occ = 0;
        if (p.smem_bytes[0] <= dev.smem_optin) {
            allow_max_dynamic_smem(k_sample_tier<0, kModelLT>, dev);
            allow_max_dynamic_smem(k_sample_tier<0, kModelIC>, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sample_tier<0, kModelIC>,
                                                          kWarpsPerBlock * 32, p.smem_bytes[0]);
        }
        p.blocks[0] = static_cast<uint32_t>(std::max(occ, 0)) * dev.sms;
        c.next_tier = p.use_cta ? static_cast<uint32_t>(kTierCta) : 1u;
        p.cta.from_list = p.use_cta && p.blocks[0] > 0 ? 1u : 0u;
    }
    // tier 1: per-warp global slot for up to r1 non-seed vertices
    {
        TierCfg& c = p.cfg[1];
        const uint32_t r = std::min<uint64_t>(r1, static_cast<uint64_t>(n));
        c.rcap = 1 + ns + r;
        c.hcap = next_pow2(2ull * std::max<uint32_t>(r, 32));
        c.hbits = log2u(c.hcap);
        c.ecap = std::max<uint32_t>(r / 4, 256);
        c.next_tier = 2;
        c.dcap = std::min<uint32_t>(c.rcap, 1024);
        c.warp_bytes = (warp_layout(c.rcap, c.hcap, c.ecap, c.dcap, true).total + 255) & ~255ull;
        p.warps_per_block[1] = kWarpsPerBlock;
        p.blocks[1] = p.use_cta ? 0u : b1 * dev.sms;
        p.smem_bytes[1] = kWarpsPerBlock * kStageBytes;
        p.scratch_bytes[1] = c.warp_bytes * p.blocks[1] * kWarpsPerBlock;
    }
    // tier 2: per-warp global slot for any cascade (|R| <= n)
    {
        TierCfg& c = p.cfg[2];
        c.rcap = 1 + static_cast<uint32_t>(n);
        c.hcap = next_pow2(2ull * std::max<uint64_t>(static_cast<uint64_t>(n), 32));
        c.hbits = log2u(c.hcap);
        c.ecap = static_cast<uint32_t>(std::max<int64_t>(std::min<int64_t>(m, 4ll * n), 1024));
        c.dcap = c.rcap;
        c.warp_bytes = (warp_layout(c.rcap, c.hcap, c.ecap, c.dcap, true).total + 255) & ~255ull;
        uint64_t warps = std::max<uint64_t>(1, t2_budget / c.warp_bytes);
        warps = std::min<uint64_t>(warps, static_cast<uint64_t>(dev.sms) * kWarpsPerBlock);
        const uint32_t blocks = static_cast<uint32_t>((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
        p.warps_per_block[2] = kWarpsPerBlock;
        p.blocks[2] = blocks;
        p.smem_bytes[2] = kWarpsPerBlock * kStageBytes;
        p.scratch_bytes[2] = c.warp_bytes * blocks * kWarpsPerBlock;
    }
    return p;
}

cudaError_t launch_sample_tier(int tier, const SampleParams& P, const TierPlan& plan,
                               uint8_t* scratch, cudaStream_t s, bool* launched)
{
    *launched = false;
    if (plan.blocks[tier] == 0) return cudaSuccess;
    if (tier == kTierCta) {
        *launched = true;
        return launch_cta_tier(P, plan.cta, plan.blocks[kTierCta], plan.smem_bytes[kTierCta], scratch, s);
    }
    TierCfg c = plan.cfg[tier];
    c.gscratch = scratch;
    // the first tier that runs takes the whole sample range; tier 0 is skipped only when the
    // seed set does not fit its shared-memory working set
    c.from_range = tier == 0 || (tier == 1 && plan.blocks[0] == 0 && !plan.use_cta);
    const dim3 grid(plan.blocks[tier]), block(kWarpsPerBlock * 32);
    const size_t sm = plan.smem_bytes[tier];
    if (P.g.lo4 == nullptr) {
        if (tier == 0) k_sample_tier<0, kModelIC><<<grid, block, sm, s>>>(P, c);
        else if (tier == 1) k_sample_tier<1, kModelIC><<<grid, block, sm, s>>>(P, c);
        else k_sample_tier<2, kModelIC><<<grid, block, sm, s>>>(P, c);
    } else {
        if (tier == 0) k_sample_tier<0, kModelLT><<<grid, block, sm, s>>>(P, c);
        else if (tier == 1) k_sample_tier<1, kModelLT><<<grid, block, sm, s>>>(P, c);
        else k_sample_tier<2, kModelLT><<<grid, block, sm, s>>>(P, c);
    }
    *launched = true;
    return cudaGetLastError();
}

}  // namespace imin
