// noalloc.cu -- imin_estimate_decrease_noalloc: one Alg. 2 call that allocates no memory.
//
// Who needs it: callers that must not allocate device memory when they call in -- code whose
// device memory is owned by another allocator with a fixed budget (a framework's caching
// allocator, a serving process that sizes everything at start-up and must not grow later), and
// latency-critical paths that cannot afford cudaMalloc/cudaFree, which may synchronize the whole
// device. The call itself is synchronous: it reads a validation flag back from the device before
// its kernel runs and the kernel's status after it, so it returns only when the counters are
// final, and it cannot be recorded into a CUDA graph by stream capture.
//
// What it does: exactly what imin_estimate_decrease computes, with the block-per-sample tier
// (sample_cta.cu), but every byte of working memory it needs besides the caller's inputs and
// output comes from one file-scope device array of kNoAllocBytes (64 MiB). Every GPU that loads
// the library holds that array until the process exits. Its limits follow from its size:
// graphs with at most kNoAllocMaxVertices vertices and at most kNoAllocMaxTheta samples per call;
// bigger requests are rejected with IMIN_ERR_INVALID. A sampled cascade that would need the
// whole-graph fallback tier (more non-tree live edges or BFS levels than the block tier holds)
// makes the call fail with IMIN_ERR_CAPACITY instead of running that tier; out_delta then holds
// partial counters and must not be used.
//
// The array is shared by every call on a device and keeps the last call's contents; each call
// clears the parts that must start at zero. Calls that overlap on the GPU (different streams or
// threads without ordering between them) race on it.
//
// Set-up: the first call on each device resolves the array's device address with
// cudaGetSymbolAddress (in host code the array's name is only a host-side stand-in, never a
// device address). The block tier's launch plan (slot layout, grid, shared memory) is computed
// once per device and graph size (n, m) and kept in a fixed table, so later calls of the same
// size make no attribute or occupancy queries; the plan's test hooks (IMIN_CTA_EDGE_CAP) are read
// only when a plan is made.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "imin.h"
#include "internal.h"

namespace imin {

namespace {

constexpr int32_t kNoAllocMaxVertices = 1 << 16;
constexpr uint32_t kNoAllocMaxTheta = 1u << 17;
constexpr uint64_t kNoAllocBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Launch plans of the block tier, per device and graph size, in a fixed table (no heap use).
struct PlanEntry {
    int device;
    int32_t n, m;
    CtaCfg cfg;
    uint32_t blocks;
    uint64_t smem;
};
constexpr int kPlanSlots = 16;
PlanEntry g_plans[kPlanSlots];
int g_plan_count = 0, g_plan_next = 0;

// The block tier's plan for (device, n, m), made on first use.
bool cta_plan(const imin_graph* g, CtaCfg* cfg, uint32_t* blocks, uint64_t* smem)
{
    std::lock_guard<std::mutex> lk(g_setup_mu);
    for (int i = 0; i < g_plan_count; ++i) {
        const PlanEntry& e = g_plans[i];
        if (e.device == g->device && e.n == g->n && e.m == g->m) {
            *cfg = e.cfg;
            *blocks = e.blocks;
            *smem = e.smem;
            return true;
        }
    }
    uint64_t slot_total = 0;
    if (!plan_cta_tier(g->dev, g->n, g->m, cfg, blocks, smem, &slot_total)) return false;
    PlanEntry& e = g_plans[g_plan_next];
    e = PlanEntry{g->device, g->n, g->m, *cfg, *blocks, *smem};
    g_plan_next = (g_plan_next + 1) % kPlanSlots;
    if (g_plan_count < kPlanSlots) ++g_plan_count;
    return true;
}

// Device address of the static array on `device` (resolved once per device).
int scratch_address(int device, uint8_t** out)
{
    if (device < 0 || device >= kMaxDevices) return fail_msg(IMIN_ERR_CUDA, "device index out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (g_scratch_ptr[device] == nullptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            char msg[160];
            std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the static scratch failed: %s",
                          cudaGetErrorString(e));
            return fail_msg(IMIN_ERR_CUDA, msg);
        }
        g_scratch_ptr[device] = p;
    }
    *out = static_cast<uint8_t*>(g_scratch_ptr[device]);
    return IMIN_OK;
}

// Marks every id in the seed/blocked bitmask; flags ids out of range (bit 0) and ids that were
// already marked -- duplicates, or a blocked vertex that is a seed (bit 1).
__global__ void k_mark_ids(const int32_t* ids, int32_t count, int32_t n, uint32_t* excl, uint32_t* bad)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int32_t v = ids[i];
        if (v < 0 || v >= n) {
            atomicOr(bad, 1u);
            continue;
        }
        const uint32_t bit = 1u << (v & 31);
        if (atomicOr(excl + (v >> 5), bit) & bit) atomicOr(bad, 2u);
    }
}

uint64_t up256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// 1: device (or managed) memory of `device`; 0: host memory; -1: device memory of another GPU.
int device_pointer(const void* p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return 0;
    return a.device == device ? 1 : -1;
}

int cuda_fail(cudaError_t e, const char* what)
{
    cudaGetLastError();
    char msg[200];
    std::snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    return fail_msg(IMIN_ERR_CUDA, msg);
}

#define NA_CUDA(call)                                 \
    do {                                              \
        const cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

}  // namespace

}  // namespace imin

using namespace imin;

extern "C" int imin_estimate_decrease_noalloc(const imin_graph* g, const int32_t* seeds,
                                              int32_t n_seeds, const int32_t* blocked,
                                              int32_t n_blocked, uint32_t theta, uint64_t key,
                                              uint32_t round, uint64_t* out_delta, void* stream)
{
    fail_msg(IMIN_OK, "");
    if (g == nullptr) return fail_msg(IMIN_ERR_INVALID, "graph handle is NULL");
    if (out_delta == nullptr) return fail_msg(IMIN_ERR_INVALID, "out_delta is NULL");
    if (seeds == nullptr) return fail_msg(IMIN_ERR_INVALID, "seeds is NULL");
    if (n_seeds < 1 || n_seeds > g->n) return fail_msg(IMIN_ERR_INVALID, "n_seeds must be in [1, n]");
    if (n_blocked < 0 || (n_blocked > 0 && blocked == nullptr))
        return fail_msg(IMIN_ERR_INVALID, "n_blocked must be >= 0 and blocked non-NULL when > 0");
    if (n_seeds + static_cast<int64_t>(n_blocked) > g->n)
        return fail_msg(IMIN_ERR_INVALID, "more seeds and blocked vertices than vertices");
    if (theta < 1) return fail_msg(IMIN_ERR_INVALID, "theta must be >= 1");
    if (g->n > kNoAllocMaxVertices) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "imin_estimate_decrease_noalloc: n = %d exceeds its static limit of %d vertices",
                      g->n, kNoAllocMaxVertices);
        return fail_msg(IMIN_ERR_INVALID, msg);
    }
    if (theta > kNoAllocMaxTheta) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "imin_estimate_decrease_noalloc: theta = %u exceeds its static limit of %u",
                      theta, kNoAllocMaxTheta);
        return fail_msg(IMIN_ERR_INVALID, msg);
    }
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    NA_CUDA(cudaSetDevice(g->device));
    uint8_t* base = nullptr;
    int rc = scratch_address(g->device, &base);
    if (rc) return rc;

    // layout of the static array for this call
    const uint32_t words = static_cast<uint32_t>((g->n + 31) / 32);
    const int where_out = device_pointer(out_delta, g->device);
    if (where_out < 0)
        return fail_msg(IMIN_ERR_INVALID, "out_delta is device memory of another GPU than the graph's");
    const bool dev_out = where_out > 0;
    uint64_t o = 0;
    const uint64_t off_ctl = o;     o = up256(o + sizeof(RoundCtl));
    const uint64_t off_bad = o;     o = up256(o + sizeof(uint32_t));
    const uint64_t off_excl = o;    o = up256(o + 4ull * words);
    const uint64_t off_seeds = o;   o = up256(o + 4ull * n_seeds);
    const uint64_t off_blocked = o; o = up256(o + 4ull * n_blocked);
    const uint64_t off_delta = o;   o = up256(o + (dev_out ? 0ull : 8ull * g->n));
    const uint64_t off_lists = o;   o = up256(o + 4ull * kTiers * theta);
    const uint64_t off_slots = o;

    CtaCfg cfg{};
    uint32_t blocks = 0;
    uint64_t smem = 0;
    if (!cta_plan(g, &cfg, &blocks, &smem))
        return fail_msg(IMIN_ERR_INTERNAL, "the block-per-sample kernel cannot be configured");
    if (off_slots + cfg.slot_bytes > kNoAllocBytes)
        return fail_msg(IMIN_ERR_INVALID, "imin_estimate_decrease_noalloc: request exceeds the static scratch");
    const uint64_t slots = (kNoAllocBytes - off_slots) / cfg.slot_bytes;
    if (slots < blocks) blocks = static_cast<uint32_t>(slots);

    RoundCtl* ctl = reinterpret_cast<RoundCtl*>(base + off_ctl);
    uint32_t* bad = reinterpret_cast<uint32_t*>(base + off_bad);
    uint32_t* excl = reinterpret_cast<uint32_t*>(base + off_excl);
    int32_t* dseeds = reinterpret_cast<int32_t*>(base + off_seeds);
    int32_t* dblocked = reinterpret_cast<int32_t*>(base + off_blocked);
    unsigned long long* delta =
        dev_out ? reinterpret_cast<unsigned long long*>(out_delta)
                : reinterpret_cast<unsigned long long*>(base + off_delta);

    // zero what must start at zero; bring the ids into the array
    NA_CUDA(cudaMemsetAsync(base, 0, off_seeds, s));  // control block, flag, bitmask
    NA_CUDA(cudaMemsetAsync(delta, 0, 8ull * g->n, s));
    NA_CUDA(cudaMemcpyAsync(dseeds, seeds, 4ull * n_seeds, cudaMemcpyDefault, s));
    if (n_blocked > 0)
        NA_CUDA(cudaMemcpyAsync(dblocked, blocked, 4ull * n_blocked, cudaMemcpyDefault, s));
    k_mark_ids<<<(n_seeds + 255) / 256, 256, 0, s>>>(dseeds, n_seeds, g->n, excl, bad);
    if (n_blocked > 0) k_mark_ids<<<(n_blocked + 255) / 256, 256, 0, s>>>(dblocked, n_blocked, g->n, excl, bad);
    NA_CUDA(cudaGetLastError());
    uint32_t hbad = 0;
    NA_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (hbad & 1u) return fail_msg(IMIN_ERR_INVALID, "seeds/blocked: vertex id out of range");
    if (hbad & 2u) return fail_msg(IMIN_ERR_INVALID, "seeds/blocked: duplicate vertex or blocked seed");

    SampleParams P{};
    P.g = dev_graph(g);
    P.seeds = dseeds;
    P.ns = static_cast<uint32_t>(n_seeds);
    P.excl = excl;
    P.key_lo = static_cast<uint32_t>(key);
    P.key_hi = static_cast<uint32_t>(key >> 32);
    P.round = round;
    P.theta = theta;
    P.delta = delta;
    P.ctl = ctl;
    P.lists = reinterpret_cast<uint32_t*>(base + off_lists);
    P.done = nullptr;
    P.stats = nullptr;
    NA_CUDA(launch_cta_tier(P, cfg, blocks, smem, base + off_slots, s));

    RoundCtl hctl;
    NA_CUDA(cudaMemcpyAsync(&hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, s));
    if (!dev_out)
        NA_CUDA(cudaMemcpyAsync(out_delta, delta, 8ull * g->n, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (hctl.error & kErrInternal) return fail_msg(IMIN_ERR_INTERNAL, "dominator iteration did not converge");
    if (hctl.count[kTierWhole] > 0)
        return fail_msg(IMIN_ERR_CAPACITY,
                        "imin_estimate_decrease_noalloc: a sampled cascade needs the whole-graph "
                        "tier, which this entry point does not run");
    return IMIN_OK;
}
