// noalloc.cu -- imin_estimate_decrease_noalloc: one Alg. 2 call that allocates no memory.
//
// Who needs it: callers that must not allocate device memory at call time -- code that runs
// while a stream is being captured into a CUDA graph (cudaMalloc is not allowed there), code
// whose device memory is owned by another allocator with a fixed budget (a framework's caching
// allocator, a serving process that pre-sizes everything at start-up), and latency-critical
// paths that cannot afford cudaMalloc/cudaFree, which may synchronize the whole device.
//
// What it does: exactly what imin_estimate_decrease computes, with the block-per-sample tier
// (sample_cta.cu), but every byte of working memory it needs besides the caller's inputs and
// output comes from one file-scope device array of kNoAllocBytes (64 MiB). Every GPU that loads
// the library holds that array until the process exits. Its limits follow from its size:
// graphs with at most kNoAllocMaxVertices vertices and at most kNoAllocMaxTheta samples per call;
// bigger requests are rejected with IMIN_ERR_INVALID. A sampled cascade that would need the
// whole-graph fallback tier (more non-tree live edges or BFS levels than the block tier holds)
// makes the call fail with IMIN_ERR_CAPACITY instead of running that tier.
//
// The array is shared by every call on a device and keeps the last call's contents; each call
// clears the parts that must start at zero. Calls that overlap on the GPU (different streams or
// threads without ordering between them) race on it.
//
// Set-up: the first call on each device resolves the array's device address with
// cudaGetSymbolAddress (in host code the array's name is only a host-side stand-in, never a
// device address) and configures the kernel's shared-memory limit; make that first call before
// any stream capture.
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

bool device_pointer(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
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
    const bool dev_out = device_pointer(out_delta);
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
    uint64_t smem = 0, slot_total = 0;
    if (!plan_cta_tier(g->dev, g->n, g->m, &cfg, &blocks, &smem, &slot_total))
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
    P.g = DevGraph{g->n, g->m, g->row_ptr, g->col, g->thr4};
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
