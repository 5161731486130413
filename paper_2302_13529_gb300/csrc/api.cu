// api.cu -- the C ABI declared in include/imin.h.
//
// Host code only: argument checks, device buffers, and the order of kernel launches that
// makes up Alg. 2 (one call), Alg. 3 (b calls, each followed by a selection) and Alg. 4
// (phase-1 calls with selection over CB, then replacement calls with an on-device stop flag).
// All launches of one entry point go to the caller's stream; per-call buffers come from the
// stream-ordered allocator and are released on the same stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "imin.h"
#include "internal.h"

using namespace imin;

namespace imin {

// Last error message of the calling thread, in a fixed buffer (recording it never allocates).
thread_local char g_err[512] = "";

int fail_msg(int code, const char* msg)
{
    std::snprintf(g_err, sizeof(g_err), "%s", msg);
    return code;
}

}  // namespace imin

namespace {

int fail(int code, const std::string& msg) { return fail_msg(code, msg.c_str()); }

int fail_cuda(cudaError_t e, const char* where)
{
    cudaGetLastError();  // clear a sticky launch error, if any
    const int code = e == cudaErrorMemoryAllocation ? IMIN_ERR_NOMEM : IMIN_ERR_CUDA;
    return fail(code, std::string(where) + ": " + cudaGetErrorString(e));
}

#define IMIN_CUDA(call)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call); \
    } while (0)

// ---- measurement hooks (not part of the method) -------------------------------------------
// Kernel kinds: the three sample tiers, the selection, everything else.
enum Kind { kKindTier0 = 0, kKindTier1, kKindTier2, kKindCta, kKindSelect, kKindOther, kKinds };

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_profile_on{0};
std::mutex g_prof_mu;
uint64_t g_prof_launches[kKinds] = {};
double g_prof_ms[kKinds] = {};
thread_local imin_stats g_last_stats = {};

// CUDA-event timing of each launch of one entry point, on the stream it is launched on.
struct CallTimer {
    cudaStream_t s;
    bool on;
    std::vector<std::tuple<int, cudaEvent_t, cudaEvent_t>> recs;
    explicit CallTimer(cudaStream_t st) : s(st), on(g_profile_on.load() != 0) {}
    ~CallTimer()
    {
        for (auto& r : recs) {
            cudaEventDestroy(std::get<1>(r));
            cudaEventDestroy(std::get<2>(r));
        }
    }
    // Record `ev` on the stream. While the stream is being captured into a CUDA graph the record
    // becomes an event-record node of the graph (cudaEventRecordExternal), so the events time the
    // kernels each time the graph runs.
    cudaError_t record(cudaEvent_t ev)
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(s, &cs);
        if (e != cudaSuccess) return e;
        if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
        return cudaEventRecord(ev, s);
    }
    // Enqueue `launch` (returns cudaError_t, sets *launched) bracketed by events.
    template <typename F>
    cudaError_t run(int kind, F&& launch)
    {
        cudaEvent_t a = nullptr, b = nullptr;
        if (on) {
            cudaError_t e = cudaEventCreate(&a);
            if (e == cudaSuccess) e = cudaEventCreate(&b);
            if (e == cudaSuccess) e = record(a);
            if (e != cudaSuccess) return e;
        }
        bool launched = false;
        cudaError_t e = launch(&launched);
        if (launched) g_launches.fetch_add(1, std::memory_order_relaxed);
        if (on) {
            if (e == cudaSuccess && launched) e = record(b);
            recs.emplace_back(launched ? kind : -1, a, b);
        }
        return e;
    }
    // After the stream has been synchronized: add the measured times to the totals.
    void collect()
    {
        if (!on) return;
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (auto& r : recs) {
            const int kind = std::get<0>(r);
            if (kind < 0) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, std::get<1>(r), std::get<2>(r)) == cudaSuccess) {
                g_prof_ms[kind] += ms;
                g_prof_launches[kind] += 1;
            }
        }
    }
};

// Captures the launches of a driver's rounds into one CUDA graph and launches it. Capture runs on
// a private stream that first waits for the caller's stream (the legacy default stream cannot be
// captured); the caller's stream then waits for the graph. Per-kernel profiling events become
// event-record nodes of the graph. Disabled by IMIN_NO_GRAPHS=1.
struct GraphScope {
    cudaStream_t user = nullptr, cap = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool on = false, capturing = false;

    static bool enabled()
    {
        const char* v = std::getenv("IMIN_NO_GRAPHS");
        return !(v && *v && *v != '0');
    }
    cudaError_t begin(cudaStream_t s)
    {
        user = s;
        on = enabled();
        if (!on) return cudaSuccess;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, user);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev, 0);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        capturing = e == cudaSuccess;
        return e;
    }
    cudaStream_t stream() const { return on ? cap : user; }
    cudaError_t end()
    {
        if (!on) return cudaSuccess;
        capturing = false;
        cudaError_t e = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, cap);
        if (e == cudaSuccess) e = cudaEventRecord(ev, cap);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(user, ev, 0);
        return e;
    }
    ~GraphScope()
    {
        if (capturing) {  // an error left the capture open: close and drop it
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cap, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev) cudaEventDestroy(ev);
        if (cap) cudaStreamDestroy(cap);
    }
};

bool is_device_ptr(const void* p)
{
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy `count` elements that may live on the host or the device into a host vector.
template <typename T>
int to_host(const T* p, int64_t count, std::vector<T>& out, cudaStream_t s, const char* what)
{
    out.resize(static_cast<size_t>(count));
    if (count == 0) return IMIN_OK;
    if (p == nullptr) return fail(IMIN_ERR_INVALID, std::string(what) + " is NULL");
    if (is_device_ptr(p)) {
        IMIN_CUDA(cudaMemcpyAsync(out.data(), p, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
        IMIN_CUDA(cudaStreamSynchronize(s));
    } else {
        std::memcpy(out.data(), p, sizeof(T) * count);
    }
    return IMIN_OK;
}

// Stream-ordered device buffers released at scope exit.
struct Arena {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit Arena(cudaStream_t st) : s(st) {}
    ~Arena()
    {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    cudaError_t alloc(T** out, uint64_t count)
    {
        void* p = nullptr;
        const uint64_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
        cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e == cudaSuccess) ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return e;
    }
};

void keep_pool_memory(int device)
{
    static bool done[64] = {};
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t threshold = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
    }
    done[device] = true;
}

int check_ids(const std::vector<int32_t>& ids, int32_t n, std::vector<uint8_t>& mark, uint8_t tag,
              const char* what)
{
    for (int32_t v : ids) {
        if (v < 0 || v >= n) return fail(IMIN_ERR_INVALID, std::string(what) + ": vertex id out of range");
        if (mark[v] != 0) {
            return fail(IMIN_ERR_INVALID, std::string(what) +
                        (mark[v] == tag ? ": duplicate vertex" : ": vertex is also a seed"));
        }
        mark[v] = tag;
    }
    return IMIN_OK;
}

// Everything one query needs on the device besides its graph.
struct Query {
    Arena arena;
    TierPlan plan{};
    int32_t* seeds = nullptr;
    uint32_t* excl = nullptr;
    unsigned long long* delta = nullptr;
    uint32_t* lists = nullptr;
    unsigned long long* stats = nullptr;
    uint8_t* scratch1 = nullptr;
    uint8_t* scratch2 = nullptr;
    uint8_t* scratch3 = nullptr;
    uint8_t* handoff = nullptr;  // the warp tier's hand-off snapshots (after the block tier's slots)
    int32_t words = 0;
    explicit Query(cudaStream_t s) : arena(s) {}
};

int setup_query(const imin_graph* g, const std::vector<int32_t>& seeds, uint32_t theta,
                unsigned long long* out_delta_dev, uint32_t cutoff, Query& q)
{
    cudaStream_t s = q.arena.s;
    q.words = (g->n + 31) / 32;
    q.plan = plan_tiers(g->dev, g->n, g->m, static_cast<uint32_t>(seeds.size()), cutoff);
    IMIN_CUDA(q.arena.alloc(&q.seeds, seeds.size()));
    IMIN_CUDA(q.arena.alloc(&q.excl, q.words));
    if (out_delta_dev != nullptr) {
        q.delta = out_delta_dev;
    } else {
        IMIN_CUDA(q.arena.alloc(&q.delta, g->n));
    }
    IMIN_CUDA(q.arena.alloc(&q.lists, static_cast<uint64_t>(kTiers) * theta));
    IMIN_CUDA(q.arena.alloc(&q.stats, kStCount));
    IMIN_CUDA(q.arena.alloc(&q.scratch1, q.plan.scratch_bytes[1]));
    IMIN_CUDA(q.arena.alloc(&q.scratch2, q.plan.scratch_bytes[2]));
    // with the warp tier in front of the block tier, one hand-off snapshot per sample it may give
    // up on, after the block tier's slots: the block tier resumes those samples where it stopped
    uint64_t handoff_bytes = 0;
    if (q.plan.use_cta && q.plan.cta.from_list && q.plan.blocks[0] > 0) {
        const Handoff h = handoff_layout(q.plan.cfg[0].rcap, q.plan.cfg[0].dcap, q.plan.cfg[0].ecap);
        q.plan.cta.handoff_stride = h.stride;
        handoff_bytes = static_cast<uint64_t>(theta) * h.stride;
    }
    IMIN_CUDA(q.arena.alloc(&q.scratch3, q.plan.scratch_bytes[kTierCta] + handoff_bytes));
    if (handoff_bytes > 0) q.handoff = q.scratch3 + q.plan.scratch_bytes[kTierCta];
    if (q.plan.use_cta) IMIN_CUDA(prepare_cta_scratch(q.plan.cta, q.plan.blocks[kTierCta], q.scratch3, s));
    IMIN_CUDA(cudaMemcpyAsync(q.seeds, seeds.data(), sizeof(int32_t) * seeds.size(),
                              cudaMemcpyHostToDevice, s));
    IMIN_CUDA(cudaMemsetAsync(q.excl, 0, sizeof(uint32_t) * q.words, s));
    IMIN_CUDA(cudaMemsetAsync(q.delta, 0, sizeof(unsigned long long) * g->n, s));
    IMIN_CUDA(cudaMemsetAsync(q.stats, 0, sizeof(unsigned long long) * kStCount, s));
    IMIN_CUDA(cudaMemsetAsync(q.scratch1, 0xFF, q.plan.scratch_bytes[1], s));
    IMIN_CUDA(cudaMemsetAsync(q.scratch2, 0xFF, q.plan.scratch_bytes[2], s));
    IMIN_CUDA(launch_build_excl(q.excl, q.seeds, static_cast<int32_t>(seeds.size()), s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return IMIN_OK;
}

// One Alg. 2 call: the sample tiers in order -- 0 (when the cutoff is not 0), 3, 2 when the
// block-per-sample tier applies, otherwise 0, 1, 2. A tier with no blocks planned is skipped.
cudaError_t enqueue_call(const SampleParams& P, const Query& q, CallTimer& T)
{
    static const int kWarpOrder[] = {0, 1, 2};
    static const int kCtaOrder[] = {0, kTierCta, kTierWhole};
    const int* order = q.plan.use_cta ? kCtaOrder : kWarpOrder;
    const int count = 3;
    for (int k = 0; k < count; ++k) {
        const int t = order[k];
        uint8_t* scr = t == 1 ? q.scratch1 : (t == 2 ? q.scratch2 : (t == kTierCta ? q.scratch3 : q.handoff));
        const int kind = t == kTierCta ? kKindCta : kKindTier0 + t;
        const cudaError_t e = T.run(kind, [&](bool* launched) {
            return launch_sample_tier(t, P, q.plan, scr, T.s, launched);
        });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_select(const SelectParams& sp, CallTimer& T)
{
    return T.run(kKindSelect, [&](bool* launched) {
        *launched = true;
        return launch_select(sp, T.s);
    });
}

void record_stats(const unsigned long long* h)
{
    imin_stats& st = g_last_stats;
    st = imin_stats{};
    for (int t = 0; t < kTiers; ++t) {
        const unsigned long long* x = h + t * kStPerTier;
        st.samples += x[kStSamples];
        st.reached += x[kStReached];
        st.examined_edges += x[kStExamined];
        st.live_edges += x[kStLive];
        st.nontree_edges += x[kStNontree];
        st.dom_passes += x[kStPasses];
        st.tier_samples[t] = x[kStSamples];
        st.tier_reached[t] = x[kStReached];
        st.tier_examined_edges[t] = x[kStExamined];
        st.tier_live_edges[t] = x[kStLive];
    }
}

SampleParams sample_params(const imin_graph* g, const Query& q, uint32_t ns, uint32_t theta,
                           uint64_t key, uint32_t round, RoundCtl* ctl, const int32_t* done)
{
    SampleParams P;
    P.g = dev_graph(g);
    P.seeds = q.seeds;
    P.ns = ns;
    P.excl = q.excl;
    P.key_lo = static_cast<uint32_t>(key);
    P.key_hi = static_cast<uint32_t>(key >> 32);
    P.round = round;
    P.theta = theta;
    P.delta = q.delta;
    P.ctl = ctl;
    P.lists = q.lists;
    P.done = done;
    P.stats = q.stats;
    return P;
}

int check_ctl(const std::vector<RoundCtl>& ctl)
{
    uint32_t err = 0;
    for (const RoundCtl& c : ctl) err |= c.error;
    if (err & kErrInternal) return fail(IMIN_ERR_INTERNAL, "dominator iteration did not converge");
    if (err & kErrCapacity)
        return fail(IMIN_ERR_CAPACITY, "a sampled cascade exceeded the largest tier's capacity");
    return IMIN_OK;
}

int common_checks(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, uint32_t theta,
                  cudaStream_t s, std::vector<int32_t>& hseeds, std::vector<uint8_t>& mark)
{
    if (g == nullptr) return fail(IMIN_ERR_INVALID, "graph handle is NULL");
    if (n_seeds < 1 || n_seeds > g->n) return fail(IMIN_ERR_INVALID, "n_seeds must be in [1, n]");
    if (theta < 1) return fail(IMIN_ERR_INVALID, "theta must be >= 1");
    if (cudaSetDevice(g->device) != cudaSuccess) return fail(IMIN_ERR_CUDA, "cudaSetDevice failed");
    int rc = to_host(seeds, n_seeds, hseeds, s, "seeds");
    if (rc) return rc;
    mark.assign(static_cast<size_t>(g->n), 0);
    return check_ids(hseeds, g->n, mark, 1, "seeds");
}

// ---- warp/block cutoff autotuner -----------------------------------------------------------
// Samples whose cascade stays within the cutoff (non-seed vertices) finish in the warp tier 0,
// whose per-sample overhead is lower; bigger ones are re-run by the block tier. The best cutoff
// depends on the graph's cascade-size distribution and on |S| (seeds take tier-0 space), so it
// is measured: after one untimed warm-up call, kTuneReps Alg. 2 calls per candidate (round 0
// of the caller's key, no blockers), interleaved across candidates so that a clock or load change
// hits all of them alike; the candidate with the smallest minimum time wins. Each call samples
// 24 graphs per resident block of the block tier (at least 8,192, at most 65,536), so that the
// end of a call -- blocks finishing their last cascades at different times -- does not decide
// the comparison. The cost is bounded: the warm-up call samples at most as many graphs as the
// caller asked for (and at most 1,024); from its time per sample, each timed call is sized to
// take about kTuneCallMs, and when fewer than 4 samples per block would fit in that time (graphs
// whose cascades are huge, where the cutoff hardly matters) the default is kept untimed. The
// choice never changes a result -- only which tier computes each sample -- and is cached per
// graph handle and seed-set size class, and process-wide under the graph's fingerprint, so that
// a new handle of the same graph reuses it.

constexpr uint32_t kCutoffs[] = {0, 64, 96, 128, 192};
constexpr int kTuneReps = 3;
constexpr float kTuneCallMs = 2.0f;

std::mutex g_tune_mu;
std::map<std::pair<uint64_t, int>, int32_t> g_tuned;  // (fingerprint, size class) -> cutoff

// Identity of a graph for the process-wide tuning cache: a 64-bit mix of its sizes, its device
// and about 4,096 evenly spaced entries of each CSR array. Two different graphs that collide
// share a cutoff, which can cost speed but never changes a result.
uint64_t fingerprint(const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                     const std::vector<uint32_t>& thr, int32_t n, int64_t m, int device)
{
    uint64_t h = 0xcbf29ce484222325ull;
    auto mix = [&](uint64_t x) {
        h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        h *= 0x100000001b3ull;
    };
    mix(static_cast<uint64_t>(n));
    mix(static_cast<uint64_t>(m));
    mix(static_cast<uint64_t>(device));
    const int64_t sr = std::max<int64_t>(1, (static_cast<int64_t>(n) + 1) / 4096);
    for (int64_t i = 0; i <= n; i += sr) mix(static_cast<uint32_t>(rp[i]));
    const int64_t se = std::max<int64_t>(1, m / 4096);
    for (int64_t e = 0; e < m; e += se) mix((static_cast<uint64_t>(static_cast<uint32_t>(col[e])) << 32) | thr[e]);
    return h;
}

uint32_t cta_blocks(const imin_graph* g, size_t ns)
{
    const TierPlan p = plan_tiers(g->dev, g->n, g->m, static_cast<uint32_t>(ns), 0);
    return std::max<uint32_t>(p.blocks[kTierCta], 1u);
}

int size_class(size_t ns)
{
    int c = 0;
    while (c < 31 && (size_t{1} << c) < ns) ++c;
    return c;
}

// Device time of one Alg. 2 call (round 0, no blockers) with the given cutoff.
// warp_done (optional): receives the number of samples the warp tier 0 finished.
int time_call(const imin_graph* g, const std::vector<int32_t>& seeds, uint64_t key, uint32_t cutoff,
              uint32_t theta, cudaStream_t s, float* ms, unsigned long long* warp_done = nullptr)
{
    Query q(s);
    int rc = setup_query(g, seeds, theta, nullptr, cutoff, q);
    if (rc) return rc;
    RoundCtl* ctl = nullptr;
    IMIN_CUDA(q.arena.alloc(&ctl, 1));
    IMIN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(RoundCtl), s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    IMIN_CUDA(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        CallTimer T(s);
        const SampleParams P = sample_params(g, q, static_cast<uint32_t>(seeds.size()), theta, key, 0,
                                             ctl, nullptr);
        e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = enqueue_call(P, q, T);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        T.collect();
    }
    std::vector<RoundCtl> hctl(1);
    unsigned long long hstats[kStCount] = {};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hctl.data(), ctl, sizeof(RoundCtl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hstats, q.stats, sizeof(hstats), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    IMIN_CUDA(e);
    if (warp_done != nullptr) *warp_done = hstats[kStSamples];  // tier 0's slots come first
    return check_ctl(hctl);
}

// theta_hint: the caller's samples per call (0: unknown), which bounds the warm-up call.
int tune_cutoff(const imin_graph* g, const std::vector<int32_t>& seeds, uint64_t key, cudaStream_t s,
                uint32_t theta_hint, uint32_t* out)
{
    constexpr int kCand = static_cast<int>(sizeof(kCutoffs) / sizeof(kCutoffs[0]));
    float warm = 0.f, t[kCand];
    const uint32_t blocks = cta_blocks(g, seeds.size());
    const uint32_t tw = std::max<uint32_t>(1, std::min<uint32_t>(1024, theta_hint ? theta_hint : 1024));
    unsigned long long warp_done = 0;
    int rc = time_call(g, seeds, key, kDefaultCutoff, tw, s, &warm, &warp_done);  // warm-up, cost
    if (rc) return rc;
    double per_sample = std::max(1e-7, static_cast<double>(warm) / tw);  // ms
    if (kTuneCallMs / per_sample < 4.0 * blocks) {
        // too costly to compare by timing: keep the warp tier only if it finished at least a
        // tenth of the warm-up's samples (otherwise its partial work is mostly thrown away)
        *out = 10 * warp_done >= tw ? kDefaultCutoff : 0u;
        return IMIN_OK;
    }
    // a small warm-up is dominated by its slowest block; re-estimate on a call of the planned size
    uint32_t theta = static_cast<uint32_t>(std::min<double>({kTuneCallMs / per_sample, 24.0 * blocks, 65536.0}));
    rc = time_call(g, seeds, key, kDefaultCutoff, theta, s, &warm);
    if (rc) return rc;
    per_sample = std::max(1e-7, static_cast<double>(warm) / theta);
    theta = static_cast<uint32_t>(std::min<double>({std::max(kTuneCallMs / per_sample, 4.0 * blocks),
                                                    24.0 * blocks, 65536.0}));
    for (int rep = 0; rep < kTuneReps; ++rep) {
        for (int i = 0; i < kCand; ++i) {
            float ms = 0.f;
            rc = time_call(g, seeds, key, kCutoffs[i], theta, s, &ms);
            if (rc) return rc;
            t[i] = rep == 0 ? ms : std::min(t[i], ms);
        }
    }
    int best = 0;
    for (int i = 1; i < kCand; ++i)
        if (t[i] < t[best]) best = i;
    *out = kCutoffs[best];
    return IMIN_OK;
}

// The cutoff for a call: IMIN_TIER0_VERTICES forces one; IMIN_AUTOTUNE=0, or a stream being
// captured (the tuner synchronizes), gives the default; otherwise the tuned value, tuning on first
// use for this graph and seed-set size class.
int cutoff_for(const imin_graph* g, const std::vector<int32_t>& seeds, uint64_t key, uint32_t theta_hint,
               cudaStream_t s, uint32_t* out)
{
    if (const char* v = std::getenv("IMIN_TIER0_VERTICES"); v && *v) {
        *out = static_cast<uint32_t>(std::strtoul(v, nullptr, 10));
        return IMIN_OK;
    }
    *out = kDefaultCutoff;
    if (const char* v = std::getenv("IMIN_AUTOTUNE"); v && *v == '0') return IMIN_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return IMIN_OK;
    }
    if (cs != cudaStreamCaptureStatusNone) return IMIN_OK;
    const int cls = size_class(seeds.size());
    std::lock_guard<std::mutex> lk(g->tune_mu);
    if (g->cutoff[cls] >= 0) {
        *out = static_cast<uint32_t>(g->cutoff[cls]);
        return IMIN_OK;
    }
    {
        std::lock_guard<std::mutex> lk2(g_tune_mu);
        const auto it = g_tuned.find({g->fingerprint, cls});
        if (it != g_tuned.end()) {
            g->cutoff[cls] = it->second;
            *out = static_cast<uint32_t>(it->second);
            return IMIN_OK;
        }
    }
    const int rc = tune_cutoff(g, seeds, key, s, theta_hint, out);
    if (rc) return rc;
    g->cutoff[cls] = static_cast<int32_t>(*out);
    std::lock_guard<std::mutex> lk2(g_tune_mu);
    g_tuned[{g->fingerprint, cls}] = static_cast<int32_t>(*out);
    return IMIN_OK;
}

}  // namespace

namespace imin {

int tuned_cutoff(const imin_graph* g, const std::vector<int32_t>& seeds, uint64_t key, uint32_t theta_hint,
                 cudaStream_t s, uint32_t* out)
{
    return cutoff_for(g, seeds, key, theta_hint, s, out);
}

}  // namespace imin

namespace {

int estimate_impl(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                  const int32_t* blocked, int32_t n_blocked, uint32_t theta, uint64_t key,
                  uint32_t round, uint64_t* out_delta, imin_stats* stats, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> hseeds, hblocked;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, theta, s, hseeds, mark);
    if (rc) return rc;
    if (out_delta == nullptr) return fail(IMIN_ERR_INVALID, "out_delta is NULL");
    if (n_blocked < 0) return fail(IMIN_ERR_INVALID, "n_blocked must be >= 0");
    rc = to_host(blocked, n_blocked, hblocked, s, "blocked");
    if (rc) return rc;
    rc = check_ids(hblocked, g->n, mark, 2, "blocked");
    if (rc) return rc;

    const bool dev_out = is_device_ptr(out_delta);
    uint32_t cutoff = 0;
    rc = cutoff_for(g, hseeds, key, theta, s, &cutoff);
    if (rc) return rc;
    Query q(s);
    rc = setup_query(g, hseeds, theta, dev_out ? reinterpret_cast<unsigned long long*>(out_delta) : nullptr,
                     cutoff, q);
    if (rc) return rc;
    RoundCtl* ctl = nullptr;
    int32_t* dblocked = nullptr;
    IMIN_CUDA(q.arena.alloc(&ctl, 1));
    IMIN_CUDA(q.arena.alloc(&dblocked, hblocked.size()));
    IMIN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(RoundCtl), s));
    if (!hblocked.empty()) {
        IMIN_CUDA(cudaMemcpyAsync(dblocked, hblocked.data(), sizeof(int32_t) * hblocked.size(),
                                  cudaMemcpyHostToDevice, s));
        IMIN_CUDA(launch_build_excl(q.excl, dblocked, n_blocked, s));
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    CallTimer T(s);
    const SampleParams P = sample_params(g, q, static_cast<uint32_t>(n_seeds), theta, key, round, ctl, nullptr);
    IMIN_CUDA(enqueue_call(P, q, T));

    std::vector<RoundCtl> hctl(1);
    unsigned long long hstats[kStCount];
    IMIN_CUDA(cudaMemcpyAsync(hctl.data(), ctl, sizeof(RoundCtl), cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaMemcpyAsync(hstats, q.stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
    if (!dev_out) {
        IMIN_CUDA(cudaMemcpyAsync(out_delta, q.delta, sizeof(uint64_t) * g->n, cudaMemcpyDeviceToHost, s));
    }
    IMIN_CUDA(cudaStreamSynchronize(s));
    T.collect();
    rc = check_ctl(hctl);
    if (rc) return rc;
    record_stats(hstats);
    if (stats != nullptr) *stats = g_last_stats;
    return IMIN_OK;
}

// Def. 3 by simulation: out_sum = sum over theta sampled graphs of |R| (seeds included).
int spread_impl(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, const int32_t* blocked,
                int32_t n_blocked, uint32_t theta, uint64_t key, uint32_t round, uint64_t* out_sum,
                void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> hseeds, hblocked;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, theta, s, hseeds, mark);
    if (rc) return rc;
    if (out_sum == nullptr) return fail(IMIN_ERR_INVALID, "out_sum is NULL");
    if (n_blocked < 0) return fail(IMIN_ERR_INVALID, "n_blocked must be >= 0");
    rc = to_host(blocked, n_blocked, hblocked, s, "blocked");
    if (rc) return rc;
    rc = check_ids(hblocked, g->n, mark, 2, "blocked");
    if (rc) return rc;

    Query q(s);
    rc = setup_query(g, hseeds, theta, nullptr, 0, q);
    if (rc) return rc;
    if (!q.plan.use_cta) return fail(IMIN_ERR_INTERNAL, "the spread kernel needs the block-per-sample tier");
    RoundCtl* ctl = nullptr;
    int32_t* dblocked = nullptr;
    unsigned long long* dsum = nullptr;
    IMIN_CUDA(q.arena.alloc(&ctl, 1));
    IMIN_CUDA(q.arena.alloc(&dblocked, hblocked.size()));
    IMIN_CUDA(q.arena.alloc(&dsum, 1));
    IMIN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(RoundCtl), s));
    IMIN_CUDA(cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), s));
    if (!hblocked.empty()) {
        IMIN_CUDA(cudaMemcpyAsync(dblocked, hblocked.data(), sizeof(int32_t) * hblocked.size(),
                                  cudaMemcpyHostToDevice, s));
        IMIN_CUDA(launch_build_excl(q.excl, dblocked, n_blocked, s));
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    CallTimer T(s);
    const SampleParams P = sample_params(g, q, static_cast<uint32_t>(n_seeds), theta, key, round, ctl, nullptr);
    IMIN_CUDA(T.run(kKindCta, [&](bool* launched) {
        *launched = true;
        return launch_spread(P, q.plan.cta, q.plan.blocks[kTierCta], q.plan.smem_bytes[kTierCta], q.scratch3,
                             dsum, s);
    }));
    std::vector<RoundCtl> hctl(1);
    unsigned long long hstats[kStCount], hsum = 0;
    IMIN_CUDA(cudaMemcpyAsync(hctl.data(), ctl, sizeof(RoundCtl), cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaMemcpyAsync(hstats, q.stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaMemcpyAsync(&hsum, dsum, sizeof(hsum), cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaStreamSynchronize(s));
    T.collect();
    if (hctl[0].error & kErrCapacity)
        return fail(IMIN_ERR_CAPACITY, "a sampled cascade exceeded the block tier's slot capacity (2^18 vertices)");
    rc = check_ctl(hctl);
    if (rc) return rc;
    record_stats(hstats);
    *out_sum = hsum;
    return IMIN_OK;
}

// ---- comparison algorithms of Sec. 5 (scored by simulation) --------------------------------

// Simulated spread of `nsets` blocker sets of k vertices each (host array hsets), on top of the
// blocked vertices hblocked: hsums[i] = sum over samples [0, theta) of call `round` of |R| with
// set i blocked. mark: 1 for seeds, 2 for hblocked, 0 otherwise (restored on return).
int spread_sets_core(const imin_graph* g, const std::vector<int32_t>& hseeds, const std::vector<int32_t>& hblocked,
                     std::vector<uint8_t>& mark, const int32_t* hsets, int64_t nsets, int32_t k, uint32_t theta,
                     uint64_t key, uint32_t round, uint64_t* hsums, cudaStream_t s)
{
    if (nsets < 0 || k < 0 || k > 64) return fail(IMIN_ERR_INVALID, "sets: need n_sets >= 0 and 0 <= set_size <= 64");
    if (nsets == 0) return IMIN_OK;
    if (static_cast<double>(nsets) * theta > 9.0e18) return fail(IMIN_ERR_INVALID, "n_sets * theta too large");
    for (int64_t i = 0; i < nsets; ++i) {
        const int32_t* set = hsets + i * k;
        int rc = IMIN_OK;
        int32_t j = 0;
        for (; j < k; ++j) {
            const int32_t v = set[j];
            if (v < 0 || v >= g->n) { rc = fail(IMIN_ERR_INVALID, "sets: vertex id out of range"); break; }
            if (mark[v] != 0) {
                rc = fail(IMIN_ERR_INVALID, "sets: a vertex is a seed, blocked, or repeated in its set");
                break;
            }
            mark[v] = 3;
        }
        for (int32_t t = 0; t < j; ++t) mark[set[t]] = 0;
        if (rc) return rc;
    }
    Query q(s);
    int rc = setup_query(g, hseeds, theta, nullptr, 0, q);
    if (rc) return rc;
    if (!q.plan.use_cta) return fail(IMIN_ERR_INTERNAL, "the spread kernel needs the block-per-sample tier");
    RoundCtl* ctl = nullptr;
    int32_t* dblocked = nullptr;
    int32_t* dsets = nullptr;
    unsigned long long* dsums = nullptr;
    unsigned long long* cursor = nullptr;
    IMIN_CUDA(q.arena.alloc(&ctl, 1));
    IMIN_CUDA(q.arena.alloc(&dblocked, hblocked.size()));
    IMIN_CUDA(q.arena.alloc(&dsets, static_cast<uint64_t>(nsets) * k));
    IMIN_CUDA(q.arena.alloc(&dsums, static_cast<uint64_t>(nsets)));
    IMIN_CUDA(q.arena.alloc(&cursor, 1));
    IMIN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(RoundCtl), s));
    IMIN_CUDA(cudaMemsetAsync(dsums, 0, sizeof(unsigned long long) * nsets, s));
    IMIN_CUDA(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
    if (k > 0)
        IMIN_CUDA(cudaMemcpyAsync(dsets, hsets, sizeof(int32_t) * nsets * k, cudaMemcpyHostToDevice, s));
    if (!hblocked.empty()) {
        IMIN_CUDA(cudaMemcpyAsync(dblocked, hblocked.data(), sizeof(int32_t) * hblocked.size(),
                                  cudaMemcpyHostToDevice, s));
        IMIN_CUDA(launch_build_excl(q.excl, dblocked, static_cast<int32_t>(hblocked.size()), s));
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    CallTimer T(s);
    const SampleParams P = sample_params(g, q, static_cast<uint32_t>(hseeds.size()), theta, key, round, ctl, nullptr);
    IMIN_CUDA(T.run(kKindCta, [&](bool* launched) {
        *launched = true;
        return launch_spread_sets(P, q.plan.cta, q.plan.blocks[kTierCta], q.plan.smem_bytes[kTierCta], q.scratch3,
                                  dsets, static_cast<uint32_t>(k),
                                  static_cast<unsigned long long>(nsets) * theta, cursor, dsums, s);
    }));
    RoundCtl hctl;
    IMIN_CUDA(cudaMemcpyAsync(&hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaMemcpyAsync(hsums, dsums, sizeof(uint64_t) * nsets, cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaStreamSynchronize(s));
    T.collect();
    if (hctl.error & kErrCapacity)
        return fail(IMIN_ERR_CAPACITY, "a sampled cascade exceeded the block tier's slot capacity (2^18 vertices)");
    if (hctl.error & kErrInternal) return fail(IMIN_ERR_INTERNAL, "the spread kernel failed");
    return IMIN_OK;
}

// Philox4x32-10 on the host (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3), for the random
// blocker baseline.
void philox_host(const uint32_t ctr[4], uint64_t key, uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = static_cast<uint32_t>(key), k1 = static_cast<uint32_t>(key >> 32);
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = 0xD2511F53ull * x0, p1 = 0xCD9E8D57ull * x2;
        const uint32_t y0 = static_cast<uint32_t>(p1 >> 32) ^ x1 ^ k0;
        const uint32_t y2 = static_cast<uint32_t>(p0 >> 32) ^ x3 ^ k1;
        x1 = static_cast<uint32_t>(p1);
        x3 = static_cast<uint32_t>(p0);
        x0 = y0;
        x2 = y2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

enum class Driver { kAdvancedGreedy, kGreedyReplace };

int greedy_impl(Driver which, const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                int32_t b, uint32_t theta, uint64_t key, int32_t* out_blockers,
                int32_t* out_count, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> hseeds;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, theta, s, hseeds, mark);
    if (rc) return rc;
    if (b < 0) return fail(IMIN_ERR_INVALID, "b must be >= 0");
    if (out_count == nullptr) return fail(IMIN_ERR_INVALID, "out_count is NULL");
    if (b > 0 && out_blockers == nullptr) return fail(IMIN_ERR_INVALID, "out_blockers is NULL");
    *out_count = 0;
    if (b == 0) return IMIN_OK;

    uint32_t cutoff = 0;
    rc = cutoff_for(g, hseeds, key, theta, s, &cutoff);
    if (rc) return rc;
    Query q(s);
    rc = setup_query(g, hseeds, theta, nullptr, cutoff, q);
    if (rc) return rc;
    int32_t* dB = nullptr;
    int32_t* flags = nullptr;  // [0] = done, [1] = vertex unblocked in the current round
    unsigned long long* part_d = nullptr;
    int32_t* part_id = nullptr;
    uint32_t* ticket = nullptr;
    const int sel_blocks = select_blocks();
    IMIN_CUDA(q.arena.alloc(&dB, static_cast<uint64_t>(b)));
    IMIN_CUDA(q.arena.alloc(&flags, 2));
    IMIN_CUDA(q.arena.alloc(&part_d, sel_blocks));
    IMIN_CUDA(q.arena.alloc(&part_id, sel_blocks));
    IMIN_CUDA(q.arena.alloc(&ticket, 1));
    IMIN_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int32_t), s));
    IMIN_CUDA(cudaMemsetAsync(ticket, 0, sizeof(uint32_t), s));

    SelectParams sp{};
    sp.delta = q.delta;
    sp.n = g->n;
    sp.excl = q.excl;
    sp.blockers = dB;
    sp.part_d = part_d;
    sp.part_id = part_id;
    sp.ticket = ticket;

    int32_t count = 0;
    std::vector<RoundCtl> hctl;
    RoundCtl* ctl = nullptr;
    CallTimer T(s);
    GraphScope G;
    if (which == Driver::kAdvancedGreedy) {
        count = std::min<int32_t>(b, g->n - n_seeds);
        if (count > 0) {
            IMIN_CUDA(q.arena.alloc(&ctl, count));
            IMIN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(RoundCtl) * count, s));
        }
        IMIN_CUDA(G.begin(s));
        T.s = G.stream();
        for (int32_t i = 0; i < count; ++i) {
            const SampleParams P = sample_params(g, q, n_seeds, theta, key, static_cast<uint32_t>(i),
                                                 ctl + i, nullptr);
            IMIN_CUDA(enqueue_call(P, q, T));
            sp.pos = i;
            IMIN_CUDA(enqueue_select(sp, T));
        }
        IMIN_CUDA(G.end());
        hctl.resize(count);
    } else {
        uint32_t* cb = nullptr;
        uint32_t* cb_count = nullptr;
        IMIN_CUDA(q.arena.alloc(&cb, q.words));
        IMIN_CUDA(q.arena.alloc(&cb_count, 1));
        IMIN_CUDA(cudaMemsetAsync(cb, 0, sizeof(uint32_t) * q.words, s));
        IMIN_CUDA(cudaMemsetAsync(cb_count, 0, sizeof(uint32_t), s));
        IMIN_CUDA(launch_build_cb(dev_graph(g), q.seeds, n_seeds, q.excl, cb, cb_count, s));
        g_launches.fetch_add(2, std::memory_order_relaxed);
        uint32_t hcb = 0;
        IMIN_CUDA(cudaMemcpyAsync(&hcb, cb_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        IMIN_CUDA(cudaStreamSynchronize(s));
        count = std::min<int32_t>(b, static_cast<int32_t>(hcb));
        const int32_t calls = 2 * count;
        if (calls > 0) {
            IMIN_CUDA(q.arena.alloc(&ctl, calls));
            IMIN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(RoundCtl) * calls, s));
        }
        IMIN_CUDA(G.begin(s));
        T.s = G.stream();
        const cudaStream_t rs = G.stream();
        uint32_t round = 0;
        // phase 1: greedy over the seeds' out-neighbours
        for (int32_t i = 0; i < count; ++i, ++round) {
            const SampleParams P = sample_params(g, q, n_seeds, theta, key, round, ctl + round, nullptr);
            IMIN_CUDA(enqueue_call(P, q, T));
            SelectParams p1 = sp;
            p1.cand = cb;
            p1.pos = i;
            IMIN_CUDA(enqueue_select(p1, T));
        }
        // phase 2: replacements in reverse insertion order, stopping when a blocker stays
        for (int32_t i = count - 1; i >= 0; --i, ++round) {
            IMIN_CUDA(T.run(kKindOther, [&](bool* launched) {
                *launched = true;
                return launch_unblock(q.excl, dB, i, flags, flags + 1, rs);
            }));
            const SampleParams P = sample_params(g, q, n_seeds, theta, key, round, ctl + round, flags);
            IMIN_CUDA(enqueue_call(P, q, T));
            SelectParams p2 = sp;
            p2.pos = i;
            p2.done = flags;
            p2.cur = flags + 1;
            IMIN_CUDA(enqueue_select(p2, T));
        }
        IMIN_CUDA(G.end());
        hctl.resize(calls);
    }

    std::vector<int32_t> hB(static_cast<size_t>(count));
    unsigned long long hstats[kStCount];
    IMIN_CUDA(cudaMemcpyAsync(hstats, q.stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
    if (count > 0) {
        IMIN_CUDA(cudaMemcpyAsync(hctl.data(), ctl, sizeof(RoundCtl) * hctl.size(), cudaMemcpyDeviceToHost, s));
        IMIN_CUDA(cudaMemcpyAsync(hB.data(), dB, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
    }
    IMIN_CUDA(cudaStreamSynchronize(s));
    T.collect();
    rc = check_ctl(hctl);
    if (rc) return rc;
    record_stats(hstats);
    if (count > 0) {
        if (is_device_ptr(out_blockers)) {
            IMIN_CUDA(cudaMemcpyAsync(out_blockers, dB, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, s));
            IMIN_CUDA(cudaStreamSynchronize(s));
        } else {
            std::memcpy(out_blockers, hB.data(), sizeof(int32_t) * count);
        }
    }
    *out_count = count;
    return IMIN_OK;
}


// ---- batched drivers ------------------------------------------------------------------------

// Queue granularity (samples per work item) of batched steps, picked by imin_autotune_batch and
// kept for the life of the process under a fingerprint of the batch: the driver and, per query,
// its graph's fingerprint, seed-set size, budget and theta.
std::mutex g_chunk_mu;
std::map<uint64_t, uint32_t> g_batch_chunk;

uint64_t batch_fingerprint(Driver which, const imin_query* qs, int32_t nq)
{
    uint64_t h = which == Driver::kGreedyReplace ? 0x9e3779b97f4a7c15ull : 0x7f4a7c159e3779b9ull;
    auto mix = [&](uint64_t x) {
        h ^= x + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        h *= 0x100000001b3ull;
    };
    for (int32_t i = 0; i < nq; ++i) {
        mix(qs[i].graph ? qs[i].graph->fingerprint : 0);
        mix((static_cast<uint64_t>(static_cast<uint32_t>(qs[i].n_seeds)) << 32) | static_cast<uint32_t>(qs[i].b));
        mix(qs[i].theta);
    }
    return h;
}

// force_chunk: samples per work item (0: the tuned value of this batch, else the default rule);
// max_steps: stop after that many steps (< 0: run to the end; used by the tuner, whose outputs
// are then partial).
int batch_impl(Driver which, imin_query* qs, int32_t nq, void* stream, uint32_t force_chunk = 0,
               int32_t max_steps = -1)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nq < 0 || (nq > 0 && qs == nullptr)) return fail(IMIN_ERR_INVALID, "queries array is NULL");
    if (nq == 0) return IMIN_OK;
    const bool gr = which == Driver::kGreedyReplace;
    // validation, host copies of the seed sets
    std::vector<std::vector<int32_t>> hseeds(nq);
    int32_t max_n = 0, max_m = 0;
    uint32_t max_ns = 0;
    for (int32_t i = 0; i < nq; ++i) {
        imin_query& Q = qs[i];
        Q.out_count = 0;
        std::vector<uint8_t> mark;
        int rc = common_checks(Q.graph, Q.seeds, Q.n_seeds, Q.theta, s, hseeds[i], mark);
        if (rc) return rc;
        if (Q.b < 0) return fail(IMIN_ERR_INVALID, "b must be >= 0");
        if (Q.b > 0 && Q.out_blockers == nullptr) return fail(IMIN_ERR_INVALID, "out_blockers is NULL");
        if (Q.graph->device != qs[0].graph->device)
            return fail(IMIN_ERR_INVALID, "all graphs of a batch must live on one device");
        max_n = std::max(max_n, Q.graph->n);
        max_m = std::max(max_m, Q.graph->m);
        max_ns = std::max<uint32_t>(max_ns, static_cast<uint32_t>(Q.n_seeds));
    }
    const imin_graph* g0 = qs[0].graph;
    // size classes: the launch of a class reserves the bitmap of its own largest graph
    std::vector<int> cls(nq);
    int32_t cls_n[kBatchClasses] = {}, cls_m[kBatchClasses] = {};
    for (int32_t i = 0; i < nq; ++i) {
        cls[i] = batch_class(qs[i].graph->n);
        cls_n[cls[i]] = std::max(cls_n[cls[i]], qs[i].graph->n);
        cls_m[cls[i]] = std::max(cls_m[cls[i]], qs[i].graph->m);
    }
    CtaCfg cfg[kBatchClasses] = {};
    uint32_t cta_blocks[kBatchClasses] = {};
    uint64_t cta_smem[kBatchClasses] = {}, cta_bytes = 0, global_bytes = 0;
    for (int k = 0; k < kBatchClasses; ++k) {
        if (cls_n[k] == 0) continue;
        uint64_t bytes = 0;
        if (!plan_batch_cta(g0->dev, cls_n[k], cls_m[k], &cfg[k], &cta_blocks[k], &cta_smem[k], &bytes))
            return fail(IMIN_ERR_INTERNAL, "the batched block-per-sample kernel cannot be configured");
        // the shared-bitmap classes run one after another on one buffer; the global-bitmap
        // class keeps its own, whose bitmaps must stay zero between samples
        if (k == kBatchGlobalClass) global_bytes = bytes;
        else cta_bytes = std::max(cta_bytes, bytes);
    }
    const TierPlan wp = plan_tiers(g0->dev, max_n, max_m, max_ns, 0);
    bool all_ic = true;  // every graph IC: the launches take the IC-only kernels
    for (int32_t i = 0; i < nq; ++i) all_ic = all_ic && qs[i].graph->model == 0;
    // the warp tier in front: queries whose seed sets fit its shared-memory working set and whose
    // graph's tuned warp/block cutoff (the single-query autotuner's, per graph and seed-set size
    // class, tuned here on first use) is not 0; the launch holds the largest of those cutoffs
    std::vector<uint8_t> warp_q(nq, 0);
    uint32_t warp_ns = 0, cutoff = 0;
    for (int32_t i = 0; i < nq; ++i) {
        if (static_cast<uint32_t>(qs[i].n_seeds) > kBatchWarpMaxSeeds) continue;
        uint32_t c = 0;
        const int rc = tuned_cutoff(qs[i].graph, hseeds[i], qs[i].key, qs[i].theta, s, &c);
        if (rc) return rc;
        if (c > 0) {
            warp_q[i] = 1;
            warp_ns = std::max<uint32_t>(warp_ns, static_cast<uint32_t>(qs[i].n_seeds));
            cutoff = std::max(cutoff, c);
        }
    }
    TierCfg wcfg{};
    uint32_t warp_blocks = 0;
    uint64_t warp_smem = 0;
    if (warp_ns == 0 || !plan_batch_warp(g0->dev, warp_ns, cutoff, &wcfg, &warp_blocks, &warp_smem))
        std::fill(warp_q.begin(), warp_q.end(), 0);

    // per-query device buffers, packed into one allocation
    struct Off { uint64_t excl, cb, delta, flags, done; };
    std::vector<Off> off(nq);
    std::vector<uint64_t> seed_off(nq + 1, 0), blk_off(nq + 1, 0);
    uint64_t total = 0;
    auto take = [&](uint64_t bytes) { const uint64_t o = total; total = align16(total + bytes); return o; };
    uint64_t sum_theta = 0;
    for (int32_t i = 0; i < nq; ++i) {
        const imin_query& Q = qs[i];
        const uint64_t words = (Q.graph->n + 31) / 32;
        off[i].excl = take(4ull * words);
        off[i].cb = take(gr ? 4ull * words : 0);
        off[i].delta = take(8ull * Q.graph->n);
        off[i].flags = take(8);
        off[i].done = take(warp_q[i] ? Q.theta : 0);
        seed_off[i + 1] = seed_off[i] + static_cast<uint64_t>(Q.n_seeds);
        blk_off[i + 1] = blk_off[i] + static_cast<uint64_t>(Q.b);
        sum_theta += Q.theta;
    }
    Arena arena(s);
    uint8_t* buf = nullptr;
    BatchQuery* dq = nullptr;
    uint8_t* cta_scratch = nullptr;
    uint8_t* whole_scratch = nullptr;
    unsigned long long* stats = nullptr;
    uint2* over = nullptr;
    uint32_t* cb_counts = nullptr;
    int32_t* dseeds = nullptr;
    int32_t* dblk = nullptr;
    IMIN_CUDA(arena.alloc(&buf, total));
    IMIN_CUDA(arena.alloc(&dseeds, seed_off[nq]));
    IMIN_CUDA(arena.alloc(&dblk, std::max<uint64_t>(blk_off[nq], 1)));
    IMIN_CUDA(arena.alloc(&dq, nq));
    uint8_t* global_scratch = nullptr;
    IMIN_CUDA(arena.alloc(&cta_scratch, cta_bytes));
    IMIN_CUDA(arena.alloc(&global_scratch, global_bytes));
    if (global_bytes > 0)
        IMIN_CUDA(prepare_cta_scratch(cfg[kBatchGlobalClass], cta_blocks[kBatchGlobalClass], global_scratch, s));
    IMIN_CUDA(arena.alloc(&whole_scratch, wp.scratch_bytes[kTierWhole]));
    IMIN_CUDA(arena.alloc(&stats, kStCount));
    // hand-off snapshots of the samples the warp tier gives up on, per size class after the
    // overflow items (at most 1 GiB in all; samples beyond the lists' room run from the start)
    const uint32_t over_cap = static_cast<uint32_t>(std::min<uint64_t>(sum_theta, 0xFFFFFFFFull));
    uint32_t handoff_stride = 0, handoff_cap = 0;
    uint64_t warp_theta = 0;
    for (int32_t i = 0; i < nq; ++i)
        if (warp_q[i]) warp_theta += qs[i].theta;
    if (warp_theta > 0) {
        const Handoff h = handoff_layout(wcfg.rcap, wcfg.dcap, wcfg.ecap);
        handoff_stride = h.stride;
        handoff_cap = static_cast<uint32_t>(
            std::min<uint64_t>(warp_theta, (1ull << 30) / (static_cast<uint64_t>(kBatchClasses) * h.stride)));
    }
    uint8_t* over_raw = nullptr;
    IMIN_CUDA(arena.alloc(&over_raw, batch_handoff_offset(over_cap) +
                                         static_cast<uint64_t>(kBatchClasses) * handoff_cap * handoff_stride));
    over = reinterpret_cast<uint2*>(over_raw);
    IMIN_CUDA(arena.alloc(&cb_counts, nq));
    IMIN_CUDA(cudaMemsetAsync(buf, 0, total, s));
    IMIN_CUDA(cudaMemsetAsync(whole_scratch, 0xFF, wp.scratch_bytes[kTierWhole], s));
    IMIN_CUDA(cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * kStCount, s));
    IMIN_CUDA(cudaMemsetAsync(cb_counts, 0, sizeof(uint32_t) * nq, s));
    std::vector<int32_t> hseed_all(seed_off[nq]);
    for (int32_t i = 0; i < nq; ++i)
        std::memcpy(hseed_all.data() + seed_off[i], hseeds[i].data(), 4ull * hseeds[i].size());
    IMIN_CUDA(cudaMemcpyAsync(dseeds, hseed_all.data(), 4ull * seed_off[nq], cudaMemcpyHostToDevice, s));
    for (int32_t i = 0; i < nq; ++i) {
        IMIN_CUDA(launch_build_excl(reinterpret_cast<uint32_t*>(buf + off[i].excl), dseeds + seed_off[i],
                                    qs[i].n_seeds, s));
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    std::vector<int32_t> count(nq);
    if (gr) {
        for (int32_t i = 0; i < nq; ++i) {
            IMIN_CUDA(launch_build_cb(dev_graph(qs[i].graph), dseeds + seed_off[i],
                                      qs[i].n_seeds, reinterpret_cast<uint32_t*>(buf + off[i].excl),
                                      reinterpret_cast<uint32_t*>(buf + off[i].cb), cb_counts + i, s));
            g_launches.fetch_add(2, std::memory_order_relaxed);
        }
        std::vector<uint32_t> hcb(nq);
        IMIN_CUDA(cudaMemcpyAsync(hcb.data(), cb_counts, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost, s));
        IMIN_CUDA(cudaStreamSynchronize(s));
        for (int32_t i = 0; i < nq; ++i) count[i] = std::min<int32_t>(qs[i].b, static_cast<int32_t>(hcb[i]));
    } else {
        for (int32_t i = 0; i < nq; ++i) count[i] = std::min<int32_t>(qs[i].b, qs[i].graph->n - qs[i].n_seeds);
    }
    std::vector<BatchQuery> hq(nq);
    int32_t steps = 0;
    for (int32_t i = 0; i < nq; ++i) {
        const imin_query& Q = qs[i];
        BatchQuery& d = hq[i];
        d.g = dev_graph(Q.graph);
        d.seeds = dseeds + seed_off[i];
        d.ns = static_cast<uint32_t>(Q.n_seeds);
        d.excl = reinterpret_cast<uint32_t*>(buf + off[i].excl);
        d.cb = gr ? reinterpret_cast<uint32_t*>(buf + off[i].cb) : nullptr;
        d.key_lo = static_cast<uint32_t>(Q.key);
        d.key_hi = static_cast<uint32_t>(Q.key >> 32);
        d.theta = Q.theta;
        d.delta = reinterpret_cast<unsigned long long*>(buf + off[i].delta);
        d.blockers = dblk + blk_off[i];
        d.count = count[i];
        d.flags = reinterpret_cast<int32_t*>(buf + off[i].flags);
        d.start = 0;
        d.gr = gr ? 1 : 0;
        d.done = warp_q[i] ? buf + off[i].done : nullptr;
        steps = std::max(steps, gr ? 2 * count[i] : count[i]);
    }
    if (max_steps >= 0) steps = std::min(steps, max_steps);
    IMIN_CUDA(cudaMemcpyAsync(dq, hq.data(), sizeof(BatchQuery) * nq, cudaMemcpyHostToDevice, s));

    // per-step item prefixes: one row per size class (queries of other classes and inactive
    // ones contribute no items) and one row, kRows - 1, for the warp tier
    // queue granularity: samples per work item, about 16 items per resident block of a step and
    // at most 16 (measured on the 256-query batch: 16 samples per item 0.912 s, 4: 0.924 s,
    // 32: 0.926 s, 64: 0.978 s, 128: 1.095 s; IMIN_BATCH_CHUNK overrides it for measurements)
    uint32_t chunk = static_cast<uint32_t>(std::max<uint64_t>(
        1, std::min<uint64_t>(16, sum_theta / (static_cast<uint64_t>(cta_blocks[0] + cta_blocks[1] +
                                                                     cta_blocks[2] + cta_blocks[3]) * 16 + 1))));
    if (force_chunk > 0) {
        chunk = force_chunk;
    } else {
        std::lock_guard<std::mutex> lk(g_chunk_mu);
        const auto it = g_batch_chunk.find(batch_fingerprint(which, qs, nq));
        if (it != g_batch_chunk.end()) chunk = it->second;
    }
    if (const char* v = std::getenv("IMIN_BATCH_CHUNK"); v && *v)
        chunk = std::max<uint32_t>(1, static_cast<uint32_t>(std::strtoul(v, nullptr, 10)));
    constexpr int kRows = kBatchClasses + 1;
    const size_t stride = static_cast<size_t>(nq) + 1;
    std::vector<unsigned long long> hprefix(static_cast<size_t>(steps) * kRows * stride, 0);
    std::vector<uint8_t> class_busy(static_cast<size_t>(steps) * kRows, 0);
    for (int32_t c = 0; c < steps; ++c) {
        for (int k = 0; k < kRows; ++k) {
            unsigned long long* pr = hprefix.data() + (static_cast<size_t>(c) * kRows + k) * stride;
            for (int32_t i = 0; i < nq; ++i) {
                const bool in_row = k < kBatchClasses ? cls[i] == k : warp_q[i] != 0;
                const bool act = in_row && (gr ? c < 2 * count[i] : c < count[i]);
                pr[i + 1] = pr[i] + (act ? (qs[i].theta + chunk - 1) / chunk : 0);
            }
            class_busy[static_cast<size_t>(c) * kRows + k] = pr[nq] > 0;
        }
    }
    unsigned long long* dprefix = nullptr;
    BatchCtl* ctl = nullptr;
    IMIN_CUDA(arena.alloc(&dprefix, std::max<uint64_t>(hprefix.size(), 1)));
    IMIN_CUDA(arena.alloc(&ctl, std::max(steps, 1)));
    if (!hprefix.empty())
        IMIN_CUDA(cudaMemcpyAsync(dprefix, hprefix.data(), sizeof(unsigned long long) * hprefix.size(),
                                  cudaMemcpyHostToDevice, s));
    IMIN_CUDA(cudaMemsetAsync(ctl, 0, sizeof(BatchCtl) * std::max(steps, 1), s));

    CallTimer T(s);
    GraphScope G;
    IMIN_CUDA(G.begin(s));
    T.s = G.stream();
    const cudaStream_t rs = G.stream();
    for (int32_t c = 0; c < steps; ++c) {
        BatchStep B{};
        B.q = dq;
        B.nq = static_cast<uint32_t>(nq);
        B.chunk = chunk;
        B.step = static_cast<uint32_t>(c);
        B.ctl = ctl + c;
        B.over = over;
        B.over_cap = over_cap;
        B.handoff_stride = handoff_stride;
        B.handoff_cap = handoff_cap;
        B.stats = stats;
        B.all_ic = all_ic ? 1u : 0u;
        if (gr) {  // phase-2 unblocking of every GreedyReplace query at this step
            IMIN_CUDA(T.run(kKindOther, [&](bool* l) { *l = true; return launch_batch_unblock(B, rs); }));
        }
        if (class_busy[static_cast<size_t>(c) * kRows + kBatchClasses]) {
            BatchStep Bw = B;
            Bw.prefix = dprefix + (static_cast<size_t>(c) * kRows + kBatchClasses) * stride;
            IMIN_CUDA(T.run(kKindTier0, [&](bool* l) {
                *l = true;
                return launch_batch_warp(Bw, wcfg, warp_blocks, warp_smem, rs);
            }));
        }
        for (int k = 0; k < kBatchClasses; ++k) {
            if (!class_busy[static_cast<size_t>(c) * kRows + k]) continue;
            BatchStep Bk = B;
            Bk.cls = static_cast<uint32_t>(k);
            Bk.prefix = dprefix + (static_cast<size_t>(c) * kRows + k) * stride;
            IMIN_CUDA(T.run(kKindCta, [&](bool* l) {
                *l = true;
                return launch_batch_cta(Bk, cfg[k], cta_blocks[k], cta_smem[k],
                                        k == kBatchGlobalClass ? global_scratch : cta_scratch, rs);
            }));
        }
        // the whole-graph and selection kernels do not read the item prefixes
        B.prefix = dprefix;
        IMIN_CUDA(T.run(kKindTier2, [&](bool* l) {
            *l = true;
            return launch_batch_whole(B, wp.cfg[kTierWhole], wp.blocks[kTierWhole], whole_scratch, rs);
        }));
        IMIN_CUDA(T.run(kKindSelect, [&](bool* l) { *l = true; return launch_batch_select(B, rs); }));
    }
    IMIN_CUDA(G.end());

    std::vector<BatchCtl> hctl(std::max(steps, 1));
    std::vector<int32_t> hblk(std::max<uint64_t>(blk_off[nq], 1));
    unsigned long long hstats[kStCount];
    IMIN_CUDA(cudaMemcpyAsync(hctl.data(), ctl, sizeof(BatchCtl) * hctl.size(), cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaMemcpyAsync(hblk.data(), dblk, 4ull * blk_off[nq], cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaMemcpyAsync(hstats, stats, sizeof(hstats), cudaMemcpyDeviceToHost, s));
    IMIN_CUDA(cudaStreamSynchronize(s));
    T.collect();
    uint32_t err = 0;
    for (int32_t c = 0; c < steps; ++c) err |= hctl[c].error;
    if (err & kErrInternal) return fail(IMIN_ERR_INTERNAL, "dominator iteration did not converge");
    if (err & kErrCapacity)
        return fail(IMIN_ERR_CAPACITY, "a sampled cascade exceeded the largest tier's capacity");
    record_stats(hstats);
    for (int32_t i = 0; i < nq; ++i) {
        imin_query& Q = qs[i];
        const int32_t* src = hblk.data() + blk_off[i];
        if (count[i] > 0) {
            if (is_device_ptr(Q.out_blockers)) {
                IMIN_CUDA(cudaMemcpyAsync(Q.out_blockers, dblk + blk_off[i], 4ull * count[i],
                                          cudaMemcpyDeviceToDevice, s));
            } else {
                std::memcpy(Q.out_blockers, src, 4ull * count[i]);
            }
        }
        Q.out_count = count[i];
    }
    IMIN_CUDA(cudaStreamSynchronize(s));
    return IMIN_OK;
}

}  // namespace

extern "C" {

int imin_abi_version(void) { return IMIN_ABI_VERSION; }

const char* imin_last_error(void) { return g_err; }

}  // extern "C"

namespace {

// Graph upload shared by the IC and LT loaders. model 1 (LT): thr[e] + 1 is edge e's share of
// 2^32; the in-edges of each vertex take consecutive intervals in ascending edge id, whose starts
// are computed here, and the shares of one vertex must not exceed 2^32.
int load_impl(int32_t n, int64_t m, const int32_t* row_ptr, const int32_t* col, const uint32_t* thr,
              int32_t model, void* stream, imin_graph** out)
{
    if (out == nullptr) return fail(IMIN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n <= 0) return fail(IMIN_ERR_INVALID, "n must be > 0");
    if (m < 0 || m >= (int64_t(1) << 31) - 4) return fail(IMIN_ERR_INVALID, "m must be in [0, 2^31 - 4)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> hrp, hcol;
    std::vector<uint32_t> hthr;
    int rc = to_host(row_ptr, static_cast<int64_t>(n) + 1, hrp, s, "row_ptr");
    if (!rc) rc = to_host(col, m, hcol, s, "col");
    if (!rc) rc = to_host(thr, m, hthr, s, "thr");
    if (rc) return rc;
    if (hrp[0] != 0 || hrp[n] != m) return fail(IMIN_ERR_INVALID, "row_ptr[0] must be 0 and row_ptr[n] == m");
    for (int32_t u = 0; u < n; ++u)
        if (hrp[u + 1] < hrp[u]) return fail(IMIN_ERR_INVALID, "row_ptr must be non-decreasing");
    for (int64_t e = 0; e < m; ++e)
        if (hcol[e] < 0 || hcol[e] >= n) return fail(IMIN_ERR_INVALID, "col entry out of range");
    std::vector<uint32_t> hlo;
    if (model == 1) {
        std::vector<uint64_t> acc(static_cast<size_t>(n), 0);
        hlo.resize(static_cast<size_t>(m));
        for (int64_t e = 0; e < m; ++e) {
            uint64_t& a = acc[static_cast<size_t>(hcol[e])];
            hlo[e] = static_cast<uint32_t>(a);
            a += static_cast<uint64_t>(hthr[e]) + 1;
            if (a > (uint64_t(1) << 32))
                return fail(IMIN_ERR_INVALID, "LT weights: the in-edge shares of a vertex exceed 2^32");
        }
    }

    imin_graph* g = new imin_graph();
    cudaGetDevice(&g->device);
    g->dev = device_info();
    g->n = n;
    g->m = static_cast<int32_t>(m);
    g->model = model;
    g->fingerprint = fingerprint(hrp, hcol, hthr, n, m, g->device) ^ (static_cast<uint64_t>(model) << 63);
    keep_pool_memory(g->device);
    const int64_t m4 = ((m + 3) / 4) * 4 + 4;  // padded so the last 16-byte group is in bounds
    hcol.resize(m4, 0);
    hthr.resize(m4, 0);
    cudaError_t e = cudaMalloc(&g->row_ptr, sizeof(int32_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->col, sizeof(int32_t) * m4);
    if (e == cudaSuccess) e = cudaMalloc(&g->thr4, sizeof(uint32_t) * m4);
    if (e == cudaSuccess && model == 1) {
        hlo.resize(m4, 0);
        e = cudaMalloc(&g->lo4, sizeof(uint32_t) * m4);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->lo4, hlo.data(), sizeof(uint32_t) * m4, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->row_ptr, hrp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->col, hcol.data(), sizeof(int32_t) * m4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->thr4, hthr.data(), sizeof(uint32_t) * m4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        imin_free_graph(g);
        return fail_cuda(e, "imin_load_graph");
    }
    *out = g;
    return IMIN_OK;
}

}  // namespace

extern "C" {

int imin_load_graph(int32_t n, int64_t m, const int32_t* row_ptr, const int32_t* col,
                    const uint32_t* thr, void* stream, imin_graph** out)
{
    g_err[0] = '\0';
    return load_impl(n, m, row_ptr, col, thr, 0, stream, out);
}

int imin_load_graph_lt(int32_t n, int64_t m, const int32_t* row_ptr, const int32_t* col,
                       const uint32_t* weight, void* stream, imin_graph** out)
{
    g_err[0] = '\0';
    return load_impl(n, m, row_ptr, col, weight, 1, stream, out);
}

int imin_graph_model(const imin_graph* g)
{
    if (g == nullptr) return fail(IMIN_ERR_INVALID, "graph handle is NULL");
    return g->model;
}

int imin_free_graph(imin_graph* g)
{
    if (g == nullptr) return IMIN_OK;
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->thr4);
    cudaFree(g->lo4);
    delete g;
    return IMIN_OK;
}

int imin_graph_info(const imin_graph* g, int32_t* n, int64_t* m)
{
    if (g == nullptr) return fail(IMIN_ERR_INVALID, "graph handle is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return IMIN_OK;
}

uint64_t imin_launch_count(void) { return g_launches.load(); }

int imin_last_stats(imin_stats* out)
{
    if (out == nullptr) return fail(IMIN_ERR_INVALID, "out is NULL");
    *out = g_last_stats;
    return IMIN_OK;
}

int imin_profile_enable(int on)
{
    g_profile_on.store(on != 0);
    return IMIN_OK;
}

int imin_profile_read(imin_profile* out, int reset)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (out != nullptr) {
        for (int k = 0; k < kKinds; ++k) {
            out->launches[k] = g_prof_launches[k];
            out->ms[k] = g_prof_ms[k];
        }
    }
    if (reset) {
        for (int k = 0; k < kKinds; ++k) {
            g_prof_launches[k] = 0;
            g_prof_ms[k] = 0.0;
        }
    }
    return IMIN_OK;
}

int imin_estimate_decrease(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                           const int32_t* blocked, int32_t n_blocked, uint32_t theta,
                           uint64_t key, uint32_t round, uint64_t* out_delta, void* stream)
{
    g_err[0] = '\0';
    return estimate_impl(g, seeds, n_seeds, blocked, n_blocked, theta, key, round, out_delta,
                         nullptr, stream);
}

int imin_estimate_decrease_stats(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                                 const int32_t* blocked, int32_t n_blocked, uint32_t theta,
                                 uint64_t key, uint32_t round, uint64_t* out_delta,
                                 imin_stats* stats, void* stream)
{
    g_err[0] = '\0';
    return estimate_impl(g, seeds, n_seeds, blocked, n_blocked, theta, key, round, out_delta,
                         stats, stream);
}

int imin_estimate_spread(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                         const int32_t* blocked, int32_t n_blocked, uint32_t theta, uint64_t key,
                         uint32_t round, uint64_t* out_sum, void* stream)
{
    g_err[0] = '\0';
    return spread_impl(g, seeds, n_seeds, blocked, n_blocked, theta, key, round, out_sum, stream);
}

int imin_autotune(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, uint64_t key,
                  void* stream, int32_t* out_cutoff)
{
    g_err[0] = '\0';
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (out_cutoff == nullptr) return fail(IMIN_ERR_INVALID, "out_cutoff is NULL");
    std::vector<int32_t> hseeds;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, 1, s, hseeds, mark);
    if (rc) return rc;
    uint32_t c = 0;
    {
        std::lock_guard<std::mutex> lk(g->tune_mu);
        rc = tune_cutoff(g, hseeds, key, s, 0, &c);
        if (rc) return rc;
        g->cutoff[size_class(hseeds.size())] = static_cast<int32_t>(c);
        std::lock_guard<std::mutex> lk2(g_tune_mu);
        g_tuned[{g->fingerprint, size_class(hseeds.size())}] = static_cast<int32_t>(c);
    }
    *out_cutoff = static_cast<int32_t>(c);
    return IMIN_OK;
}

int imin_autotune_batch(imin_query* queries, int32_t n_queries, int32_t driver, void* stream,
                        int32_t* out_chunk)
{
    g_err[0] = '\0';
    if (out_chunk == nullptr) return fail(IMIN_ERR_INVALID, "out_chunk is NULL");
    if (driver != 0 && driver != 1) return fail(IMIN_ERR_INVALID, "driver must be 0 (AG) or 1 (GR)");
    if (n_queries < 0 || (n_queries > 0 && queries == nullptr)) return fail(IMIN_ERR_INVALID, "queries array is NULL");
    *out_chunk = 0;
    if (n_queries == 0) return IMIN_OK;
    const Driver which = driver == 1 ? Driver::kGreedyReplace : Driver::kAdvancedGreedy;
    // the tuning calls write into scratch outputs, never into the caller's
    std::vector<imin_query> q(queries, queries + n_queries);
    std::vector<std::vector<int32_t>> outs(static_cast<size_t>(n_queries));
    for (int32_t i = 0; i < n_queries; ++i) {
        outs[i].assign(static_cast<size_t>(std::max(q[i].b, 1)), 0);
        q[i].out_blockers = outs[i].data();
    }
    constexpr uint32_t kChunks[] = {4, 8, 16, 32, 64};
    constexpr int32_t kTuneSteps = 3;
    int rc = batch_impl(which, q.data(), n_queries, stream, 16, kTuneSteps);  // warm-up, cutoff tuning
    if (rc) return rc;
    double best_s = 0;
    uint32_t best = 16;
    for (int rep = 0; rep < 2; ++rep) {
        for (uint32_t c : kChunks) {
            const auto t0 = std::chrono::steady_clock::now();
            rc = batch_impl(which, q.data(), n_queries, stream, c, kTuneSteps);
            if (rc) return rc;
            const double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if ((rep == 0 && c == kChunks[0]) || s < best_s) {
                best_s = s;
                best = c;
            }
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_chunk_mu);
        g_batch_chunk[batch_fingerprint(which, queries, n_queries)] = best;
    }
    *out_chunk = static_cast<int32_t>(best);
    return IMIN_OK;
}

int imin_advanced_greedy(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                         uint32_t theta, uint64_t key, int32_t* out_blockers, int32_t* out_count,
                         void* stream)
{
    g_err[0] = '\0';
    return greedy_impl(Driver::kAdvancedGreedy, g, seeds, n_seeds, b, theta, key, out_blockers,
                       out_count, stream);
}

int imin_batch_advanced_greedy(imin_query* queries, int32_t n_queries, void* stream)
{
    g_err[0] = '\0';
    return batch_impl(Driver::kAdvancedGreedy, queries, n_queries, stream);
}

int imin_batch_greedy_replace(imin_query* queries, int32_t n_queries, void* stream)
{
    g_err[0] = '\0';
    return batch_impl(Driver::kGreedyReplace, queries, n_queries, stream);
}

int imin_greedy_replace(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                        uint32_t theta, uint64_t key, int32_t* out_blockers, int32_t* out_count,
                        void* stream)
{
    g_err[0] = '\0';
    return greedy_impl(Driver::kGreedyReplace, g, seeds, n_seeds, b, theta, key, out_blockers,
                       out_count, stream);
}

int imin_estimate_spread_sets(const imin_graph* g, const int32_t* seeds, int32_t n_seeds,
                              const int32_t* blocked, int32_t n_blocked, const int32_t* sets,
                              int32_t n_sets, int32_t set_size, uint32_t theta, uint64_t key,
                              uint32_t round, uint64_t* out_sums, void* stream)
{
    g_err[0] = '\0';
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> hseeds, hblocked, hsets;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, theta, s, hseeds, mark);
    if (rc) return rc;
    if (n_blocked < 0 || n_sets < 0 || set_size < 0)
        return fail(IMIN_ERR_INVALID, "n_blocked, n_sets and set_size must be >= 0");
    if (n_sets > 0 && out_sums == nullptr) return fail(IMIN_ERR_INVALID, "out_sums is NULL");
    rc = to_host(blocked, n_blocked, hblocked, s, "blocked");
    if (!rc) rc = check_ids(hblocked, g->n, mark, 2, "blocked");
    if (!rc) rc = to_host(sets, static_cast<int64_t>(n_sets) * set_size, hsets, s, "sets");
    if (rc) return rc;
    std::vector<uint64_t> hsums(static_cast<size_t>(n_sets));
    rc = spread_sets_core(g, hseeds, hblocked, mark, hsets.data(), n_sets, set_size, theta, key, round,
                          hsums.data(), s);
    if (rc || n_sets == 0) return rc;
    if (is_device_ptr(out_sums)) {
        IMIN_CUDA(cudaMemcpyAsync(out_sums, hsums.data(), sizeof(uint64_t) * n_sets, cudaMemcpyHostToDevice, s));
        IMIN_CUDA(cudaStreamSynchronize(s));
    } else {
        std::memcpy(out_sums, hsums.data(), sizeof(uint64_t) * n_sets);
    }
    return IMIN_OK;
}

int imin_baseline_greedy(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b, uint32_t r,
                         uint64_t key, int32_t* out_blockers, int32_t* out_count, void* stream)
{
    g_err[0] = '\0';
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> hseeds;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, r, s, hseeds, mark);
    if (rc) return rc;
    if (b < 0) return fail(IMIN_ERR_INVALID, "b must be >= 0");
    if (out_count == nullptr) return fail(IMIN_ERR_INVALID, "out_count is NULL");
    if (b > 0 && out_blockers == nullptr) return fail(IMIN_ERR_INVALID, "out_blockers is NULL");
    *out_count = 0;
    std::vector<int32_t> B, cand;
    std::vector<uint64_t> sums;
    for (int32_t i = 0; i < b; ++i) {
        cand.clear();
        for (int32_t u = 0; u < g->n; ++u)
            if (mark[u] == 0) cand.push_back(u);
        if (cand.empty()) break;
        sums.resize(cand.size());
        // the common spread of G[V \ B] cancels in the decrease: the largest decrease is the
        // smallest spread with u blocked (strict '<' in ascending id keeps the smallest id)
        rc = spread_sets_core(g, hseeds, B, mark, cand.data(), static_cast<int64_t>(cand.size()), 1, r, key,
                              static_cast<uint32_t>(i), sums.data(), s);
        if (rc) return rc;
        size_t x = 0;
        for (size_t t = 1; t < cand.size(); ++t)
            if (sums[t] < sums[x]) x = t;
        B.push_back(cand[x]);
        mark[cand[x]] = 2;
    }
    if (!B.empty()) {
        if (is_device_ptr(out_blockers)) {
            IMIN_CUDA(cudaMemcpyAsync(out_blockers, B.data(), 4 * B.size(), cudaMemcpyHostToDevice, s));
            IMIN_CUDA(cudaStreamSynchronize(s));
        } else {
            std::memcpy(out_blockers, B.data(), 4 * B.size());
        }
    }
    *out_count = static_cast<int32_t>(B.size());
    return IMIN_OK;
}

int imin_exact_blockers(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b, uint32_t r,
                        uint64_t key, int32_t* out_blockers, int32_t* out_count, void* stream)
{
    g_err[0] = '\0';
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> hseeds;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, r, s, hseeds, mark);
    if (rc) return rc;
    if (b < 0) return fail(IMIN_ERR_INVALID, "b must be >= 0");
    if (out_count == nullptr) return fail(IMIN_ERR_INVALID, "out_count is NULL");
    if (b > 0 && out_blockers == nullptr) return fail(IMIN_ERR_INVALID, "out_blockers is NULL");
    *out_count = 0;
    std::vector<int32_t> cand;
    for (int32_t u = 0; u < g->n; ++u)
        if (mark[u] == 0) cand.push_back(u);
    const int32_t c = static_cast<int32_t>(cand.size());
    const int32_t k = std::min(b, c);
    if (k > 64) return fail(IMIN_ERR_INVALID, "exact: at most 64 blockers");
    double subsets = 1.0;  // C(c, k)
    for (int32_t i = 0; i < k; ++i) subsets = subsets * (c - i) / (i + 1);
    if (subsets > 1.0e8) return fail(IMIN_ERR_INVALID, "exact: more than 10^8 blocker sets to score");
    constexpr int64_t kChunk = 1 << 16;
    std::vector<int32_t> idx(static_cast<size_t>(k)), sets, best_set;
    std::vector<uint64_t> sums;
    for (int32_t i = 0; i < k; ++i) idx[i] = i;
    uint64_t best = 0;
    bool have = false, more = true;
    const std::vector<int32_t> none;
    while (more) {
        // the next chunk of k-subsets in lexicographic order of their index vectors
        sets.clear();
        int64_t count = 0;
        while (more && count < kChunk) {
            for (int32_t i = 0; i < k; ++i) sets.push_back(cand[idx[i]]);
            ++count;
            int32_t i = k - 1;
            while (i >= 0 && idx[i] == c - k + i) --i;
            if (i < 0) {
                more = false;
            } else {
                ++idx[i];
                for (int32_t t = i + 1; t < k; ++t) idx[t] = idx[t - 1] + 1;
            }
        }
        sums.resize(static_cast<size_t>(count));
        rc = spread_sets_core(g, hseeds, none, mark, sets.data(), count, k, r, key, 0, sums.data(), s);
        if (rc) return rc;
        for (int64_t t = 0; t < count; ++t) {
            if (!have || sums[t] < best) {
                have = true;
                best = sums[t];
                best_set.assign(sets.begin() + t * k, sets.begin() + (t + 1) * k);
            }
        }
    }
    if (k > 0) {
        if (is_device_ptr(out_blockers)) {
            IMIN_CUDA(cudaMemcpyAsync(out_blockers, best_set.data(), 4ull * k, cudaMemcpyHostToDevice, s));
            IMIN_CUDA(cudaStreamSynchronize(s));
        } else {
            std::memcpy(out_blockers, best_set.data(), 4ull * k);
        }
    }
    *out_count = k;
    return IMIN_OK;
}

int imin_out_degree_blockers(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b,
                             int32_t* out_blockers, int32_t* out_count)
{
    g_err[0] = '\0';
    std::vector<int32_t> hseeds;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, 1, nullptr, hseeds, mark);
    if (rc) return rc;
    if (b < 0 || out_count == nullptr || (b > 0 && out_blockers == nullptr))
        return fail(IMIN_ERR_INVALID, "b must be >= 0 and the outputs non-NULL");
    std::vector<int32_t> rp(static_cast<size_t>(g->n) + 1);
    IMIN_CUDA(cudaMemcpy(rp.data(), g->row_ptr, sizeof(int32_t) * (g->n + 1), cudaMemcpyDeviceToHost));
    std::vector<int32_t> cand;
    for (int32_t u = 0; u < g->n; ++u)
        if (mark[u] == 0) cand.push_back(u);
    std::stable_sort(cand.begin(), cand.end(), [&](int32_t a, int32_t c) {
        return rp[a + 1] - rp[a] > rp[c + 1] - rp[c];
    });
    const int32_t k = std::min<int32_t>(b, static_cast<int32_t>(cand.size()));
    for (int32_t i = 0; i < k; ++i) out_blockers[i] = cand[i];
    *out_count = k;
    return IMIN_OK;
}

int imin_random_blockers(const imin_graph* g, const int32_t* seeds, int32_t n_seeds, int32_t b, uint64_t key,
                         int32_t* out_blockers, int32_t* out_count)
{
    g_err[0] = '\0';
    std::vector<int32_t> hseeds;
    std::vector<uint8_t> mark;
    int rc = common_checks(g, seeds, n_seeds, 1, nullptr, hseeds, mark);
    if (rc) return rc;
    if (b < 0 || out_count == nullptr || (b > 0 && out_blockers == nullptr))
        return fail(IMIN_ERR_INVALID, "b must be >= 0 and the outputs non-NULL");
    std::vector<int32_t> cand;
    for (int32_t u = 0; u < g->n; ++u)
        if (mark[u] == 0) cand.push_back(u);
    const int32_t c = static_cast<int32_t>(cand.size());
    const int32_t k = std::min(b, c);
    for (int32_t t = 0; t < k; ++t) {
        const uint32_t ctr[4] = {static_cast<uint32_t>(t), 0u, 0u, 0xC0000000u};
        uint32_t w[4];
        philox_host(ctr, key, w);
        const int32_t pick = t + static_cast<int32_t>((static_cast<uint64_t>(w[0]) * static_cast<uint64_t>(c - t)) >> 32);
        std::swap(cand[t], cand[pick]);
        out_blockers[t] = cand[t];
    }
    *out_count = k;
    return IMIN_OK;
}

}  // extern "C"
