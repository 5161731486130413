// server.cu -- continuous-batching request server for AdvancedGreedy / GreedyReplace queries.
//
// A worker thread owns one CUDA stream and runs steps. Each step advances the admitted requests
// of one graph-size class by one greedy round through the batched kernels (batch.cu): the
// block-per-sample launch over their samples, the whole-graph fallback, and one selection launch
// with a block per request slot. The class a step serves is the one with the least GPU time so
// far among the classes with requests (a class that becomes busy joins at the smallest time of
// the busy ones), so requests on small graphs are not held to the pace of the large graphs'
// rounds; a request that sits a step out keeps its round count (its start step moves with the
// step counter). Requests are admitted
// between steps, in arrival order, while a slot is free and their device state (counters,
// masks, seeds, blockers) fits the memory budget; a request joins at the current step, so its
// own round index is step - start and its random stream is exactly the one the single-query
// driver uses. Finished requests are retired between steps: their blockers are copied to the
// host, their device memory returns to the budget, and waiters are woken.
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "imin.h"
#include "internal.h"

using namespace imin;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kAG = 0;
constexpr int kGR = 1;
constexpr int kPrefixRows = kBatchClasses + 1;  // item prefix rows: size classes, warp tier
constexpr uint32_t kMaxOvertakes = 4;  // later requests of a class that may pass one waiting at the cap

struct Req {
    uint64_t ticket = 0;
    int driver = kAG;
    const imin_graph* g = nullptr;
    std::vector<int32_t> seeds;
    int32_t b = 0;
    uint32_t theta = 0;
    uint64_t key = 0;
    // device state
    int slot = -1;
    uint32_t start = 0;
    int32_t count = 0;
    uint64_t bytes = 0;
    uint8_t* mem = nullptr;
    uint64_t off_seeds = 0, off_excl = 0, off_cb = 0, off_delta = 0, off_blk = 0, off_done = 0;
    bool warp = false;  // its samples go to the warp tier first
    uint32_t cutoff = 0;  // its graph's tuned warp/block cutoff (set at admission)
    uint32_t overtaken = 0;  // later requests of its class admitted while it waited at the cap
    // result
    bool done = false;
    int status = IMIN_OK;
    std::vector<int32_t> result;
    Clock::time_point t_submit, t_done;
};

uint64_t up16(uint64_t x) { return (x + 15) & ~uint64_t(15); }

void plan_request(Req& r, uint32_t cutoff)
{
    const uint64_t words = (static_cast<uint64_t>(r.g->n) + 31) / 32;
    r.warp = cutoff > 0 && r.seeds.size() <= kBatchWarpMaxSeeds;
    uint64_t o = 0;
    r.off_seeds = o; o = up16(o + 4ull * r.seeds.size());
    r.off_excl = o;  o = up16(o + 4ull * words);
    r.off_cb = o;    o = up16(o + (r.driver == kGR ? 4ull * words : 0));
    r.off_delta = o; o = up16(o + 8ull * r.g->n);
    r.off_blk = o;   o = up16(o + 4ull * (r.b > 0 ? r.b : 1));
    r.off_done = o;  o = up16(o + (r.warp ? r.theta : 0));
    r.bytes = o;
}

}  // namespace

struct imin_server {
    uint64_t budget = 0;
    int32_t max_active = 0;
    uint64_t class_cap = 0;  // sampled graphs per step one size class may batch
    int device = 0;
    DeviceInfo dev;
    cudaStream_t s = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    int fatal = IMIN_OK;
    char fatal_msg[256] = "";
    uint64_t next_ticket = 1;
    std::deque<Req*> pending;
    std::vector<Req*> slots;
    std::unordered_map<uint64_t, Req*> reqs;
    uint64_t used = 0;
    // counters
    imin_server_stats st{};

    // device buffers owned by the worker
    BatchQuery* dq = nullptr;
    int32_t* dflags = nullptr;             // [max_active][2]
    unsigned long long* dprefix = nullptr;  // [kPrefixRows][max_active + 1]
    BatchCtl* dctl = nullptr;
    uint32_t* dcb_count = nullptr;          // [max_active]
    uint2* dover = nullptr;
    uint64_t over_cap = 0;
    // pinned host staging
    BatchQuery* hq = nullptr;
    unsigned long long* hprefix = nullptr;
    int32_t* hflags = nullptr;
    BatchCtl* hctl = nullptr;
    uint32_t* hcb = nullptr;
    // kernel plans, grown with the largest graph admitted so far
    int32_t cls_n[kBatchClasses] = {}, cls_m[kBatchClasses] = {};
    CtaCfg cfg[kBatchClasses] = {};
    uint32_t cta_blocks[kBatchClasses] = {};
    uint64_t cta_smem[kBatchClasses] = {};
    uint8_t* cta_scratch[kBatchClasses] = {};
    int32_t whole_n = 0, whole_m = 0;
    uint32_t whole_ns = 0;
    TierPlan whole{};
    uint8_t* whole_scratch = nullptr;
    // the warp tier, planned for the largest seed set among the requests it serves
    uint32_t cutoff = 0;
    uint32_t warp_ns = 0;
    bool warp_ok = false;
    TierCfg wcfg{};
    uint32_t warp_blocks = 0;
    uint64_t warp_smem = 0;
    uint32_t step = 0;
    // GPU time each size class has had (milliseconds of its steps) and which classes were busy
    double class_ms[kBatchClasses] = {};
    bool class_was_busy[kBatchClasses] = {};

    int choose_class(const std::vector<Req*>& active);
    void run();
    int grow_plans(const std::vector<Req*>& active);
    void finish(Req* r, int status);
    void fail_all(int status, const char* msg);
};

namespace {

#define SRV_CUDA(call)                                                                   \
    do {                                                                                 \
        const cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                         \
            cudaGetLastError();                                                          \
            char m_[200];                                                                \
            std::snprintf(m_, sizeof(m_), "%s: %s", #call, cudaGetErrorString(e_));     \
            fail_all(e_ == cudaErrorMemoryAllocation ? IMIN_ERR_NOMEM : IMIN_ERR_CUDA, m_); \
            return;                                                                      \
        }                                                                                \
    } while (0)

DevGraph dev_graph_of(const imin_graph* g) { return dev_graph(g); }

}  // namespace

void imin_server::finish(Req* r, int status)
{
    r->status = status;
    r->done = true;
    r->t_done = Clock::now();
    if (r->mem != nullptr) {
        cudaFreeAsync(r->mem, s);
        r->mem = nullptr;
    }
    if (r->slot >= 0) {
        slots[r->slot] = nullptr;
        r->slot = -1;
    }
    used -= r->bytes;
    r->bytes = 0;
    st.completed += 1;
}

void imin_server::fail_all(int status, const char* msg)
{
    std::lock_guard<std::mutex> lk(mu);
    fatal = status;
    std::snprintf(fatal_msg, sizeof(fatal_msg), "%s", msg);
    for (Req* r : slots)
        if (r != nullptr) finish(r, status);
    for (Req* r : pending) {
        r->status = status;
        r->done = true;
        r->t_done = Clock::now();
    }
    pending.clear();
    cv_done.notify_all();
}

int imin_server::grow_plans(const std::vector<Req*>& active)
{
    // size classes: re-plan a class when a larger graph joins it
    for (Req* r : active) {
        const int k = batch_class(r->g->n);
        if (r->g->n <= cls_n[k] && r->g->m <= cls_m[k]) continue;
        cls_n[k] = std::max(cls_n[k], r->g->n);
        cls_m[k] = std::max(cls_m[k], r->g->m);
        uint64_t bytes = 0;
        if (!plan_batch_cta(dev, cls_n[k], cls_m[k], &cfg[k], &cta_blocks[k], &cta_smem[k], &bytes))
            return IMIN_ERR_INTERNAL;
        if (cta_scratch[k]) cudaFreeAsync(cta_scratch[k], s);
        if (cudaMallocAsync(&cta_scratch[k], bytes, s) != cudaSuccess) return IMIN_ERR_NOMEM;
        if (prepare_cta_scratch(cfg[k], cta_blocks[k], cta_scratch[k], s) != cudaSuccess) return IMIN_ERR_CUDA;
    }
    bool regrow = false;
    for (Req* r : active) {
        if (r->g->n > whole_n || r->g->m > whole_m || r->seeds.size() > whole_ns) {
            whole_n = std::max(whole_n, r->g->n);
            whole_m = std::max(whole_m, r->g->m);
            whole_ns = std::max<uint32_t>(whole_ns, static_cast<uint32_t>(r->seeds.size()));
            regrow = true;
        }
    }
    uint32_t ns_w = warp_ns, c_w = cutoff;
    for (Req* r : active) {
        if (!r->warp) continue;
        ns_w = std::max<uint32_t>(ns_w, static_cast<uint32_t>(r->seeds.size()));
        c_w = std::max(c_w, r->cutoff);
    }
    if (ns_w > warp_ns || c_w > cutoff) {
        warp_ns = ns_w;
        cutoff = c_w;
        warp_ok = plan_batch_warp(dev, warp_ns, cutoff, &wcfg, &warp_blocks, &warp_smem);
    }
    if (regrow) {
        whole = plan_tiers(dev, whole_n, whole_m, whole_ns, 0);
        if (whole_scratch) cudaFreeAsync(whole_scratch, s);
        const uint64_t bytes = whole.scratch_bytes[kTierWhole];
        if (cudaMallocAsync(&whole_scratch, bytes, s) != cudaSuccess) return IMIN_ERR_NOMEM;
        if (cudaMemsetAsync(whole_scratch, 0xFF, bytes, s) != cudaSuccess) return IMIN_ERR_CUDA;
    }
    return IMIN_OK;
}

int imin_server::choose_class(const std::vector<Req*>& active)
{
    bool busy[kBatchClasses] = {};
    for (Req* r : active) busy[batch_class(r->g->n)] = true;
    double floor_ms = -1.0;
    for (int k = 0; k < kBatchClasses; ++k)
        if (busy[k] && class_was_busy[k] && (floor_ms < 0 || class_ms[k] < floor_ms)) floor_ms = class_ms[k];
    int best = -1;
    for (int k = 0; k < kBatchClasses; ++k) {
        if (busy[k] && !class_was_busy[k] && floor_ms >= 0) class_ms[k] = std::max(class_ms[k], floor_ms);
        class_was_busy[k] = busy[k];
        if (busy[k] && (best < 0 || class_ms[k] < class_ms[best])) best = k;
    }
    return best;
}

void imin_server::run()
{
    cudaSetDevice(device);
    std::vector<Req*> admitted;
    for (;;) {
        admitted.clear();
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                // admission: arrival order within a size class, while a slot is free, the state
                // fits the budget and the class's samples per step stay under the cap (a class
                // at its cap is passed over, not waited for)
                uint64_t class_samples[kBatchClasses] = {};
                Req* waiting[kBatchClasses] = {};  // the oldest pending request of the class that did not fit
                for (Req* r : slots)
                    if (r != nullptr) class_samples[batch_class(r->g->n)] += r->theta;
                for (auto it = pending.begin(); it != pending.end();) {
                    Req* r = *it;
                    const int k = batch_class(r->g->n);
                    // later requests of a class that fit under its cap may pass one that does not,
                    // kMaxOvertakes of them at most; then the class waits for it
                    const bool held = waiting[k] != nullptr && waiting[k]->overtaken >= kMaxOvertakes;
                    if (held || (class_samples[k] > 0 && class_samples[k] + r->theta > class_cap)) {
                        if (waiting[k] == nullptr) waiting[k] = r;
                        ++it;
                        continue;
                    }
                    int free_slot = -1;
                    for (int i = 0; i < max_active; ++i)
                        if (slots[i] == nullptr) {
                            free_slot = i;
                            break;
                        }
                    if (free_slot < 0 || (used + r->bytes > budget && used > 0)) break;
                    it = pending.erase(it);
                    r->slot = free_slot;
                    slots[free_slot] = r;
                    used += r->bytes;
                    class_samples[k] += r->theta;
                    if (waiting[k] != nullptr) waiting[k]->overtaken += 1;
                    admitted.push_back(r);
                    st.admitted += 1;
                }
                bool any = !admitted.empty();
                for (Req* r : slots) any = any || r != nullptr;
                if (any) break;
                if (stop) return;
                cv_work.wait(lk);
            }
        }

        // set up the newly admitted requests; each takes its graph's tuned warp/block cutoff
        // (tuned on this stream the first time a graph and seed-set size class is seen)
        bool need_cb = false;
        for (Req* r : admitted) {
            if (r->warp) {
                const int rc = tuned_cutoff(r->g, r->seeds, r->key, r->theta, s, &r->cutoff);
                if (rc != IMIN_OK) {
                    fail_all(rc, "warp/block cutoff tuning failed");
                    return;
                }
                r->warp = r->cutoff > 0;
            }
            SRV_CUDA(cudaMallocAsync(&r->mem, r->bytes, s));
            SRV_CUDA(cudaMemsetAsync(r->mem, 0, r->bytes, s));
            SRV_CUDA(cudaMemcpyAsync(r->mem + r->off_seeds, r->seeds.data(), 4ull * r->seeds.size(),
                                     cudaMemcpyHostToDevice, s));
            int32_t* dseeds = reinterpret_cast<int32_t*>(r->mem + r->off_seeds);
            uint32_t* excl = reinterpret_cast<uint32_t*>(r->mem + r->off_excl);
            SRV_CUDA(launch_build_excl(excl, dseeds, static_cast<int32_t>(r->seeds.size()), s));
            SRV_CUDA(cudaMemsetAsync(dflags + 2 * r->slot, 0, 2 * sizeof(int32_t), s));
            if (r->driver == kGR) {
                SRV_CUDA(cudaMemsetAsync(dcb_count + r->slot, 0, sizeof(uint32_t), s));
                SRV_CUDA(launch_build_cb(dev_graph_of(r->g), dseeds, static_cast<int32_t>(r->seeds.size()), excl,
                                         reinterpret_cast<uint32_t*>(r->mem + r->off_cb), dcb_count + r->slot, s));
                need_cb = true;
            }
        }
        if (need_cb) {
            SRV_CUDA(cudaMemcpyAsync(hcb, dcb_count, sizeof(uint32_t) * max_active, cudaMemcpyDeviceToHost, s));
            SRV_CUDA(cudaStreamSynchronize(s));
        }
        std::vector<Req*> finished_now;
        for (Req* r : admitted) {
            r->start = step;
            r->count = r->driver == kGR ? std::min<int32_t>(r->b, static_cast<int32_t>(hcb[r->slot]))
                                        : std::min<int32_t>(r->b, r->g->n - static_cast<int32_t>(r->seeds.size()));
            if (r->count <= 0) finished_now.push_back(r);
        }

        // the active set, the class this step serves, and the descriptors (a request of another
        // class is uploaded with a start beyond this step, which the kernels treat as inactive)
        std::vector<Req*> active;
        for (Req* r : slots)
            if (r != nullptr && r->count > 0) active.push_back(r);
        const int serve = choose_class(active);
        auto served = [serve](const Req* r) { return batch_class(r->g->n) == serve; };
        {
            const int rc = grow_plans(active);
            if (rc != IMIN_OK) {
                fail_all(rc, "the batched kernels cannot be configured for the admitted graphs");
                return;
            }
        }
        uint64_t sum_theta = 0;
        std::memset(hq, 0, sizeof(BatchQuery) * max_active);
        for (Req* r : active) {
            BatchQuery& d = hq[r->slot];
            d.g = dev_graph_of(r->g);
            d.seeds = reinterpret_cast<int32_t*>(r->mem + r->off_seeds);
            d.ns = static_cast<uint32_t>(r->seeds.size());
            d.excl = reinterpret_cast<uint32_t*>(r->mem + r->off_excl);
            d.cb = r->driver == kGR ? reinterpret_cast<uint32_t*>(r->mem + r->off_cb) : nullptr;
            d.key_lo = static_cast<uint32_t>(r->key);
            d.key_hi = static_cast<uint32_t>(r->key >> 32);
            d.theta = r->theta;
            d.delta = reinterpret_cast<unsigned long long*>(r->mem + r->off_delta);
            d.blockers = reinterpret_cast<int32_t*>(r->mem + r->off_blk);
            d.count = r->count;
            d.flags = dflags + 2 * r->slot;
            d.start = served(r) ? r->start : step + 1;
            d.gr = r->driver == kGR ? 1 : 0;
            d.done = r->warp && warp_ok ? r->mem + r->off_done : nullptr;
            if (served(r)) sum_theta += r->theta;
        }
        if (sum_theta > over_cap) {
            if (dover) cudaFreeAsync(dover, s);
            over_cap = sum_theta;
            SRV_CUDA(cudaMallocAsync(&dover, sizeof(uint2) * over_cap, s));
        }
        // one mixed schedule per slot: AdvancedGreedy is active for rounds < count, GreedyReplace
        // for rounds < 2*count until its stop flag (checked on the device)
        // item prefixes: one row per size class, then the warp tier's row
        const uint32_t chunk = 16;
        const size_t stride = static_cast<size_t>(max_active) + 1;
        bool class_busy[kPrefixRows] = {};
        for (int k = 0; k < kPrefixRows; ++k) {
            unsigned long long* pr = hprefix + k * stride;
            pr[0] = 0;
            for (int i = 0; i < max_active; ++i) {
                const Req* r = slots[i];
                const bool in_row = r != nullptr && (k < kBatchClasses ? batch_class(r->g->n) == k
                                                                        : r->warp && warp_ok);
                const bool act = in_row && r->count > 0 && served(r);
                pr[i + 1] = pr[i] + (act ? (r->theta + chunk - 1) / chunk : 0);
            }
            class_busy[k] = pr[max_active] > 0;
        }
        bool any_gr = false;
        for (Req* r : active) any_gr = any_gr || r->driver == kGR;
        if (!active.empty()) {
            SRV_CUDA(cudaMemcpyAsync(dq, hq, sizeof(BatchQuery) * max_active, cudaMemcpyHostToDevice, s));
            SRV_CUDA(cudaMemcpyAsync(dprefix, hprefix, sizeof(unsigned long long) * kPrefixRows * stride,
                                     cudaMemcpyHostToDevice, s));
            const Clock::time_point t_step = Clock::now();
            SRV_CUDA(cudaMemsetAsync(dctl, 0, sizeof(BatchCtl), s));
            BatchStep B{};
            B.q = dq;
            B.nq = static_cast<uint32_t>(max_active);
            B.chunk = chunk;
            B.step = step;
            B.ctl = dctl;
            B.over = dover;
            B.over_cap = static_cast<uint32_t>(std::min<uint64_t>(over_cap, 0xFFFFFFFFull));
            B.stats = nullptr;
            B.prefix = dprefix;
            B.all_ic = 1;
            for (Req* r : active)
                if (served(r)) B.all_ic = B.all_ic && r->g->model == 0 ? 1u : 0u;
            // every slot follows its own driver's schedule (BatchQuery::gr)
            if (any_gr) SRV_CUDA(launch_batch_unblock(B, s));
            if (class_busy[kBatchClasses]) {
                BatchStep Bw = B;
                Bw.prefix = dprefix + kBatchClasses * stride;
                SRV_CUDA(launch_batch_warp(Bw, wcfg, warp_blocks, warp_smem, s));
            }
            for (int k = 0; k < kBatchClasses; ++k) {
                if (!class_busy[k]) continue;
                BatchStep Bk = B;
                Bk.cls = static_cast<uint32_t>(k);
                Bk.prefix = dprefix + k * stride;
                SRV_CUDA(launch_batch_cta(Bk, cfg[k], cta_blocks[k], cta_smem[k], cta_scratch[k], s));
            }
            SRV_CUDA(launch_batch_whole(B, whole.cfg[kTierWhole], whole.blocks[kTierWhole], whole_scratch, s));
            SRV_CUDA(launch_batch_select(B, s));
            SRV_CUDA(cudaMemcpyAsync(hctl, dctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
            SRV_CUDA(cudaMemcpyAsync(hflags, dflags, sizeof(int32_t) * 2 * max_active, cudaMemcpyDeviceToHost, s));
            SRV_CUDA(cudaStreamSynchronize(s));
            if (hctl->error != 0) {
                fail_all(hctl->error & kErrInternal ? IMIN_ERR_INTERNAL : IMIN_ERR_CAPACITY,
                         "a batched step reported a kernel error");
                return;
            }
            class_ms[serve] += std::chrono::duration<double, std::milli>(Clock::now() - t_step).count();
            for (Req* r : active) {
                if (!served(r)) {
                    r->start += 1;  // sat this step out: its next round is still step + 1 - start
                    continue;
                }
                const int32_t rr = static_cast<int32_t>(step - r->start);
                const bool last = r->driver == kAG ? rr + 1 >= r->count
                                                   : (hflags[2 * r->slot] != 0 || rr + 1 >= 2 * r->count);
                if (last) finished_now.push_back(r);
                st.samples += r->theta;
            }
            st.steps += 1;
            ++step;
        }

        // retire finished requests
        if (!finished_now.empty()) {
            std::vector<std::vector<int32_t>> res(finished_now.size());
            for (size_t i = 0; i < finished_now.size(); ++i) {
                Req* r = finished_now[i];
                res[i].resize(static_cast<size_t>(std::max(r->count, 0)));
                if (r->count > 0)
                    SRV_CUDA(cudaMemcpyAsync(res[i].data(), r->mem + r->off_blk, 4ull * r->count,
                                             cudaMemcpyDeviceToHost, s));
            }
            SRV_CUDA(cudaStreamSynchronize(s));
            std::lock_guard<std::mutex> lk(mu);
            for (size_t i = 0; i < finished_now.size(); ++i) {
                finished_now[i]->result.swap(res[i]);
                finish(finished_now[i], IMIN_OK);
            }
            cv_done.notify_all();
        }
    }
}

extern "C" {

int imin_server_create(const imin_server_config* cfg, imin_server** out)
{
    fail_msg(IMIN_OK, "");
    if (out == nullptr) return fail_msg(IMIN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    imin_server* srv = new imin_server();
    cudaGetDevice(&srv->device);
    srv->dev = device_info();
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    srv->budget = (cfg && cfg->memory_budget) ? cfg->memory_budget : static_cast<uint64_t>(free_b / 4);
    srv->max_active = (cfg && cfg->max_active > 0) ? cfg->max_active : 256;
    srv->class_cap = (cfg && cfg->max_class_samples > 0) ? static_cast<uint64_t>(cfg->max_class_samples) : 200000u;
    srv->cutoff = 0;
    srv->slots.assign(srv->max_active, nullptr);
    const size_t stride = static_cast<size_t>(srv->max_active) + 1;
    cudaError_t e = cudaStreamCreateWithFlags(&srv->s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&srv->dq, sizeof(BatchQuery) * srv->max_active);
    if (e == cudaSuccess) e = cudaMalloc(&srv->dflags, sizeof(int32_t) * 2 * srv->max_active);
    if (e == cudaSuccess) e = cudaMalloc(&srv->dprefix, sizeof(unsigned long long) * kPrefixRows * stride);
    if (e == cudaSuccess) e = cudaMalloc(&srv->dctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMalloc(&srv->dcb_count, sizeof(uint32_t) * srv->max_active);
    if (e == cudaSuccess) e = cudaMallocHost(&srv->hq, sizeof(BatchQuery) * srv->max_active);
    if (e == cudaSuccess) e = cudaMallocHost(&srv->hprefix, sizeof(unsigned long long) * kPrefixRows * stride);
    if (e == cudaSuccess) e = cudaMallocHost(&srv->hflags, sizeof(int32_t) * 2 * srv->max_active);
    if (e == cudaSuccess) e = cudaMallocHost(&srv->hctl, sizeof(BatchCtl));
    if (e == cudaSuccess) e = cudaMallocHost(&srv->hcb, sizeof(uint32_t) * srv->max_active);
    if (e != cudaSuccess) {
        cudaGetLastError();
        imin_server_destroy(srv);
        return fail_msg(IMIN_ERR_NOMEM, "imin_server_create: device or pinned memory allocation failed");
    }
    srv->worker = std::thread([srv] { srv->run(); });
    *out = srv;
    return IMIN_OK;
}

int imin_server_submit(imin_server* srv, int32_t driver, const imin_graph* g, const int32_t* seeds,
                       int32_t n_seeds, int32_t b, uint32_t theta, uint64_t key, uint64_t* ticket)
{
    fail_msg(IMIN_OK, "");
    if (srv == nullptr || g == nullptr || ticket == nullptr)
        return fail_msg(IMIN_ERR_INVALID, "server, graph and ticket must be non-NULL");
    if (driver != kAG && driver != kGR) return fail_msg(IMIN_ERR_INVALID, "driver must be 0 (AG) or 1 (GR)");
    if (n_seeds < 1 || n_seeds > g->n || seeds == nullptr) return fail_msg(IMIN_ERR_INVALID, "n_seeds must be in [1, n]");
    if (b < 0 || theta < 1) return fail_msg(IMIN_ERR_INVALID, "b must be >= 0 and theta >= 1");
    if (g->device != srv->device) return fail_msg(IMIN_ERR_INVALID, "graph lives on another device");
    Req* r = new Req();
    r->driver = driver;
    r->g = g;
    r->b = b;
    r->theta = theta;
    r->key = key;
    r->seeds.resize(static_cast<size_t>(n_seeds));
    cudaPointerAttributes a;
    const bool dev_ptr = cudaPointerGetAttributes(&a, seeds) == cudaSuccess &&
                         (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev_ptr) {
        if (cudaMemcpy(r->seeds.data(), seeds, 4ull * n_seeds, cudaMemcpyDeviceToHost) != cudaSuccess) {
            delete r;
            return fail_msg(IMIN_ERR_CUDA, "copying the seeds failed");
        }
    } else {
        std::memcpy(r->seeds.data(), seeds, 4ull * n_seeds);
    }
    std::vector<uint8_t> mark(static_cast<size_t>(g->n), 0);
    for (int32_t v : r->seeds) {
        if (v < 0 || v >= g->n || mark[v]) {
            delete r;
            return fail_msg(IMIN_ERR_INVALID, "seeds: out of range or duplicate");
        }
        mark[v] = 1;
    }
    plan_request(*r, 1);  // room for the warp tier's done flags; admission decides whether it runs
    if (r->bytes > srv->budget) {
        delete r;
        return fail_msg(IMIN_ERR_NOMEM, "the request's device state exceeds the server's memory budget");
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->fatal != IMIN_OK) {
            delete r;
            return fail_msg(srv->fatal, srv->fatal_msg);
        }
        r->ticket = srv->next_ticket++;
        srv->reqs[r->ticket] = r;
        srv->pending.push_back(r);
        srv->st.submitted += 1;
        *ticket = r->ticket;
    }
    srv->cv_work.notify_one();
    return IMIN_OK;
}

int imin_server_wait(imin_server* srv, uint64_t ticket, int64_t timeout_ms, int32_t* out_blockers,
                     int32_t capacity, int32_t* out_count, double* latency_ms)
{
    fail_msg(IMIN_OK, "");
    if (srv == nullptr) return fail_msg(IMIN_ERR_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return fail_msg(IMIN_ERR_INVALID, "unknown or already collected ticket");
    Req* r = it->second;
    auto ready = [r] { return r->done; };
    if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail_msg(IMIN_ERR_TIMEOUT, "the request has not finished yet");
    const int status = r->status;
    if (status == IMIN_OK) {
        const int32_t cnt = static_cast<int32_t>(r->result.size());
        if (cnt > 0 && (out_blockers == nullptr || capacity < cnt)) return fail_msg(IMIN_ERR_INVALID, "out_blockers too small");
        if (cnt > 0) std::memcpy(out_blockers, r->result.data(), 4ull * cnt);
        if (out_count) *out_count = cnt;
        if (latency_ms)
            *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    }
    srv->reqs.erase(it);
    delete r;
    if (status != IMIN_OK) return fail_msg(status, srv->fatal_msg[0] ? srv->fatal_msg : "the request failed");
    return IMIN_OK;
}

int imin_server_get_stats(imin_server* srv, imin_server_stats* out)
{
    if (srv == nullptr || out == nullptr) return fail_msg(IMIN_ERR_INVALID, "server and out must be non-NULL");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->st;
    out->memory_in_use = srv->used;
    out->pending = srv->pending.size();
    return IMIN_OK;
}

int imin_server_destroy(imin_server* srv)
{
    if (srv == nullptr) return IMIN_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();  // finishes admitted and pending work first
    for (auto& kv : srv->reqs) delete kv.second;
    if (srv->s) cudaStreamSynchronize(srv->s);
    for (int k = 0; k < kBatchClasses; ++k) cudaFree(srv->cta_scratch[k]);
    cudaFree(srv->whole_scratch);
    cudaFree(srv->dover);
    cudaFree(srv->dq);
    cudaFree(srv->dflags);
    cudaFree(srv->dprefix);
    cudaFree(srv->dctl);
    cudaFree(srv->dcb_count);
    cudaFreeHost(srv->hq);
    cudaFreeHost(srv->hprefix);
    cudaFreeHost(srv->hflags);
    cudaFreeHost(srv->hctl);
    cudaFreeHost(srv->hcb);
    if (srv->s) cudaStreamDestroy(srv->s);
    delete srv;
    return IMIN_OK;
}

}  // extern "C"
