// select.cu -- blocker selection for the greedy drivers (Alg. 3 lines "x <- argmax", Alg. 4
// phases 1 and 2) and the small mask kernels around it.
//
// The argmax follows the paper's scan: candidates in ascending vertex id, x replaced only on a
// strictly larger counter, so among equal counters the smallest id wins. As a reduction this
// is the order (larger counter first, then smaller id), which is associative, so the grid can
// reduce in any order and still return the scan's answer.
#include "internal.h"
#include "select_dev.cuh"

namespace imin {

namespace {

using namespace sel;

constexpr int kSelBlocksPerSm = 2;

__global__ void __launch_bounds__(kSelThreads) k_select(SelectParams p)
{
    if (p.done != nullptr && *reinterpret_cast<const volatile int32_t*>(p.done) != 0) return;
    unsigned long long bd = 0;
    int32_t bi = kNone;  // (0, kNone) loses to every real candidate
    const int32_t stride = gridDim.x * blockDim.x;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
        const unsigned long long d = p.delta[v];
        if (d != 0) p.delta[v] = 0;  // counters restart from zero for the next call
        const uint32_t bit = 1u << (v & 31);
        const bool cand = p.cand != nullptr ? (p.cand[v >> 5] & bit) != 0 : (p.excl[v >> 5] & bit) == 0;
        if (cand && better(d, v, bd, bi)) {
            bd = d;
            bi = v;
        }
    }
    block_best<kSelThreads>(bd, bi);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        p.part_d[blockIdx.x] = bd;
        p.part_id[blockIdx.x] = bi;
        __threadfence();
        last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    bd = 0;
    bi = kNone;
    for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += blockDim.x) {
        const unsigned long long d = __ldcg(p.part_d + b);
        const int32_t i = __ldcg(p.part_id + b);
        if (better(d, i, bd, bi)) {
            bd = d;
            bi = i;
        }
    }
    block_best<kSelThreads>(bd, bi);
    if (threadIdx.x == 0) {
        *p.ticket = 0;
        if (bi != kNone) {
            p.blockers[p.pos] = bi;
            atomicOr(p.excl + (bi >> 5), 1u << (bi & 31));
            if (p.cand != nullptr) atomicAnd(p.cand + (bi >> 5), ~(1u << (bi & 31)));
            if (p.done != nullptr && p.cur != nullptr && *p.cur == bi) *p.done = 1;
        }
    }
}

// GreedyReplace phase 2, step "B <- B \ {u}": unblock the vertex at position pos.
__global__ void k_unblock(uint32_t* excl, const int32_t* blockers, int32_t pos, const int32_t* done,
                          int32_t* cur)
{
    if (*done != 0) return;
    const int32_t u = blockers[pos];
    *cur = u;
    atomicAnd(excl + (u >> 5), ~(1u << (u & 31)));
}

__global__ void k_build_excl(uint32_t* excl, const int32_t* ids, int32_t count)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const int32_t v = ids[i];
        atomicOr(excl + (v >> 5), 1u << (v & 31));
    }
}

// CB = N_out(S) \ S (Alg. 4 line 1 with merged seeds) as a bit mask, and its size.
__global__ void k_build_cb(DevGraph g, const int32_t* seeds, int32_t ns, const uint32_t* excl,
                           uint32_t* cb)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int s = warp; s < ns; s += nwarps) {
        const int32_t u = seeds[s];
        for (int32_t e = g.row_ptr[u] + lane; e < g.row_ptr[u + 1]; e += 32) {
            const int32_t v = g.col[e];
            if (((excl[v >> 5] >> (v & 31)) & 1u) == 0) atomicOr(cb + (v >> 5), 1u << (v & 31));
        }
    }
}

__global__ void k_popcount(const uint32_t* bits, int32_t words, uint32_t* out)
{
    uint32_t c = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
        c += __popc(bits[i]);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_down_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

int g_sms = 0;

}  // namespace

int select_blocks()
{
    if (g_sms == 0) g_sms = device_info().sms;
    return g_sms * kSelBlocksPerSm;
}

cudaError_t launch_select(const SelectParams& p, cudaStream_t s)
{
    k_select<<<select_blocks(), kSelThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_unblock(uint32_t* excl, const int32_t* blockers, int32_t pos, const int32_t* done,
                           int32_t* cur, cudaStream_t s)
{
    k_unblock<<<1, 1, 0, s>>>(excl, blockers, pos, done, cur);
    return cudaGetLastError();
}

cudaError_t launch_build_excl(uint32_t* excl, const int32_t* ids, int32_t count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int blocks = (count + 255) / 256;
    k_build_excl<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(excl, ids, count);
    return cudaGetLastError();
}

cudaError_t launch_build_cb(const DevGraph& g, const int32_t* seeds, int32_t ns,
                            const uint32_t* excl, uint32_t* cb, uint32_t* cb_count,
                            cudaStream_t s)
{
    const int blocks = (ns * 32 + 255) / 256;
    k_build_cb<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(g, seeds, ns, excl, cb);
    const int32_t words = (g.n + 31) / 32;
    const int pb = (words + 255) / 256;
    k_popcount<<<pb < 1024 ? pb : 1024, 256, 0, s>>>(cb, words, cb_count);
    return cudaGetLastError();
}

}  // namespace imin
