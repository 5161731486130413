// select_dev.cuh -- the order used by every blocker selection (Alg. 3/4 argmax): a larger
// counter wins, equal counters go to the smaller vertex id. This is exactly the outcome of the
// paper's scan (candidates in ascending id, x replaced only on a strictly larger counter), and
// as a comparison it is associative, so reductions in any order return the scan's answer.
#pragma once

#include "imin_dev.cuh"

namespace imin {
namespace sel {

constexpr int kSelThreads = 512;
constexpr int32_t kNone = 0x7FFFFFFF;  // (0, kNone) loses to every real candidate

__device__ __forceinline__ bool better(unsigned long long d1, int32_t i1, unsigned long long d2,
                                       int32_t i2)
{
    return d1 > d2 || (d1 == d2 && i1 < i2);
}

__device__ __forceinline__ void warp_best(unsigned long long& d, int32_t& id)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long od = __shfl_down_sync(kFull, d, o);
        const int32_t oi = __shfl_down_sync(kFull, id, o);
        if (better(od, oi, d, id)) {
            d = od;
            id = oi;
        }
    }
}

// Block-wide best of (d, id); result valid in thread 0.
template <int kThreads>
__device__ __forceinline__ void block_best(unsigned long long& d, int32_t& id)
{
    __shared__ unsigned long long sd[kThreads / 32];
    __shared__ int32_t si[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    warp_best(d, id);
    if (lane == 0) {
        sd[wid] = d;
        si[wid] = id;
    }
    __syncthreads();
    if (wid == 0) {
        d = lane < kThreads / 32 ? sd[lane] : 0ull;
        id = lane < kThreads / 32 ? si[lane] : kNone;
        warp_best(d, id);
    }
}

}  // namespace sel
}  // namespace imin
