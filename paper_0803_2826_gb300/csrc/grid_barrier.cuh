// grid_barrier.cuh -- bounded barrier over all blocks of a cooperative launch.
//
// bar[0] counts arrivals, bar[1] is the generation, bar[2] the abort flag.
// The last block to arrive resets the count and advances the generation; the
// others poll the generation at most `spin_limit` times (with a short sleep),
// then set LB_DERR_BARRIER in *err and the abort flag and leave.  Every block
// sees the abort flag after the barrier, so all of them return instead of
// waiting on a block that will never arrive.  Returns false when the caller
// must stop.
#pragma once

#include "lbfluct.h"

namespace lbi {

__device__ __forceinline__ bool grid_barrier(unsigned int *bar, unsigned int *err, unsigned int spin_limit)
{
    __shared__ int stop;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vbar = bar;
        const unsigned int gen = vbar[1];
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar[0], 1u) + 1u;
        if (arrived == gridDim.x * gridDim.y * gridDim.z) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            unsigned int spins = 0;
            while (vbar[1] == gen && vbar[2] == 0u) {
                if (++spins > spin_limit) {
                    atomicOr(err, LB_DERR_BARRIER);
                    atomicExch(&bar[2], 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        stop = vbar[2] != 0u;
    }
    __syncthreads();
    return !stop;
}

}  // namespace lbi
