// grid_barrier.cuh -- bounded barrier over all blocks of a cooperative launch.
//
// bar[0] is the arrival word, bar[2] the abort flag (bar[1] is unused).  On
// each barrier block 0 adds 2^31 - (nblocks - 1) to bar[0] and every other
// block adds 1: together exactly 2^31, and every partial sum stays below
// 2^31, so the top bit of bar[0] flips at the last arrival and the low 31
// bits return to zero.  A block waits until the top bit differs from the one
// its own atomic returned: one atomic and the polling per barrier, no reset
// and no generation word.  The poll gives up after `spin_limit` rounds (with
// a short sleep each), sets LB_DERR_BARRIER in *err and the abort flag, which
// the other blocks check while they wait, so that all of them return instead
// of waiting on a block that will never arrive.  After a timeout the low bits
// are no longer zero: the owner resets bar[] to zero before the next launch.
// Returns false when the caller must stop.
#pragma once

#include "lbfluct.h"

namespace lbi {

// The barrier in two halves, for work that touches nothing another block
// reads before the barrier ends (it can then run while the other blocks
// arrive): grid_arrive publishes this block's writes and adds its arrival,
// grid_wait polls as above.  *ticket (block-shared) carries the arrival
// word's value from one half to the other.
__device__ __forceinline__ void grid_arrive(unsigned int *bar, unsigned int *ticket)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
        const bool first = (blockIdx.x | blockIdx.y | blockIdx.z) == 0;
        __threadfence();  // this block's writes before its arrival
        *ticket = atomicAdd(&bar[0], first ? 0x80000000u - (nb - 1u) : 1u);
    }
}

__device__ __forceinline__ bool grid_wait(unsigned int *bar, unsigned int *err, unsigned int spin_limit,
                                          const unsigned int *ticket)
{
    __shared__ int stop;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int old = *ticket;
        volatile unsigned int *vbar = bar;
        unsigned int spins = 0;
        int s = 0;
        while (((vbar[0] ^ old) & 0x80000000u) == 0u) {
            if (++spins > spin_limit) {
                atomicOr(err, LB_DERR_BARRIER);
                atomicExch(&bar[2], 1u);
                s = 1;
                break;
            }
            if ((spins & 63u) == 0u && vbar[2] != 0u) {  // another block gave up
                s = 1;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();  // the other blocks' writes after it
        stop = s;
    }
    __syncthreads();
    return !stop;
}

__device__ __forceinline__ bool grid_barrier(unsigned int *bar, unsigned int *err, unsigned int spin_limit)
{
    __shared__ unsigned int ticket;
    grid_arrive(bar, &ticket);
    return grid_wait(bar, err, spin_limit, &ticket);
}

}  // namespace lbi
