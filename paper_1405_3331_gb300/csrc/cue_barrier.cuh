// cue_barrier.cuh -- the bounded grid barrier of the cooperative kernels
// (the persistent coupled-step engine, the breadth-first search).
#pragma once

#include "cue_internal.h"

namespace cue {

// ---------------------------------------------------------------- grid barrier
// Ticket barrier: the 64-bit arrival counter only grows (it is zeroed per launch).
// A block's thread 0 takes a ticket with one acquire-release atomic (the
// release publishes the block's writes, which the preceding __syncthreads
// orders before it), and the barrier is passed once the counter reaches the
// next multiple of `expected`: the last arrival needs no second write, and
// the others poll with acquire loads, a bounded number of times.  Returns
// false when the launch is aborting.
__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long *p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(PBar *bar, unsigned expected, long long limit, unsigned *status)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int *vabort = &bar->abort;
        int ok = *vabort ? 0 : 1;
        if (ok) {
            const unsigned long long ticket = atom_add_acq_rel(&bar->count, 1ull);
            const unsigned long long target = (ticket / expected + 1ull) * expected;
            long long it = 0;
            while (ld_acquire(&bar->count) < target) {
                if (*vabort) {
                    ok = 0;
                    break;
                }
                if (++it > limit) {
                    flag_status(status, kStatusTimeout);
                    atomicExch(&bar->abort, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace cue
