// A grid-wide barrier for persistent cooperative launches, with a hook for the
// last block to arrive: it runs a short serial step (a fixed-order reduction
// of per-block partials, a row swap) while every other block waits, then
// releases them.  Arrival: a fence and an atomicAdd on bar[0]; release: a
// fence and a st.release of the barrier number b to bar[1]; waiting: polls of
// bar[1] by ld.acquire with a short sleep, bounded: after GS_SPIN_LIMIT polls
// the block sets DEV_TIMEOUT in the status word and the caller returns.  The
// two words are zeroed before the launch; b counts 1, 2, ... in every block,
// so bar[0] reaches b * gridDim.x.  Data written by other blocks before a
// barrier is read after it with ld.global.cg (L2), never from a possibly stale
// L1 line.  The caller passes two distinct shared flags to gs_arrive and
// gs_wait (a slow reader of one flag must not see the other's write).
#pragma once

#include "dme_internal.h"

namespace dme {

constexpr unsigned GS_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned gs_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void gs_st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Arrive at barrier b; true (in every thread of the block) for the last block.
__device__ __forceinline__ bool gs_arrive(unsigned* bar, unsigned b, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned old = atomicAdd(&bar[0], 1u);
        *s_flag = old == b * gridDim.x - 1;
    }
    __syncthreads();
    const bool last = *s_flag != 0;
    if (last) __threadfence();
    return last;
}

// The last block, after its serial step: release barrier b.
__device__ __forceinline__ void gs_release(unsigned* bar, unsigned b) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        gs_st_release(&bar[1], b);
    }
}

// Every other block: wait for the release of barrier b; false after a timeout.
__device__ __forceinline__ bool gs_wait(unsigned* bar, unsigned b, int* status, int* s_flag) {
    if (threadIdx.x == 0) {
        unsigned it = 0;
        int ok = 1;
        while (gs_ld_acquire(&bar[1]) < b) {
            if (++it > GS_SPIN_LIMIT) {
                atomicOr(status, DEV_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

}  // namespace dme
