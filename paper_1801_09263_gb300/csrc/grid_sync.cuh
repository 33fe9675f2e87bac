// Grid-wide barrier with a time limit for persistent kernels launched
// cooperatively (all CTAs co-resident).
#pragma once

#include <cuda_runtime.h>

namespace lace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr unsigned long long kBarrierLimitNs = 2000000000ull;  // 2 s

// bar[0] counts arrivals, bar[1] is the generation, bar[2] the error flag
// (all zero at launch).  A CTA whose wait runs out sets the flag and returns
// false (the same for every thread of the CTA); it then leaves the kernel,
// so the other CTAs run out of time at their next barrier and leave too.
// gen is the caller's per-CTA generation count; limit_ns bounds one wait.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen, int* abort_sh,
                                             unsigned long long limit_ns = kBarrierLimitNs) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = gen + 1;
        int timed_out = 0;
        __threadfence();
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], target);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(&bar[1]) != target) {
                __nanosleep(32);
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(&bar[2], 1u);
                    timed_out = 1;
                    break;
                }
            }
        }
        __threadfence();
        gen = target;
        *abort_sh = timed_out;
    }
    __syncthreads();
    return !*abort_sh;
}

}  // namespace lace
