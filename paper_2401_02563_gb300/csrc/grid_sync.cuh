// Device synchronisation helpers shared by the persistent kernels: acquire/release accesses
// and a bounded grid-wide barrier for cooperative launches.
#pragma once
#include <cuda_runtime.h>

namespace kairos {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (all blocks resident) on the counters of C
// (fields bar_count, bar_gen, err).  Every wait is bounded: past `limit` polls the block
// records `timeout_code` in C->err and leaves.  Returns true when the launch may go on (no
// error recorded anywhere).
template <typename Ctr>
__device__ __forceinline__ bool grid_sync(Ctr *c, int *s_flag, unsigned long long limit, int timeout_code) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(&c->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (ld_acquire(&c->bar_gen) == gen) {
                if (++spins > limit) {
                    atomicCAS(&c->err, 0, timeout_code);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        *s_flag = __ldcg(&c->err);
    }
    __syncthreads();
    return *s_flag == 0;
}

}  // namespace kairos
