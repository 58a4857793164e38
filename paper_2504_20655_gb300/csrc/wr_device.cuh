// Device helpers shared by the kernels: coherent loads, cp.async staging,
// the bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wr_internal.h"

namespace wr {

constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

// Loads that bypass L1: rows and frontier stamps are written by other SMs
// between grid barriers, and L1 is not coherent across SMs.
__device__ __forceinline__ uint32_t ld_l2(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ int32_t ld_l2(const int32_t* p) { return __ldcg(p); }
__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
    return *reinterpret_cast<const volatile unsigned*>(p);
}

// 16-byte global -> shared copy through L2 only (cp.async.cg).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Grid-wide barrier for a co-resident (cooperative) grid.  The barrier's two
// words, count (low) and generation (high), are one 64-bit word: a block
// arrives with one atomic add, and the last arrival resets the count and
// advances the generation with a second one.  Every wait is bounded by
// max_spins iterations; on expiry it records WR_ETIMEOUT in *err and returns
// false, and every block then leaves the kernel.
__device__ __forceinline__ bool grid_sync(GridBar* bar, int* err, unsigned long long max_spins) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* word = reinterpret_cast<unsigned long long*>(bar);
        __threadfence();
        const unsigned long long old = atomicAdd(word, 1ull);
        const unsigned gen = static_cast<unsigned>(old >> 32);
        if (static_cast<unsigned>(old) == gridDim.x - 1) {
            atomicAdd(word, (1ull << 32) - gridDim.x);  // count back to 0, generation + 1
        } else {
            unsigned long long spins = 0;
            while (static_cast<unsigned>(*reinterpret_cast<volatile unsigned long long*>(word) >> 32) == gen) {
                if ((spins & 63) == 63 && ld_volatile(err) != 0) break;
                if (++spins > max_spins) {
                    atomicCAS(err, 0, WR_ETIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok = ld_volatile(err) == 0;  // one decision per block
    }
    __syncthreads();
    return ok != 0;
}

// Lane mask of the lanes below this one.
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace wr
