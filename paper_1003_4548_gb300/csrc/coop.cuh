// coop.cuh -- grid-wide barrier of the cooperative solver kernels (elliptic
// relaxation and pressure projection).
#pragma once

#include "pdf_internal.cuh"

namespace coop {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace coop

// Grid-wide barrier of a cooperative launch: arrival by an acq_rel atomic on
// one counter (bar[0]); the last block resets it and bumps the generation
// word (bar[1]), the others poll that word with acquire loads (measured
// ~2.4 us on GB300 for 80-161 blocks). The wait is bounded by spin_max polls
// (SPIN_DEFAULT, about 1-2 s, unless the context sets a limit): on expiry the
// block sets ST_BARRIER in *status and proceeds.
constexpr long long SPIN_DEFAULT = 1ll << 22;

__device__ __forceinline__ void grid_barrier(unsigned* bar, int* status, long long spin_max) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* gen = bar + 1;
        unsigned* top = bar;
        const unsigned g0 = coop::ld_acquire(gen);
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        unsigned arrived;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(top) : "memory");
        if (arrived + 1u == gridDim.x) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(top) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
        } else {
            long long spins = 0;
            while (coop::ld_acquire(gen) == g0) {
                if (++spins > spin_max) {
                    set_status(status, ST_BARRIER);
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
}

// The same barrier for a kernel that tracks the generation word itself: gen
// holds, in thread 0, the generation the last barrier completed (read once at
// kernel start, before the first barrier, with coop_generation), so a
// barrier costs one atomic arrival and the polls, without a first read.
__device__ __forceinline__ unsigned coop_generation(const unsigned* bar) { return coop::ld_acquire(bar + 1); }

__device__ __forceinline__ void grid_barrier_gen(unsigned* bar, int* status, unsigned& gen, long long spin_max) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned* g = bar + 1;
        unsigned* top = bar;
        gen += 1u;  // the generation this barrier completes
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        unsigned arrived;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(top) : "memory");
        if (arrived + 1u == gridDim.x) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(top) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(g) : "memory");
        } else {
            long long spins = 0;
            while ((int)(coop::ld_acquire(g) - gen) < 0) {
                if (++spins > spin_max) {
                    set_status(status, ST_BARRIER);
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
    }
    __syncthreads();
}
