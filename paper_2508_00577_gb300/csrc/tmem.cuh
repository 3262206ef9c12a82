// Tensor memory (TMEM) allocation for the lattice Boltzmann kernels.
//
// Blackwell gives every SM 256 KB of TMEM: 128 lanes x 512 columns of 32-bit words.  A
// warp reaches the 32 lanes of its quarter (warp index mod 4) with the 32x32b shape of
// tcgen05.ld / tcgen05.st: thread l of the warp reads or writes lane 32 (w mod 4) + l,
// so a thread owns one lane and keeps values in consecutive columns of it.  The D3Q27
// kernel (fused3d.cu) keeps there the populations a thread pulls in one stage of its
// pipeline and collides three planes later; no tensor-core instruction is issued.
//
// Allocation is per CTA, by one warp, in a power of two of columns (>= 32); the
// columns of all CTAs resident on an SM must fit in its 512, which the kernels ensure
// through their occupancy (registers or shared memory), so an allocation never waits.
#pragma once

#include <cstdint>

namespace evlbm {
namespace tmem {

// Allocates `cols` columns for the CTA (call from one whole warp); the base address is
// written to *slot (shared memory).  The caller publishes it with fence_sync().
__device__ __forceinline__ void alloc(uint32_t *slot, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(slot)), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// Frees the CTA's columns (one whole warp, after fence_sync() of all threads' accesses).
__device__ __forceinline__ void dealloc(uint32_t base, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols) : "memory");
}
// CTA barrier ordering TMEM allocation / accesses before it with those after it.
__device__ __forceinline__ void fence_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// TMEM address of column 0 of the lane quarter of warp `warp` (lane field in bits 16+).
__device__ __forceinline__ uint32_t lane_base(uint32_t base, int warp)
{
    return base + ((uint32_t)(32 * (warp & 3)) << 16);
}

}  // namespace tmem
}  // namespace evlbm
