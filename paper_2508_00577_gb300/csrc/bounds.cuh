// Bounds-checked builds (compiled with -DEVLBM_BOUNDS_CHECK, library libevlbm_bc.so):
// every checked access compares its index with the extent of the array it touches.  An
// index out of range is counted in a device word of the translation unit and the
// access is skipped (a load returns 0); nothing traps, so a faulty index shows up as a
// count read on the host (lbm_bounds_violations) while the GPU stays usable.  Without
// the macro the checks compile to nothing.
#pragma once

#include <cuda_runtime.h>

namespace evlbm {

#ifdef EVLBM_BOUNDS_CHECK
static __device__ unsigned long long g_oob;

__device__ __forceinline__ bool in_bounds(unsigned long long i, unsigned long long n)
{
    if (i < n) return true;
    atomicAdd(&g_oob, 1ull);
    return false;
}

// Host reader of this translation unit's counter: >= 0 the count, -2 CUDA error.
#define EVLBM_DEFINE_OOB_READER(name)                                                   \
    long long name()                                                                    \
    {                                                                                   \
        unsigned long long v = 0;                                                       \
        if (cudaMemcpyFromSymbol(&v, evlbm::g_oob, sizeof(v)) != cudaSuccess) return -2; \
        return (long long)v;                                                            \
    }
#else
__device__ __forceinline__ constexpr bool in_bounds(unsigned long long, unsigned long long) { return true; }

#define EVLBM_DEFINE_OOB_READER(name) \
    long long name() { return -1; }
#endif

}  // namespace evlbm
