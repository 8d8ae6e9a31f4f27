// Index checks of the bounds-checking build.
//
// Built with -DBGW_BOUNDS=1 (the libbgwchi_bounds.so variant), the kernels
// test every index they read from a device map (cube, inverse, gather and
// scatter maps of the FFT passes, the k + q map of the pair weights) against
// the range it must lie in.  An index out of range skips the access and sets
// bit `site` of a device status word; nothing traps or asserts.  Each
// translation unit has its own word (the library is built without
// relocatable device code); bgw_bounds_check reads and clears them all.
// In the default build the checks compile to nothing.
#pragma once
#include <cuda_runtime.h>

#ifndef BGW_BOUNDS
#define BGW_BOUNDS 0
#endif

namespace bgw {
enum BoundsSite {
    kBoundsCubeMap = 0,      // cube cell -> coefficient index (sphere -> grid, x lines)
    kBoundsInverseMap = 1,   // coefficient -> cube cell (one-kernel sphere -> grid)
    kBoundsGatherMap = 2,    // G -> kept-cube cell (matrix elements, gather)
    kBoundsScatterMap = 3,   // kept-cube cell -> G (matrix elements, scatter)
    kBoundsKMap = 4          // k -> grid index of k + q (pair weights)
};
}  // namespace bgw

#if BGW_BOUNDS
static __device__ unsigned int g_bgw_bounds_word;

__device__ __forceinline__ bool bgw_in_bounds(bool ok, int site) {
    if (!ok) atomicOr(&g_bgw_bounds_word, 1u << site);
    return ok;
}
#define BGW_IN_BOUNDS(cond, site) bgw_in_bounds((cond), (site))

// This translation unit's word, then cleared (waits for the device).
static inline cudaError_t bgw_bounds_take(unsigned *out) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_bgw_bounds_word, sizeof(unsigned));
    const unsigned zero = 0u;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bgw_bounds_word, &zero, sizeof(unsigned));
    return e;
}
#else
#define BGW_IN_BOUNDS(cond, site) true
static inline cudaError_t bgw_bounds_take(unsigned *out) {
    *out = 0u;
    return cudaSuccess;
}
#endif
