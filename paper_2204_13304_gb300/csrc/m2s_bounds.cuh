// Range checks of global-memory indices, compiled in by -DM2S_DEBUG_BOUNDS
// (the library variant that build.py makes with M2S_BUILD_VARIANT=bounds).
// A checked access tests its index against the extent it must stay in; a
// violation skips the access and counts it in this translation unit's error
// word, keeping the source line and index of the first one.  Nothing traps
// and nothing faults.  m2s_debug_bounds_read collects and clears the words.
// In the normal build every check is the constant true.
#pragma once
#include "m2s_internal.cuh"

namespace m2s {

#ifdef M2S_DEBUG_BOUNDS
namespace {
__device__ unsigned long long g_bounds[3];  // violations, first line, first index
}

__device__ __forceinline__ bool bounds_ok(long long i, long long n, int line) {
    if ((unsigned long long)i < (unsigned long long)n) return true;
    if (atomicAdd(&g_bounds[0], 1ULL) == 0ULL) {
        g_bounds[1] = (unsigned long long)line;
        g_bounds[2] = (unsigned long long)i;
    }
    return false;
}
#define M2S_IN(i, n) (::m2s::bounds_ok((long long)(i), (long long)(n), __LINE__))

// Host side: this translation unit's record into out[0..2] (violations,
// first line, first index), then cleared.
#define M2S_BOUNDS_READER(name)                                                              \
    cudaError_t name(long long* out) {                                                       \
        unsigned long long v[3];                                                             \
        cudaError_t e = cudaMemcpyFromSymbol(v, g_bounds, sizeof v);                         \
        if (e != cudaSuccess) return e;                                                      \
        for (int k = 0; k < 3; ++k) out[k] = (long long)v[k];                                \
        const unsigned long long z[3] = {0ULL, 0ULL, 0ULL};                                  \
        return cudaMemcpyToSymbol(g_bounds, z, sizeof z);                                    \
    }
#else
#define M2S_IN(i, n) true
#define M2S_BOUNDS_READER(name)                 \
    cudaError_t name(long long* out) {          \
        out[0] = -1;                            \
        out[1] = out[2] = 0;                    \
        return cudaSuccess;                     \
    }
#endif

}  // namespace m2s
