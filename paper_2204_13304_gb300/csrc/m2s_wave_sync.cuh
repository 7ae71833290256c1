// Device-side synchronisation shared by the wavefront sweeps: bounded
// producer waits, progress publication and the ticketed unit loop with its
// self-resetting exit protocol (see k_wave.cu for the scheme).
#pragma once
#include <climits>

#include "m2s_internal.cuh"

namespace m2s {
namespace wave {

constexpr int BIAS = 1 << 20;
constexpr int DONE = INT_MAX;

// Wait until every producer of the unit has published at least `need`.
// Returns false if the sweep was aborted (timeout here or elsewhere).
__device__ __forceinline__ bool wait_producers(const int* flags, int4 pr, int need, int* cached,
                                               DevStatus* status, long long spin_ns) {
    const int lane = threadIdx.x & 31;
    int ok = 1, cache = 0;
    if (lane == 0) {
        unsigned long long t0 = 0;
        for (;;) {
            int m = INT_MAX;
            if (pr.x >= 0) m = min(m, ld_acquire_gpu(flags + pr.x));
            if (pr.y >= 0) m = min(m, ld_acquire_gpu(flags + pr.y));
            if (pr.z >= 0) m = min(m, ld_acquire_gpu(flags + pr.z));
            if (m >= need) { cache = m; break; }
            if (ld_relaxed_gpu(&status->abort)) { ok = 0; break; }
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            else if ((long long)(now - t0) > spin_ns) {
                atomicCAS(&status->err, 0, (int)M2S_ERR_TIMEOUT);
                atomicExch(&status->abort, 1);
                ok = 0;
                break;
            }
            __nanosleep(40);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    *cached = __shfl_sync(0xffffffffu, cache, 0);
    __syncwarp();
    return ok != 0;
}

__device__ __forceinline__ void publish(int* flag, int value) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) st_release_gpu(flag, value);
}

// Ticket loop and exit protocol shared by both stencils.
template <typename UnitFn>
__device__ __forceinline__ void run_units(int n_units, int* flags, int* ctrl, DevStatus* status,
                                          UnitFn fn, int stall_unit = -1) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&ctrl[0], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_units) break;
        int ab = 0;
        if (lane == 0) ab = ld_relaxed_gpu(&status->abort);
        ab = __shfl_sync(0xffffffffu, ab, 0);
        if (ab) continue;  // drain tickets quickly after an abort
        if (t == stall_unit) continue;
        fn(t);
    }
    __syncwarp();
    int last = 0;
    if (lane == 0) {
        __threadfence();
        last = (atomicAdd(&ctrl[1], 1) == (int)gridDim.x - 1);
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {
        __threadfence();
        for (int i = lane; i < n_units; i += 32) flags[i] = 0;
        __syncwarp();
        if (lane == 0) {
            ctrl[0] = 0;
            ctrl[1] = 0;
            status->abort = 0;
            __threadfence();
        }
    }
}

}  // namespace wave
}  // namespace m2s
