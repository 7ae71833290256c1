// Exact-order 27-point Gauss-Seidel sweep, CTA-pipelined wavefront.
//
// The method is the same as in k_wave.cu (paper Sec. 4.3.3 SymGS; Sec. 6.1
// SewTh): every point is updated in lexicographic order from the new values
// of its 13 lower neighbours and the precomputed old-neighbour sum Q, on the
// point hyperplane t = x + 2y + 4z with rows (u, v) = (y + z, z).  What
// changes is how the wavefront is mapped onto the GPU, after measuring a
// GB300: an L2 hit costs ~460 cycles, a GPU-scope release (membar) ~830
// cycles of stall, a shared-memory handoff between warps ~250 cycles, a
// global producer->consumer handoff ~1800 cycles, and FP64 instructions
// issue at one warp-instruction per ~64 cycles per SM sub-partition.
//
//  * Units are CTAs of W compute warps stacked in v (warp w owns K-1
//    computing planes plus one halo plane below them) and 32 lanes in u
//    (lanes 0-1 are halo rows).  Warps of a CTA hand rows to each other
//    through CTA-scope progress words in shared memory.
//  * One extra "service" warp per CTA publishes the compute warps' progress
//    to global memory (acquire at CTA scope, fence at GPU scope, store), so
//    the compute warps never stall on a GPU-scope membar.
//  * Q, b and halo rows are prefetched D steps ahead into a register ring
//    (the step loop is unrolled by D so the ring is statically indexed): no
//    memory latency sits on the per-step dependency chain; a consumer waits
//    for its producers to have published step t + D before prefetching it.
//  * The 13-neighbour sum is evaluated separably: each row keeps its row
//    3-sum H, the lane below passes H and S2 = H(u-1) + H(u), and the 3x3
//    plane sum G = S2(u-1) + H(u) flows to the plane above: 9 floating-point
//    operations per point.
// Halo rows written by other CTAs or warps are loaded with ld.global.cg
// (L2, coherent) after an acquire of the producer's progress word.
#include <algorithm>
#include <climits>
#include <vector>

#include "m2s_internal.cuh"
#include "m2s_wave_sync.cuh"

namespace m2s {

namespace {

using namespace wave;

template <typename T>
struct CtaArgs {
    int nx, ny, nz;
    i64 n, off;
    int rev;
    long long spin_ns;
    const T* Qin;
    T* Qout;
    const T* b;
    T* x;
    const int2* origin;  // (u0, v0) per CTA unit
    const int4* prod;    // left, below, below-left CTA units
    int n_units;
    int* flags;          // n_units * W progress words
    int* ctrl;
    DevStatus* status;
    double* rz;          // per-unit partials of b.x (W per unit) or NULL
    int stall_unit;
};

__device__ __forceinline__ int ld_acquire_cta_smem(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v)
                 : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta_smem(int* p, int v) {
    asm volatile("st.release.cta.shared::cta.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)),
                 "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_gpu(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Producers of one compute warp: up to three global words and one word of
// a sibling warp in shared memory.
struct Prods {
    const int* g[3];
    int ng;
    const int* s;  // shared-memory word or NULL
};

// Bounded wait until every producer word is >= need.  Returns the minimum
// seen (>= need) in *cached, or false if the sweep was aborted.
__device__ __forceinline__ bool wait_all(const Prods& pr, int need, int* cached,
                                         DevStatus* status, long long spin_ns) {
    const int lane = threadIdx.x & 31;
    int ok = 1, cache = 0;
    if (lane == 0) {
        unsigned long long t0 = 0;
        for (;;) {
            int m = INT_MAX;
            for (int i = 0; i < pr.ng; ++i) m = min(m, ld_acquire_gpu(pr.g[i]));
            if (pr.s) m = min(m, ld_acquire_cta_smem(pr.s));
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
            __nanosleep(32);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    *cached = __shfl_sync(0xffffffffu, cache, 0);
    __syncwarp();
    return ok != 0;
}

// Shared-memory staging of one compute warp (pitch 33 keeps the lane index
// conflict-free).  A = Q (computing rows) or x (halo rows), B = b.
template <typename T, int K, int CH>
struct WarpStage {
    T inA[2][K][CH][33];
    T inB[2][K - 1][CH][33];
    T outX[K - 1][CH][33];
    T outQ[K - 1][CH][33];
};

__device__ __forceinline__ void cp_async4(void* dst, const void* src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
}

template <typename T, int K, int W, int CH>
__device__ __forceinline__ void compute_warp(const CtaArgs<T>& a, int t, int w, int* sflag,
                                             WarpStage<T, K, CH>& sm) {
    constexpr int S_COMP = K - 1;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int2 org = a.origin[t];
    const int4 pu = a.prod[t];
    const int vbase = org.y + w * S_COMP - 1;  // plane of slot 0
    const int u0m2 = org.x - 2;                // u of lane 0
    const int tbase = 2 * u0m2 + 2 * vbase;
    const T inv26 = Lit<T>::inv26();
    const i64 dir = a.rev ? -1 : 1;

    Prods pr;
    pr.ng = 0;
    pr.s = nullptr;
    if (pu.x >= 0) pr.g[pr.ng++] = a.flags + pu.x * W + w;  // halo lanes
    if (w > 0) {
        pr.s = sflag + (w - 1);                                 // halo plane
        if (pu.x >= 0) pr.g[pr.ng++] = a.flags + pu.x * W + (w - 1);
    } else {
        if (pu.y >= 0) pr.g[pr.ng++] = a.flags + pu.y * W + (W - 1);
        if (pu.z >= 0) pr.g[pr.ng++] = a.flags + pu.z * W + (W - 1);
    }
    const bool has_prod = pr.ng > 0 || pr.s != nullptr;

    // row (r, j) of this warp: u = u0m2 + r, v = vbase + j; returns the
    // address of x = 0 (forward or reflected) or -1 if the row is outside.
    auto row_base = [&](int r, int j) -> i64 {
        const int v = vbase + j, y = u0m2 + r - v;
        if (v < 0 || v >= a.nz || y < 0 || y >= a.ny) return -1;
        const i64 rb = ((i64)v * a.ny + y) * a.nx;
        return a.rev ? a.off + a.n - 1 - rb : a.off + rb;
    };
    // own rows
    i64 base[K];
#pragma unroll
    for (int j = 0; j < K; ++j) base[j] = row_base(lane, j);
    const bool halo_lane = lane < 2;

    T xm1[K], xm2[K], h1[K], h2[K], s21[K], s22[K], g1[K];
#pragma unroll
    for (int j = 0; j < K; ++j) xm1[j] = xm2[j] = h1[j] = h2[j] = s21[j] = s22[j] = g1[j] = T(0);

    const int S = a.nx + 2 * 31 + 2 * (K - 1) + 1;  // steps until every row is done
    const int nchunks = (S + CH - 1) / CH;
    int cached = 0;
    // halo values of the next chunk travel through registers (.cg loads):
    // slot 0: 32 rows x CH (lane r = q % 32 ... one row per lane, CH values);
    // slots >= 1: rows 0-1 x CH values -> lanes 0..2*CH-1, one value each.
    T hv0[CH];
    T hv1[K];

    // Issue the loads of chunk c into buffer c & 1.  Returns false on abort.
    auto issue = [&](int c) -> bool {
        const int c0 = c * CH;
        if (c0 >= S) {
#pragma unroll
            for (int e = 0; e < CH; ++e) hv0[e] = T(0);
#pragma unroll
            for (int j = 0; j < K; ++j) hv1[j] = T(0);
            return true;
        }
        const int tneed = c0 + CH - 1 + tbase + BIAS;
        if (has_prod && tneed > cached) {
            if (!wait_all(pr, tneed, &cached, a.status, a.spin_ns)) return false;
        }
        const int bsel = c & 1;
        // computing rows: Q and b by cp.async (read-only in this launch)
#pragma unroll
        for (int j = 1; j < K; ++j) {
#pragma unroll
            for (int m = 0; m < CH; ++m) {
                const int q = lane + 32 * m;
                const int r = q / CH, e = q - (q / CH) * CH;
                const int xx = c0 + e - 2 * r - 2 * j;
                const i64 rbse = row_base(r, j);
                T* dA = &sm.inA[bsel][j][e][r];
                T* dB = &sm.inB[bsel][j - 1][e][r];
                if (r >= 2) {
                    if (rbse >= 0 && xx >= 0 && xx < a.nx) {
                        const i64 p = rbse + dir * xx;
                        cp_async4(dA, a.Qin + p, sizeof(T));
                        cp_async4(dB, a.b + p, sizeof(T));
                    } else {
                        *dA = T(0);
                        *dB = T(0);
                    }
                }
            }
        }
        // halo rows of slot 0: lane r loads its row's CH values
        {
            const i64 rbse = row_base(lane, 0);
#pragma unroll
            for (int e = 0; e < CH; ++e) {
                const int xx = c0 + e - 2 * lane;
                hv0[e] = (rbse >= 0 && xx >= 0 && xx < a.nx) ? __ldcg(a.x + rbse + dir * xx) : T(0);
            }
        }
        // halo rows 0-1 of slots >= 1: lane q < 2*CH loads (row q/CH, e = q%CH)
#pragma unroll
        for (int j = 1; j < K; ++j) {
            T v = T(0);
            if (lane < 2 * CH) {
                const int r = lane / CH, e = lane - (lane / CH) * CH;
                const int xx = c0 + e - 2 * r - 2 * j;
                const i64 rbse = row_base(r, j);
                if (rbse >= 0 && xx >= 0 && xx < a.nx) v = __ldcg(a.x + rbse + dir * xx);
            }
            hv1[j] = v;
        }
        return true;
    };
    // complete the loads of chunk c: land the halo registers, wait for the
    // asynchronous copies, make everything visible to the whole warp
    auto land = [&](int c) {
        const int bsel = c & 1;
#pragma unroll
        for (int e = 0; e < CH; ++e) sm.inA[bsel][0][e][lane] = hv0[e];
#pragma unroll
        for (int j = 1; j < K; ++j)
            if (lane < 2 * CH) sm.inA[bsel][j][lane - (lane / CH) * CH][lane / CH] = hv1[j];
        cp_async_commit_wait_all();
        __syncwarp();
    };
    // write chunk c's outputs (coalesced along each row) and publish it
    auto flush = [&](int c) {
        const int c0 = c * CH;
        __syncwarp();
#pragma unroll
        for (int j = 1; j < K; ++j) {
#pragma unroll
            for (int m = 0; m < CH; ++m) {
                const int q = lane + 32 * m;
                const int r = q / CH, e = q - (q / CH) * CH;
                if (r < 2) continue;
                const int xx = c0 + e - 2 * r - 2 * j;
                const i64 rbse = row_base(r, j);
                if (rbse >= 0 && xx >= 0 && xx < a.nx) {
                    const i64 p = rbse + dir * xx;
                    a.x[p] = sm.outX[j - 1][e][r];
                    if (a.Qout) a.Qout[p] = sm.outQ[j - 1][e][r];
                }
            }
        }
        __syncwarp();
        if (lane == 0) st_release_cta_smem(sflag + w, c0 + CH - 1 + tbase + BIAS);
    };

    bool ok = issue(0);
    if (ok) land(0);
    double rz = 0.0;
    for (int c = 0; ok && c < nchunks; ++c) {
        ok = issue(c + 1);
        if (!ok) break;
        const int bsel = c & 1;
#pragma unroll
        for (int e = 0; e < CH; ++e) {
            const int s = c * CH + e;
            T hu1[K], hu2[K], su2[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                hu1[j] = __shfl_up_sync(FULL, h1[j], 1);
                hu2[j] = __shfl_up_sync(FULL, h2[j], 1);
                su2[j] = (j < K - 1) ? __shfl_up_sync(FULL, s22[j], 1) : T(0);
            }
            T X[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int xx = s - 2 * lane - 2 * j;
                const bool in = base[j] >= 0 && xx >= 0 && xx < a.nx;
                const T va = sm.inA[bsel][j][e][lane];
                T v = T(0);
                if (j > 0 && !halo_lane) {
                    if (in) {
                        const T vb = sm.inB[bsel][j - 1][e][lane];
                        const T N = (xm1[j] + hu1[j]) + g1[j - 1];
                        v = (va + N) * inv26;
                        sm.outX[j - 1][e][lane] = v;
                        sm.outQ[j - 1][e][lane] = vb + N;
                        if (a.rz) rz = fma((double)vb, (double)v, rz);
                    }
                } else {
                    v = va;  // halo row (0 outside the grid)
                }
                X[j] = v;
            }
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const T H = (xm2[j] + xm1[j]) + X[j];
                xm2[j] = xm1[j];
                xm1[j] = X[j];
                h2[j] = h1[j];
                h1[j] = H;
                if (j < K - 1) {
                    const T S2 = hu2[j] + H;
                    const T G = su2[j] + H;
                    s22[j] = s21[j];
                    s21[j] = S2;
                    g1[j] = G;
                }
            }
        }
        flush(c);
        land(c + 1);
    }
    __syncwarp();
    if (lane == 0) st_release_cta_smem(sflag + w, ok ? DONE : DONE - 1);
    if (a.rz) {
        for (int o = 16; o > 0; o >>= 1) rz += __shfl_down_sync(FULL, rz, o);
        if (lane == 0) a.rz[(i64)t * W + w] = ok ? rz : 0.0;
    }
}

// Forwards the compute warps' CTA-scope progress to their global words.
template <int W>
__device__ __forceinline__ void service_warp(int* flags, int t, const int* sflag, DevStatus* status) {
    const int lane = threadIdx.x & 31;
    int last = 0;
    for (;;) {
        int v = DONE;
        if (lane < W) v = ld_acquire_cta_smem(sflag + lane);
        const int fresh = (lane < W && v != last) ? 1 : 0;
        if (__any_sync(0xffffffffu, fresh)) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            // DONE - 1 marks an aborted warp: nothing to forward
            if (fresh && v != DONE - 1) st_relaxed_gpu(flags + t * W + lane, v);
            last = v;
        }
        const int done = (lane < W) ? (v >= DONE - 1) : 1;
        if (__all_sync(0xffffffffu, done)) break;
        int ab = 0;
        if (lane == 0) ab = ld_relaxed_gpu(&status->abort);
        ab = __shfl_sync(0xffffffffu, ab, 0);
        if (ab) break;
        __nanosleep(64);
    }
}

template <typename T, int K, int W, int D>
__global__ void __launch_bounds__((W + 1) * 32, 1) gs27_cta_kernel(CtaArgs<T> a) {
    __shared__ int sflag[W];
    __shared__ int s_ticket;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    WarpStage<T, K, D>* stages = reinterpret_cast<WarpStage<T, K, D>*>(dyn_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&a.ctrl[0], 1);
        if (threadIdx.x < W) sflag[threadIdx.x] = 0;
        __syncthreads();
        const int t = s_ticket;
        if (t >= a.n_units) break;
        int ab = 0;
        if (threadIdx.x == 0) ab = ld_relaxed_gpu(&a.status->abort) || t == a.stall_unit;
        ab = __syncthreads_or(ab);
        if (!ab) {
            if (warp < W) compute_warp<T, K, W, D>(a, t, warp, sflag, stages[warp]);
            else service_warp<W>(a.flags, t, sflag, a.status);
        }
        __syncthreads();
    }
    // exit protocol: the last CTA out resets the counters for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int last = atomicAdd(&a.ctrl[1], 1) == (int)gridDim.x - 1;
        s_ticket = last;
    }
    __syncthreads();
    if (s_ticket) {
        __threadfence();
        for (int i = threadIdx.x; i < a.n_units * W; i += blockDim.x) a.flags[i] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            a.ctrl[0] = 0;
            a.ctrl[1] = 0;
            a.status->abort = 0;
            __threadfence();
        }
    }
    (void)lane;
}

}  // namespace

// Shapes of the CTA wavefront per element type: K register slots per lane
// (one halo plane + K-1 computed planes), W compute warps per CTA, and D the
// chunk length in steps (inputs are staged one chunk ahead, outputs flushed
// and published once per chunk).
template <typename T> struct CtaShape;
template <> struct CtaShape<double> { static constexpr int K = 2, W = 4, D = 4; };
template <> struct CtaShape<float> { static constexpr int K = 5, W = 4, D = 8; };

template <typename T>
size_t cta_smem_bytes() {
    return sizeof(WarpStage<T, CtaShape<T>::K, CtaShape<T>::D>) * CtaShape<T>::W;
}

template <typename T>
cudaError_t build_cta_units(Dims d, WaveUnits* out) {
    constexpr int K = CtaShape<T>::K, W = CtaShape<T>::W, D = CtaShape<T>::D;
    std::vector<int2> org;
    std::vector<int4> prod;
    // a CTA unit is 30 rows in u and W*(K-1) planes in v
    build_units_host(30, 1, 1, W * (K - 1) + 1, d, org, prod);
    WaveUnits u{};
    u.n_units = (int)org.size();
    u.K = K;
    u.stencil = 27;
    cudaError_t e;
    const size_t nu = std::max<size_t>(org.size(), 1);
    if ((e = cudaMalloc(&u.d_origin, nu * sizeof(int2))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&u.d_prod, nu * sizeof(int4))) != cudaSuccess) { free_wave_units(&u); return e; }
    if ((e = cudaMalloc(&u.d_flags, nu * W * sizeof(int))) != cudaSuccess) { free_wave_units(&u); return e; }
    if ((e = cudaMalloc(&u.d_ctrl, 2 * sizeof(int))) != cudaSuccess) { free_wave_units(&u); return e; }
    if (!org.empty() &&
        ((e = cudaMemcpy(u.d_origin, org.data(), org.size() * sizeof(int2), cudaMemcpyHostToDevice)) !=
             cudaSuccess ||
         (e = cudaMemcpy(u.d_prod, prod.data(), prod.size() * sizeof(int4), cudaMemcpyHostToDevice)) !=
             cudaSuccess)) {
        free_wave_units(&u);
        return e;
    }
    if ((e = cudaMemset(u.d_flags, 0, nu * W * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(u.d_ctrl, 0, 2 * sizeof(int))) != cudaSuccess) {
        free_wave_units(&u);
        return e;
    }
    int per_sm = 0;
    const size_t smem = cta_smem_bytes<T>();
    cudaFuncSetAttribute(gs27_cta_kernel<T, K, W, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs27_cta_kernel<T, K, W, D>, (W + 1) * 32,
                                                  smem);
    u.grid = wave_grid(u.n_units, per_sm);
    *out = u;
    return cudaGetLastError();
}

int cta_units_per_rz(int dtype_is_f64) { return dtype_is_f64 ? CtaShape<double>::W : CtaShape<float>::W; }

template <typename T>
cudaError_t launch_gs27_cta(const WaveUnits& u, const WaveCall& c, Dims d, const T* Qin, T* Qout,
                            const T* b, T* x, cudaStream_t st) {
    constexpr int K = CtaShape<T>::K, W = CtaShape<T>::W, D = CtaShape<T>::D;
    if (u.n_units == 0) return cudaSuccess;
    CtaArgs<T> a;
    a.nx = d.nx;
    a.ny = d.ny;
    a.nz = d.nz;
    a.n = d.n;
    a.off = d.off;
    a.rev = c.rev;
    a.spin_ns = c.spin_ns;
    a.Qin = Qin;
    a.Qout = Qout;
    a.b = b;
    a.x = x;
    a.origin = u.d_origin;
    a.prod = u.d_prod;
    a.n_units = u.n_units;
    a.flags = u.d_flags;
    a.ctrl = u.d_ctrl;
    a.status = c.status;
    a.rz = c.rz_partials;
    a.stall_unit = c.stall_unit;
    gs27_cta_kernel<T, K, W, D><<<u.grid, (W + 1) * 32, cta_smem_bytes<T>(), st>>>(a);
    return cudaGetLastError();
}

template cudaError_t build_cta_units<double>(Dims, WaveUnits*);
template cudaError_t build_cta_units<float>(Dims, WaveUnits*);
template cudaError_t launch_gs27_cta<double>(const WaveUnits&, const WaveCall&, Dims, const double*,
                                             double*, const double*, double*, cudaStream_t);
template cudaError_t launch_gs27_cta<float>(const WaveUnits&, const WaveCall&, Dims, const float*,
                                            float*, const float*, float*, cudaStream_t);

}  // namespace m2s
