// 27-point (HPCG) SpMV y = A x and the fused CG step (p = z + beta p,
// q = A p, p.q) on plane tiles staged in shared memory by TMA.
//
// Operator (paper Sec. 7.1 HPCG; Sec. 4.3.1 SpMV): a_pp = 26, a_pq = -1 on
// the in-domain points of the 3x3x3 box, out-of-domain neighbours dropped.
// The box sum is evaluated separably, as in k_stencil27.cu: row 3-sums H,
// 3x3 plane sums S2, box = S2(z-1) + S2(z) + S2(z+1), y = 27 x_p - box.
//
// GB300 mapping.  A CTA of 4 warps owns a tile of 32 V points in x (V = 16
// bytes / element: one 16-byte vector per thread and row) by 32 rows in y and
// marches a chunk of z planes.  Each plane of the tile with a one-point halo
// (box 34 V x 34 rows, 544 B per row) is fetched by one
// cp.async.bulk.tensor.3d into a ring of shared-memory stages, NS planes
// ahead of the plane being computed, each stage completing on its mbarrier.
// The tensor map's zero fill of out-of-range coordinates is exactly the
// operator's dropped neighbours, so no boundary test guards a load.  A
// thread owns V x-points of 8 rows: it reads its 10 box rows (one 16-byte
// and two scalar shared loads each), forms H with a pair sum shared by its
// two inner points, S2 with a pair sum shared by two rows, and keeps the
// plane sums of the two previous planes and the centre values of the
// previous plane in registers.  FP64: 6.4 FP64 operations per point (7.5 in
// the plain separable form).  The grid is one wave: tiles x z-chunks sized
// to the SM count.
//
// Used where the rows are 16-byte aligned (nx * sizeof(T) a multiple of 16,
// vector bases aligned); otherwise the launchers fall back to st27_kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "m2s_internal.cuh"

namespace m2s {

namespace {

constexpr int kWarpsY = 4;              // warps per CTA
constexpr int kRows = 8;                // rows per thread
constexpr int kTileY = kWarpsY * kRows; // 32 rows per tile
constexpr int kBoxY = kTileY + 2;       // 34 box rows
constexpr int kThreads = 32 * kWarpsY;  // 128
constexpr long long kWaitNs = 2000000000LL;  // bound of every mbarrier wait

template <typename T> struct Vec;
template <> struct Vec<double> {
    static constexpr int V = 2;
    typedef double2 t;
};
template <> struct Vec<float> {
    static constexpr int V = 4;
    typedef float4 t;
};

template <typename T> constexpr int tile_x() { return 32 * Vec<T>::V; }       // 64 / 128
template <typename T> constexpr int box_x() { return 34 * Vec<T>::V; }        // 68 / 136
template <typename T> constexpr int stage_elems() { return box_x<T>() * kBoxY; }
template <typename T> constexpr unsigned stage_bytes() {
    return (unsigned)(stage_elems<T>() * sizeof(T));  // 18,496 B
}
// distance between the arrays of the stage ring: each TMA destination starts
// on a 128-byte boundary
template <typename T> constexpr int slot_elems() {
    return (int)(((stage_bytes<T>() + 127u) / 128u) * 128u / sizeof(T));
}

// CTAs resident per SM the grid is sized for (shared memory: SPMV 4 stages
// of one array, the fused CG step 3 stages of two arrays).
constexpr int kStagesSpmv = 4, kStagesPcg = 3;
constexpr int kCtasSpmv = 3, kCtasPcg = 2;

// ---------------------------------------------------------------------------
// mbarrier and TMA (PTX ISA: mbarrier, cp.async.bulk.tensor)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of `bar`: false once kWaitNs have passed.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((long long)(global_ns() - t0) > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map,
                                            unsigned long long* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <typename T>
struct TmaArgs {
    Dims d;
    int zc;              // planes per z-chunk
    T* y;                // y = A x (or q = A p)
    T* pout;             // fused CG step: p = z + beta p_in is stored here
    const double* beta;  // fused CG step: device beta; NULL => p = z
    double* partials;    // fused CG step: one p.q partial per CTA
    int* err;            // status word: M2S_ERR_TIMEOUT when a stage never lands
};

template <typename T>
__device__ __forceinline__ void ld_vec(const T* p, T (&v)[Vec<T>::V]) {
    const typename Vec<T>::t w = *reinterpret_cast<const typename Vec<T>::t*>(p);
    if constexpr (Vec<T>::V == 2) {
        v[0] = w.x, v[1] = w.y;
    } else {
        v[0] = w.x, v[1] = w.y, v[2] = w.z, v[3] = w.w;
    }
}
template <typename T>
__device__ __forceinline__ void st_vec(T* p, const T (&v)[Vec<T>::V]) {
    typename Vec<T>::t w;
    if constexpr (Vec<T>::V == 2) {
        w.x = v[0], w.y = v[1];
    } else {
        w.x = v[0], w.y = v[1], w.z = v[2], w.w = v[3];
    }
    *reinterpret_cast<typename Vec<T>::t*>(p) = w;
}

// Row 3-sums H of the thread's V points in one box row (left halo value,
// the V values, right halo value), a pair sum shared by two neighbours:
// H(2m) = a(2m-1) + (a(2m) + a(2m+1)), H(2m+1) = (a(2m) + a(2m+1)) + a(2m+2).
template <typename T>
__device__ __forceinline__ void row_sums(const T* row, T (&h)[Vec<T>::V], T (&c)[Vec<T>::V]) {
    constexpr int V = Vec<T>::V;
    ld_vec<T>(row, c);
    const T l = row[-1], r = row[V];
#pragma unroll
    for (int k = 0; k < V; k += 2) {
        const T pr = c[k] + c[k + 1];
        h[k] = (k == 0 ? l : c[k - 1]) + pr;
        h[k + 1] = pr + (k + 2 == V ? r : c[k + 2]);
    }
}

template <typename T, bool PCG, int NS>
__global__ void __launch_bounds__(kThreads, PCG ? kCtasPcg : kCtasSpmv)
    st27_tma_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mp,
                    TmaArgs<T> a) {
    constexpr int V = Vec<T>::V;
    constexpr int BX = box_x<T>();
    constexpr int SE = stage_elems<T>();
    constexpr int SL = slot_elems<T>();
    constexpr int NA = PCG ? 2 : 1;  // arrays per stage (z and p_in)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* const stage = reinterpret_cast<T*>(smem_raw);
    __shared__ __align__(8) unsigned long long full[NS];
    __shared__ double wsum[kWarpsY];

    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int nx = a.d.nx, ny = a.d.ny, nz = a.d.nz;
    const int x0 = blockIdx.x * tile_x<T>(), y0 = blockIdx.y * kTileY;
    const int z0 = blockIdx.z * a.zc, zend = min(z0 + a.zc, nz);
    const int nplanes = zend - z0 + 2;  // planes z0 - 1 .. zend
    const bool two = PCG && a.beta != nullptr;
    const unsigned bytes = stage_bytes<T>() * (two ? 2u : 1u);
    const T beta = two ? (T)(*a.beta) : T(0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // thread 0 starts plane i into stage i % NS; a plane outside the grid is
    // not loaded (it is zero), its stage phase completes with a plain arrive
    auto issue = [&](int i) {
        const int zl = z0 - 1 + i;
        const int s = i % NS;
        if (zl < 0 || zl >= nz) {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[s]))
                         : "memory");
            return;
        }
        mbar_expect_tx(&full[s], bytes);
        T* dst = stage + (size_t)s * NA * SL;
        tma_load_3d(dst, &mx, &full[s], x0 - V, y0 - 1, zl);
        if (two) tma_load_3d(dst + SL, &mp, &full[s], x0 - V, y0 - 1, zl);
    };
    if (threadIdx.x == 0)
        for (int i = 0; i < NS && i < nplanes; ++i) issue(i);

    // per thread: V x-points of kRows rows; the plane sums of the two
    // previous planes and the centre values of the previous plane
    T s2m2[kRows][V], s2m1[kRows][V], cm1[kRows][V];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
        for (int k = 0; k < V; ++k) s2m2[r][k] = s2m1[r][k] = cm1[r][k] = T(0);
    double part = 0.0;
    bool failed = false;
    const int gx = x0 + V * tx;
    const int gy0 = y0 + ty * kRows;
    const bool colok = gx < nx;

    for (int i = 0; i < nplanes; ++i) {
        const int zl = z0 - 1 + i, s = i % NS;
        const bool live = zl >= 0 && zl < nz;
        if (!failed && !mbar_wait(&full[s], (unsigned)(i / NS) & 1u)) failed = true;
        T* buf = stage + (size_t)s * NA * SL;
        if (two) {
            // p = z + beta p_in over the whole box, in place in the z half
            if (live && !failed)
                for (int e = threadIdx.x * V; e < SE; e += kThreads * V) {
                    T zv[V], pv[V];
                    ld_vec<T>(buf + e, zv);
                    ld_vec<T>(buf + SL + e, pv);
#pragma unroll
                    for (int k = 0; k < V; ++k) zv[k] = fma(beta, pv[k], zv[k]);
                    st_vec<T>(buf + e, zv);
                }
            __syncthreads();
        }
        // output plane zo = zl - 1 (its upper neighbours are plane zl)
        const int zo = zl - 1;
        const bool outz = zo >= z0 && zo < zend && colok && !failed;
        const T* row0 = buf + (ty * kRows) * BX + V + V * tx;  // box row of y = gy0 - 1
        const bool rd = live && !failed;
        T hA[V], hB[V], cB[V], tmp[V];
        if (rd) {
            row_sums<T>(row0, hA, tmp);
            row_sums<T>(row0 + BX, hB, cB);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) hA[k] = hB[k] = cB[k] = T(0);
        }
        const i64 pbase = a.d.off + ((i64)zo * ny + gy0) * nx + gx;
        auto emit = [&](int r, const T (&s2)[V], const T (&c)[V]) {
            if (outz && gy0 + r < ny) {
                T yv[V];
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const T box = (s2m2[r][k] + s2m1[r][k]) + s2[k];
                    yv[k] = fma(T(27), cm1[r][k], -box);
                    if constexpr (PCG) part = fma((double)cm1[r][k], (double)yv[k], part);
                }
                st_vec<T>(a.y + pbase + (i64)r * nx, yv);
                if constexpr (PCG) st_vec<T>(a.pout + pbase + (i64)r * nx, cm1[r]);
            }
#pragma unroll
            for (int k = 0; k < V; ++k) {
                s2m2[r][k] = s2m1[r][k];
                s2m1[r][k] = s2[k];
                cm1[r][k] = c[k];
            }
        };
#pragma unroll
        for (int m = 0; m < kRows / 2; ++m) {
            T hC[V], hD[V], cC[V], cD[V], q[V], s0[V], s1[V];
            if (rd) {
                row_sums<T>(row0 + (2 * m + 2) * BX, hC, cC);
                row_sums<T>(row0 + (2 * m + 3) * BX, hD, cD);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) hC[k] = hD[k] = cC[k] = cD[k] = T(0);
            }
#pragma unroll
            for (int k = 0; k < V; ++k) {
                q[k] = hB[k] + hC[k];
                s0[k] = hA[k] + q[k];
                s1[k] = q[k] + hD[k];
            }
            emit(2 * m, s0, cB);
            emit(2 * m + 1, s1, cC);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                hA[k] = hC[k];
                hB[k] = hD[k];
                cB[k] = cD[k];
            }
        }
        // the p pass wrote stage s through the generic proxy; order those
        // writes before the TMA that refills the stage
        if (two) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();  // every thread is done with stage s
        if (threadIdx.x == 0 && !failed && i + NS < nplanes) issue(i + NS);
    }

    if (failed) {
        atomicCAS(a.err, 0, (int)M2S_ERR_TIMEOUT);
        // wait (bounded) for the loads this CTA still has in flight
        if (threadIdx.x == 0)
            for (int i = max(0, nplanes - NS); i < nplanes; ++i)
                mbar_wait(&full[i % NS], (unsigned)(i / NS) & 1u);
        __syncthreads();
    }
    if constexpr (PCG) {
        // fixed-shape reduction: warp tree, then the warp sums in order
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (tx == 0) wsum[ty] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int w = 0; w < kWarpsY; ++w) sum += wsum[w];
            const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            a.partials[bid] = sum;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps (the driver's cuTensorMapEncodeTiled, reached
// through the runtime's entry-point query so that nothing links libcuda),
// grid sizing, launchers.
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// 3-D map of one problem's [nz][ny][nx] array with the kernel's box.
template <typename T>
bool make_map(CUtensorMap* m, const T* base, const Dims& d) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)d.nx * sizeof(T),
                                   (cuuint64_t)d.nx * d.ny * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x<T>(), (cuuint32_t)kBoxY, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(m, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
              3, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// One wave: tiles x z-chunks, the chunk count filling the SMs' CTA slots.
template <typename T>
dim3 tma_grid(const Dims& d, int ctas_per_sm, int* zc) {
    const int gx = (d.nx + tile_x<T>() - 1) / tile_x<T>();
    const int gy = (d.ny + kTileY - 1) / kTileY;
    const int slots = sm_count() * ctas_per_sm;
    int chunks = std::max(1, std::min(d.nz, slots / std::max(1, gx * gy)));
    *zc = (d.nz + chunks - 1) / chunks;
    chunks = (d.nz + *zc - 1) / *zc;
    return dim3(gx, gy, chunks);
}

template <typename T, bool PCG, int NS>
cudaError_t tma_launch(const Dims& d, const CUtensorMap& mx, const CUtensorMap& mp,
                       TmaArgs<T> a, cudaStream_t st) {
    constexpr size_t smem = (size_t)NS * (PCG ? 2 : 1) * slot_elems<T>() * sizeof(T);
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(st27_tma_kernel<T, PCG, NS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 g = tma_grid<T>(d, PCG ? kCtasPcg : kCtasSpmv, &a.zc);
    st27_tma_kernel<T, PCG, NS><<<g, kThreads, smem, st>>>(mx, mp, a);
    return cudaGetLastError();
}

}  // namespace

bool st27_tma_shape_ok(const Dims& d, size_t elem) {
    return d.n > 0 && ((size_t)d.nx * elem) % 16 == 0 && ((size_t)d.off * elem) % 16 == 0 &&
           encode_fn() != nullptr;
}

int st27_tma_pcg_partials(const Dims& d) {
    int zc = 0;
    const dim3 g = tma_grid<double>(d, kCtasPcg, &zc);
    return (int)(g.x * g.y * g.z);
}

// y = A x on one problem's level through the TMA kernel.  Returns
// cudaErrorNotSupported (nothing launched) where the shape or the vectors'
// alignment does not allow it; the caller then uses st27_kernel.
template <typename T>
cudaError_t launch_spmv27_tma(const Dims& d, const T* x, T* y, int* err, cudaStream_t st) {
    if (!st27_tma_shape_ok(d, sizeof(T)) || !aligned16(x) || !aligned16(y) || !err)
        return cudaErrorNotSupported;
    CUtensorMap mx;
    if (!make_map<T>(&mx, x + d.off, d)) return cudaErrorNotSupported;
    TmaArgs<T> a{};
    a.d = d;
    a.y = y;
    a.err = err;
    return tma_launch<T, false, kStagesSpmv>(d, mx, mx, a, st);
}

// p = z + beta p_in (beta NULL: p = z), q = A p, one p.q partial per CTA
// (st27_tma_pcg_partials of them, in block order).
cudaError_t launch_pspmv_dot_tma(const Dims& d, const double* z, const double* pin, double* pout,
                                 double* q, const double* beta, double* partials, int* err,
                                 cudaStream_t st) {
    if (!st27_tma_shape_ok(d, sizeof(double)) || !aligned16(z) || !aligned16(pin) ||
        !aligned16(pout) || !aligned16(q) || !err)
        return cudaErrorNotSupported;
    CUtensorMap mz, mp;
    if (!make_map<double>(&mz, z + d.off, d)) return cudaErrorNotSupported;
    if (beta && !make_map<double>(&mp, pin + d.off, d)) return cudaErrorNotSupported;
    TmaArgs<double> a{};
    a.d = d;
    a.y = q;
    a.pout = pout;
    a.beta = beta;
    a.partials = partials;
    a.err = err;
    return tma_launch<double, true, kStagesPcg>(d, mz, beta ? mp : mz, a, st);
}

template cudaError_t launch_spmv27_tma<double>(const Dims&, const double*, double*, int*,
                                               cudaStream_t);
template cudaError_t launch_spmv27_tma<float>(const Dims&, const float*, float*, int*,
                                              cudaStream_t);

}  // namespace m2s
