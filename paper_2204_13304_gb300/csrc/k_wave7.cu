// Exact-order 7-point (variable kappa) Gauss-Seidel sweep, CTA-pipelined
// wavefront.
//
// Paper Sec. 4.3.3 (Seidel-style stencils) and Sec. 6.1 (SewTh): every point
// is updated in lexicographic order from the new values of its 3 lower
// neighbours and the old-neighbour sum Q:
//     x_p = (Q_p + k_x x_{p-e_x} + k_y x_{p-e_y} + k_z x_{p-e_z}) / a_pp,
//     Q'_p = b_p + (the same lower sum)            (next sweep's Q),
// and the backward sweep is the forward sweep in reflected index space, with
// the coefficients of the upper faces (kr) in place of the lower ones (kf).
// Points of the hyperplane t = x + y + z are independent.
//
// GPU mapping: a unit is a CTA of W warps; warp w owns plane z = z0 + w, lane
// l row y = y0 - 1 + l (lane 0 replays row y0 - 1 of the unit to the left
// from its mailbox, lanes 1-31 compute).  At local step s lane l of warp w is
// at x = s - l - w: every thread of the CTA is on the same hyperplane, the
// y - 1 neighbour is the lane below one step earlier (a shuffle of its
// previous value), the z - 1 neighbour the warp below one step earlier
// (a tagged shared-memory ring) or, for warp 0, the top warp of the unit
// underneath (tagged mailbox).  The synchronisation pieces are those of the
// 27-point sweep (k_wave2.cu): tagged words, a vote per step, bounded polls.
#include <algorithm>
#include <climits>
#include <type_traits>
#include <vector>

#include "m2s_cta.cuh"
#include "m2s_internal.cuh"
#include "m2s_wave_sync.cuh"

namespace m2s {

namespace {

using namespace wave;
using namespace cta;

constexpr int LANES7 = 31;  // computing rows per unit

template <typename T>
struct Cta7Args {
    int rev;
    long long spin_ns;
    const T* Qin;
    T* Qout;
    const T* b;
    T* x;
    const T* kp;  // per point (k_x, k_y, k_z, 1/a_pp) of the lower
                  // neighbours in sweep order (packed level array)
    const int4* units;  // (y0, z0, problem, first b.x partial), ticket order
    const Dims* dims;   // per problem: extent and packed offset
    int n_units;
    int* ctrl;
    DevStatus* status;
    double* rz;
    int stall_unit;
    u64* mbox;
};

// The four coefficients of a point: one 32-byte (FP64: two 16-byte loads)
// or one 16-byte (FP32) read-only load, one sector per lane.
__device__ __forceinline__ void ld_pack(const double* p, double* a, double* b, double* c,
                                        double* d) {
    const double2 u = __ldg(reinterpret_cast<const double2*>(p));
    const double2 v = __ldg(reinterpret_cast<const double2*>(p) + 1);
    *a = u.x, *b = u.y, *c = v.x, *d = v.y;
}
__device__ __forceinline__ void ld_pack(const float* p, float* a, float* b, float* c, float* d) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(p));
    *a = u.x, *b = u.y, *c = u.z, *d = u.w;
}

template <typename T, int W>
struct Cta7Shared {
    typename Tagged<T>::W ring[W][RING][32];
    volatile int prog[W];
};

template <typename T, int W, int D, int RD, int ROLE>
__device__ __forceinline__ void sweep7_warp(const Cta7Args<T>& a, int t, int w,
                                            Cta7Shared<T, W>& sh, unsigned tag) {
    typedef typename Tagged<T>::W TW;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int4 un = a.units[t];
    const Dims dm = a.dims[un.z];
    const int y = un.x - 1 + lane;
    const int z = un.y + w;
    const bool halo = lane == 0;
    const bool rv = y >= 0 && y < dm.ny && z < dm.nz;
    // ROLE: -1 read from w; 0 the bottom warp, 1 a middle one, 2 the top one
    const bool bottom = ROLE < 0 ? w == 0 : ROLE == 0;
    const bool topw = ROLE < 0 ? w == W - 1 : ROLE == 2;
    const bool ring_in = !bottom;
    const bool ring_out = !topw;
    const bool mb_out = !halo && (lane == 31 || topw);
    const bool zmb = bottom && z >= 1;  // plane below from the unit underneath
    const int nx = dm.nx;
    // direction: RD = 0 forward, 1 backward (compile time), -1 read at run time
    const bool rev = RD < 0 ? a.rev != 0 : RD == 1;
    typedef typename std::conditional<(RD < 0), i64, int>::type StepT;
    const StepT dir = rev ? -1 : 1;
    const i64 r = rv ? ((i64)z * dm.ny + y) * nx : 0;
    const i64 L = rev ? dm.n - 1 - r : r;  // problem-local index of x = 0
    const i64 szd = dir * (i64)nx * dm.ny;   // index step of the z - 1 neighbour
    const T* Q = a.Qin + dm.off;
    const T* B = a.b + dm.off;
    const T* KP = a.kp + 4 * dm.off;
    T* Xo = a.x + dm.off;
    T* Qo = a.Qout ? a.Qout + dm.off : nullptr;
    // this problem's mailbox (indexed by the problem-local point)
    u64* const mbox = a.mbox + dm.off * (sizeof(T) == 8 ? 2 : 1);
    const bool want_rz = sizeof(T) == 8 && a.rz != nullptr;
    const int S = nx + LANES7 + W;

    T xm1 = 0;
    // prefetch ring: Q, b, the three coefficients and 1/a_pp (computing
    // lanes) or the mailbox words of the replayed row (lane 0); the mailbox
    // words of the plane below (warp 0)
    T rq[D], rb[D], r0[D], r1[D], r2[D], rd[D], rz0[D], rz1[D];
    auto fetch = [&](int k, int s) {
        const int xx = s - lane - w;
        T q = 0, bv = 0, c0 = 0, c1 = 0, c2 = 0, dd = 0, m0 = 0, m1 = 0;
        if (rv && (unsigned)xx < (unsigned)nx) {
            const i64 p = L + dir * xx;
            if (!halo) {
                q = __ldg(Q + p);
                bv = __ldg(B + p);
                ld_pack(KP + 4 * p, &c0, &c1, &c2, &dd);
                if (zmb) tw_to_regs(mb_load<T>(mbox, p - szd), &m0, &m1);
            } else {
                tw_to_regs(mb_load<T>(mbox, p), &q, &bv);
            }
        }
        rq[k] = q;
        rb[k] = bv;
        r0[k] = c0;
        r1[k] = c1;
        r2[k] = c2;
        rd[k] = dd;
        rz0[k] = m0;
        rz1[k] = m1;
    };
#pragma unroll
    for (int k = 0; k < D; ++k) fetch(k, k);

    double rzs = 0.0;
    bool ok = true;
    int cachedC = -(1 << 30);
    auto fail = [&]() -> bool {
        int ab = 0;
        if (lane == 0) ab = ld_relaxed_gpu(&a.status->abort);
        return __shfl_sync(FULL, ab, 0) != 0;
    };
    auto timeout = [&]() {
        if (lane == 0) {
            atomicCAS(&a.status->err, 0, (int)M2S_ERR_TIMEOUT);
            atomicExch(&a.status->abort, 1);
        }
    };
    auto step = [&](int s, int k) {
        const int xx = s - lane - w;
        const T q = rq[k], bv = rb[k], c0 = r0[k], c1 = r1[k], c2 = r2[k], dd = rd[k];
        const T m0 = rz0[k], m1 = rz1[k];
        fetch(k, s + D);
        const bool in = rv && (unsigned)xx < (unsigned)nx;
        const bool comp = in && !halo;
        // replayed row (lane 0), plane below (mailbox for warp 0, ring of the
        // warp below, which writes an entry at each of its steps; this
        // warp's step s reads the entry of its step s - 1)
        T X1 = 0, zv = 0;
        bool okx = true, okz = true, okr = true;
        if (in && halo) okx = Tagged<T>::unpack(regs_to_tw(q, bv), tag, &X1);
        if (comp && zmb) okz = Tagged<T>::unpack(regs_to_tw(m0, m1), tag, &zv);
        // the x - 1 and y - 1 terms of N need only the previous step: issued
        // before the wait, they overlap it (same order of operations)
        const T hu = __shfl_up_sync(FULL, xm1, 1);  // row y - 1 at this x
        T N = c0 * xm1;
        N = fma(c1, hu, N);
        const TW* re = ring_in ? &sh.ring[w - 1][(s - 1) & (RING - 1)][lane] : nullptr;
        const unsigned rtag = (unsigned)(s - 1 + BIAS);
        if (ring_in && s >= 1) okr = Tagged<T>::unpack(*(volatile const TW*)re, rtag, &zv);
        if (!__all_sync(FULL, okx && okz && okr)) {
            // poll only what is missing; the abort word and the clock are
            // read once every 32 polls
            const i64 p = L + dir * xx;
            unsigned long long t0 = 0;
            for (int it = 1;; ++it) {
                if (!okr) okr = Tagged<T>::unpack(*(volatile const TW*)re, rtag, &zv);
                if (!okx) okx = Tagged<T>::unpack(mb_load<T>(mbox, p), tag, &X1);
                if (!okz) okz = Tagged<T>::unpack(mb_load<T>(mbox, p - szd), tag, &zv);
                if (__all_sync(FULL, okx && okz && okr)) break;
                if ((it & 31) == 0) {
                    const unsigned long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    if (fail()) { ok = false; return; }
                    if ((long long)(now - t0) > a.spin_ns) { timeout(); ok = false; return; }
                }
            }
        }
        if (comp) {
            N = fma(c2, zv, N);
            X1 = (q + N) * dd;
            const i64 p = L + dir * xx;
            Xo[p] = X1;
            if (Qo) Qo[p] = bv + N;
            if constexpr (sizeof(T) == 8) {
                if (want_rz) rzs = fma((double)bv, (double)X1, rzs);
            }
            if (mb_out) mb_store<T>(mbox, p, X1, tag);
        } else if (!in) {
            X1 = T(0);
        }
        xm1 = X1;
        if (ring_out) {
            // back-pressure: the entry this step overwrites (step s - RING)
            // must have been read by the warp above (at its step s - RING + 1)
            const int old = s - RING;
            if (old >= 0 && old + 1 > cachedC) {
                int c = 0, okk = 1;
                if (lane == 0) {
                    unsigned long long t0 = 0;
                    for (int it = 1;; ++it) {
                        c = sh.prog[w + 1];
                        if (c >= old + 1) break;
                        if ((it & 31) != 0) continue;
                        const unsigned long long now = global_ns();
                        if (t0 == 0) t0 = now;
                        if (ld_relaxed_gpu(&a.status->abort) || (long long)(now - t0) > a.spin_ns) {
                            atomicCAS(&a.status->err, 0, (int)M2S_ERR_TIMEOUT);
                            atomicExch(&a.status->abort, 1);
                            okk = 0;
                            break;
                        }
                    }
                }
                okk = __shfl_sync(FULL, okk, 0);
                cachedC = __shfl_sync(FULL, c, 0);
                if (!okk) { ok = false; return; }
            }
            sh.ring[w][s & (RING - 1)][lane] = Tagged<T>::pack(X1, (unsigned)(s + BIAS));
        }
        __syncwarp();
        if (lane == 0) sh.prog[w] = s;
    };
    for (int s0 = 0; ok && s0 < S; s0 += D) {
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (ok) step(s0 + k, k);
    }
    __syncwarp();
    if (lane == 0) sh.prog[w] = INT_MAX;
    if (want_rz) {
        for (int o = 16; o > 0; o >>= 1) rzs += __shfl_down_sync(FULL, rzs, o);
        if (lane == 0) a.rz[(i64)un.w + w] = ok ? rzs : 0.0;
    }
}

// FP32 warps run a copy of the step compiled for their role, which drops
// the role tests from the step (256^3 FP32 sweep 0.65 -> 0.62 ms with the
// loop unrolled four deep; eight deep, the three copies took 1.04 ms).  FP64
// keeps one copy: with three, the 256^3 sweep was unchanged (0.92 ms) but
// the batched solve of 64 problems of 32^3-128^3 went 1.80 -> 2.21 s (its
// finest-level sweep 1.30 -> 1.66 ms).
template <typename T>
constexpr bool kRoles7 = sizeof(T) == 4;

template <typename T, int W, int D, int RD>
__global__ void __launch_bounds__(W * 32, 1) gs7_cta_kernel(Cta7Args<T> a) {
    __shared__ int s_ticket;
    __shared__ unsigned s_tag;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    Cta7Shared<T, W>& sh = *reinterpret_cast<Cta7Shared<T, W>*>(dyn_smem);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tag = (unsigned)ld_relaxed_gpu(&a.ctrl[2]) + 1u;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&a.ctrl[0], 1);
        // ring tags of an earlier unit of this CTA could match a step of
        // this unit: clear the rings
        for (int i = threadIdx.x; i < W * RING * 32; i += blockDim.x)
            (&sh.ring[0][0][0])[i] = Tagged<T>::zero();
        if (threadIdx.x < W) sh.prog[threadIdx.x] = -(1 << 30);
        __syncthreads();
        const int t = s_ticket;
        if (t >= a.n_units) break;
        int ab = 0;
        if (threadIdx.x == 0) ab = ld_relaxed_gpu(&a.status->abort) || t == a.stall_unit;
        ab = __syncthreads_or(ab);
        if (!ab) {
            if constexpr (kRoles7<T>) {
                if (warp == 0)
                    sweep7_warp<T, W, D, RD, 0>(a, t, warp, sh, s_tag);
                else if (warp == W - 1)
                    sweep7_warp<T, W, D, RD, 2>(a, t, warp, sh, s_tag);
                else
                    sweep7_warp<T, W, D, RD, 1>(a, t, warp, sh, s_tag);
            } else {
                sweep7_warp<T, W, D, RD, -1>(a, t, warp, sh, s_tag);
            }
        }
        __syncthreads();
    }
    // exit protocol: the last CTA out resets the ticket and advances the tag
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int last = atomicAdd(&a.ctrl[1], 1) == (int)gridDim.x - 1;
        if (last) {
            a.ctrl[0] = 0;
            a.ctrl[1] = 0;
            a.ctrl[2] = a.ctrl[2] + 1;
            a.status->abort = 0;
            __threadfence();
        }
    }
}

template <typename T> struct Cta7Shape;
// RD0 / RD1: the direction template argument of the forward / backward
// launches (0 and 1 compile the direction in; -1 reads it at run time).
// Measured on a GB300 (variable-kappa 256^3 MG-PCG): compiled-in directions
// take the 256^3 sweep from 0.98 to 0.97 ms (FP64) and 0.72 to 0.71 ms
// (FP32), the solves from 2.54 to 2.50 s and 1.99 to 1.95 s.  D is the
// prefetch depth in steps and the unrolling of the step loop: 4 for both,
// so that the role copies of the FP32 step fit the instruction cache.
template <> struct Cta7Shape<double> { static constexpr int W = 8, D = 4, RD0 = 0, RD1 = 1; };
template <> struct Cta7Shape<float> { static constexpr int W = 8, D = 4, RD0 = 0, RD1 = 1; };

template <typename T>
size_t cta7_smem_bytes() {
    return sizeof(Cta7Shared<T, Cta7Shape<T>::W>);
}

}  // namespace

// Unit table of one level for all problems of a grid (one launch per level):
// units of 31 rows x W planes, ordered within a problem by the step at which
// they could start on an idle GPU (the unit to the right lags 31 steps, the
// unit above W; producers, left and below, have smaller keys, so the order
// is topological), problems merged by the same key.
template <typename T>
cudaError_t build_cta7_units(const std::vector<Dims>& dims, WaveUnits* out) {
    constexpr int W = Cta7Shape<T>::W, D = Cta7Shape<T>::D;
    struct Item {
        long long key;
        int z0, problem, local, y0;
    };
    std::vector<Item> items;
    std::vector<int> rzpre(dims.size() + 1, 0);
    i64 words = 0;
    for (size_t i = 0; i < dims.size(); ++i) {
        const Dims& d = dims[i];
        const int NY = (d.ny + LANES7 - 1) / LANES7, NZ = (d.nz + W - 1) / W;
        std::vector<Item> mine;
        for (int Z = 0; Z < NZ; ++Z)
            for (int Y = 0; Y < NY; ++Y)
                mine.push_back(Item{(long long)Y * LANES7 + (long long)Z * W, Z * W, (int)i, 0,
                                    Y * LANES7});
        std::stable_sort(mine.begin(), mine.end(), [](const Item& a, const Item& b) {
            return a.key != b.key ? a.key < b.key : a.z0 < b.z0;
        });
        for (size_t k = 0; k < mine.size(); ++k) {
            mine[k].local = (int)k;
            items.push_back(mine[k]);
        }
        rzpre[i + 1] = rzpre[i] + (int)mine.size() * W;
        words += std::max<i64>(d.n, 0) * (sizeof(T) == 8 ? 2 : 1);
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
        if (a.key != b.key) return a.key < b.key;
        return a.problem != b.problem ? a.problem < b.problem : a.z0 < b.z0;
    });
    std::vector<int4> units(items.size());
    for (size_t k = 0; k < items.size(); ++k)
        units[k] = make_int4(items[k].y0, items[k].z0, items[k].problem,
                             rzpre[items[k].problem] + items[k].local * W);
    WaveUnits u{};
    u.n_units = (int)units.size();
    u.K = 2;
    u.W = W;
    u.stencil = 7;
    u.np = (int)dims.size();
    u.n_rz = rzpre.back();
    cudaError_t e;
    const size_t nu = std::max<size_t>(units.size(), 1);
    if ((e = cudaMalloc(&u.d_units, nu * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_dims, std::max<size_t>(dims.size(), 1) * sizeof(Dims))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_rzpre, rzpre.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_ctrl, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_mbox, (size_t)std::max<i64>(words, 1) * sizeof(u64))) != cudaSuccess) {
        free_wave_units(&u);
        return e;
    }
    if ((!units.empty() && (e = cudaMemcpy(u.d_units, units.data(), units.size() * sizeof(int4),
                                           cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (!dims.empty() && (e = cudaMemcpy(u.d_dims, dims.data(), dims.size() * sizeof(Dims),
                                          cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(u.d_rzpre, rzpre.data(), rzpre.size() * sizeof(int),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(u.d_ctrl, 0, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(u.d_mbox, 0, (size_t)std::max<i64>(words, 1) * sizeof(u64))) != cudaSuccess) {
        free_wave_units(&u);
        return e;
    }
    const size_t smem = cta7_smem_bytes<T>();
    constexpr int R0 = Cta7Shape<T>::RD0, R1 = Cta7Shape<T>::RD1;
    cudaFuncSetAttribute(gs7_cta_kernel<T, W, D, R0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaFuncSetAttribute(gs7_cta_kernel<T, W, D, R1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int per_sm = 0, per_sm1 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs7_cta_kernel<T, W, D, R0>, W * 32,
                                                  smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm1, gs7_cta_kernel<T, W, D, R1>, W * 32,
                                                  smem);
    per_sm = std::min(per_sm, per_sm1);
    u.grid = wave_grid(u.n_units, per_sm);
    *out = u;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs7_cta(const WaveUnits& u, const WaveCall& c, const KappaLevel<T>& k,
                           const T* Qin, T* Qout, const T* b, T* x, cudaStream_t st) {
    constexpr int W = Cta7Shape<T>::W, D = Cta7Shape<T>::D;
    if (u.n_units == 0) return cudaSuccess;
    Cta7Args<T> a;
    a.rev = c.rev;
    a.spin_ns = c.spin_ns;
    a.Qin = Qin;
    a.Qout = Qout;
    a.b = b;
    a.x = x;
    // sweep order's lower faces: kf (forward) or the upper faces kr
    // (backward sweep = forward sweep in reflected index space), packed
    // with 1/a_pp
    a.kp = k.pack[c.rev ? 1 : 0];
    a.units = u.d_units;
    a.dims = u.d_dims;
    a.n_units = u.n_units;
    a.ctrl = u.d_ctrl;
    a.status = c.status;
    a.rz = c.rz_partials;
    a.stall_unit = c.stall_unit;
    a.mbox = u.d_mbox;
    constexpr int R0 = Cta7Shape<T>::RD0, R1 = Cta7Shape<T>::RD1;
    if (c.rev)
        gs7_cta_kernel<T, W, D, R1><<<u.grid, W * 32, cta7_smem_bytes<T>(), st>>>(a);
    else
        gs7_cta_kernel<T, W, D, R0><<<u.grid, W * 32, cta7_smem_bytes<T>(), st>>>(a);
    return cudaGetLastError();
}

template cudaError_t build_cta7_units<double>(const std::vector<Dims>&, WaveUnits*);
template cudaError_t build_cta7_units<float>(const std::vector<Dims>&, WaveUnits*);
template cudaError_t launch_gs7_cta<double>(const WaveUnits&, const WaveCall&,
                                            const KappaLevel<double>&, const double*, double*,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_gs7_cta<float>(const WaveUnits&, const WaveCall&,
                                           const KappaLevel<float>&, const float*, float*,
                                           const float*, float*, cudaStream_t);

}  // namespace m2s
