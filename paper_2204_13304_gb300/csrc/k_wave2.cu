// Exact-order 27-point Gauss-Seidel sweep, CTA-pipelined wavefront.
//
// The method is the same as in k_wave.cu (paper Sec. 4.3.3 SymGS; Sec. 6.1
// SewTh): every point is updated in lexicographic order from the new values
// of its 13 lower neighbours and the precomputed old-neighbour sum Q, on the
// point hyperplane t = x + 2y + 4z with rows (u, v) = (y + z, z).  What
// changes is how the wavefront is mapped onto the GPU, after measuring a
// GB300: an FP64 warp instruction occupies a sub-partition's FP64 pipe for
// ~64 clocks (dependent latency ~66), an L2 hit costs ~460 clocks, a
// GPU-scope release ~830 clocks of stall and drains the warp's outstanding
// loads, a shared-memory handoff between warps ~250 clocks and a global
// producer->consumer handoff ~1800.
//
//  * Units are CTAs of W compute warps (4 or 8, chosen at run time) stacked
//    in v, one computed plane per warp, and 32 lanes in u: lanes 0-1 replay
//    the two rows of the unit to the left, warp 0 also replays the plane
//    below from the unit underneath.  Units take tickets in topological
//    order, sorted by the step at which they can start; one CTA runs per
//    SM, and each warp runs a copy of the step compiled for its role
//    (bottom, middle or top warp of the unit).
//  * Values crossing units travel through a mailbox of tagged words (value
//    and launch tag in one 64-bit relaxed store): a reader that sees the
//    current tag has the value, so neither side fences.  Warps of a CTA
//    pass their plane sums G through tagged shared-memory rings, with
//    back-pressure from the consumer's progress word.
//  * Q, b and replayed rows are prefetched D steps ahead into a register
//    ring (the step loop is unrolled by D so the ring is statically
//    indexed).  A warp votes once per step on all its tag checks; only a
//    failed vote enters the bounded poll.
//  * The 13-neighbour sum is evaluated separably: each row keeps its row
//    3-sum H, the lane below passes H and S2 = H(u-1) + H(u), and the 3x3
//    plane sum G = S2(u-1) + H(u) flows to the plane above.
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

template <typename T>
struct CtaArgs {
    int rev;
    long long spin_ns;
    // packed level arrays of all problems.  Qin and Qout hold the
    // old-neighbour sums pre-scaled by 1/26 (Q/26), so a point's update
    // (Q + N)/26 is one FMA, N * (1/26) + Q/26.  b is b/26 when Qout is
    // written (Qout = N * (1/26) + b/26) and b itself when rz is (b.x): a
    // sweep never does both.
    const T* Qin;
    T* Qout;
    const T* b;
    T* x;
    const int4* units;  // (u0, v0, problem, first b.x partial) per unit
    const Dims* dims;   // per problem: extent and packed offset
    int n_units;
    int* ctrl;
    DevStatus* status;
    double* rz;          // b.x partials (W per unit) or NULL
    int stall_unit;
    unsigned long long* mbox;  // tagged x of the rows the unit to the right replays
    unsigned long long* mbg;   // tagged plane sums G the unit above reads
    const long long* mboff;    // per problem: first value of its mbox and mbg slices
};

// Mailbox rows (units are 30 rows u x W planes v, origins (30 U, W V)).
// mbox: the rows u = 30 U + 28, 30 U + 29 of each plane v, written by lanes
// 30-31 of unit U and replayed by the halo lanes 0-1 of unit U + 1: row
// slot (v, U, u mod 30 - 28).  mbg: the plane sums G at the rows of the
// planes v = W m, written by the top warp of the unit below and read by warp
// 0 of the unit starting at v: row slot (m, u).  Values of a row are
// contiguous in the sweep's own x, so the mailboxes hold ~1/15 and ~1/W of a
// level instead of a value per point.
__host__ __device__ inline int mb_rows_u(int ny, int nz) { return ny + nz - 1; }
__host__ __device__ inline int mb_cols(int ny, int nz) { return (mb_rows_u(ny, nz) - 1) / 30 + 1; }
inline i64 mbox_values(const Dims& d) { return (i64)d.nz * mb_cols(d.ny, d.nz) * 2 * d.nx; }
inline i64 mbg_values(const Dims& d, int W) {
    return (i64)((d.nz - 1) / W + 1) * mb_rows_u(d.ny, d.nz) * d.nx;
}

// One compute warp of a CTA unit: lane = row u (lanes 0-1 replay the rows
// of the unit to the left), plane v1 = org.y + w is computed, plane
// v0 = v1 - 1 below it is replayed (warp 0 reads it from the producers'
// mailbox and forms its sums; warps above take the finished plane sums G of
// the warp below from its shared-memory ring).  Rows that other units read
// (lanes 30-31, and the top warp's plane) are also written to the mailbox
// with the launch tag.  The step is written for the fewest instructions:
// one warp vote per step for all tag checks, and the work that needs only
// the previous step issued ahead of the wait.  RD is the direction: 0
// forward, 1 backward, -1 read from the launch arguments; ROLE the warp's
// place in the unit (-1: read from w).
// Measured on a GB300 (256^3 sweeps inside the MG-PCG solve): a
// compile-time direction makes the FP32 sweep 8 % faster (1.24 -> 1.15 ms)
// and the FP64 sweep 2 % slower (1.69 -> 1.72 ms), so FP32 launches use
// RD = 0 / 1 and FP64 launches RD = -1.
template <typename T, int W, int D, int RD, int ROLE>
__device__ __forceinline__ void compute_warp(const CtaArgs<T>& a, int t, int w,
                                             CtaShared<T, W>& sh, unsigned tag) {
    typedef typename Tagged<T>::W TW;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int4 un = a.units[t];
    const int2 org = make_int2(un.x, un.y);
    const Dims dd = a.dims[un.z];
    const int v1 = org.y + w;
    const int u = org.x - 2 + lane;
    const int tbase = 2 * (org.x - 2) + 2 * (v1 - 1);
    const T inv26 = Lit<T>::inv26();
    const bool halo = lane < 2;
    // ROLE: -1 read from w; 0 the bottom warp, 1 a middle one, 2 the top one
    const bool ring_in = ROLE < 0 ? w > 0 : ROLE != 0;
    const bool ring_out = ROLE < 0 ? w < W - 1 : ROLE != 2;
    const bool top = ROLE < 0 ? w == W - 1 : ROLE == 2;
    const bool mb_out = !halo && lane >= 30;
    const int nx = dd.nx;
    const int y1 = u - v1;
    const bool rv1 = v1 < dd.nz && y1 >= 0 && y1 < dd.ny;
    // plane sums of the plane below from the unit underneath (warp 0), and
    // for the unit above (top warp: published at the point of the row above)
    const bool g_in = !ring_in && v1 >= 1;
    const int yu = u - (v1 + 1);
    const bool g_out = top && !halo && v1 + 1 < dd.nz && yu >= 0 && yu < dd.ny;
    const bool rev = RD < 0 ? a.rev != 0 : RD == 1;
    // a 64-bit step read at run time, or a 32-bit compile-time one
    typedef typename std::conditional<(RD < 0), i64, int>::type StepT;
    const StepT step_dir = rev ? -1 : 1;
    // problem-local index of x = 0 of this row
    const i64 r1 = ((i64)v1 * dd.ny + y1) * nx;
    const i64 L1 = rev ? dd.n - 1 - r1 : r1;
    // mailbox rows of this lane, in the sweep's own coordinates
    const int NU = mb_rows_u(dd.ny, dd.nz);
    const i64 mrow = (u >= 0 && (halo || mb_out))
                         ? (((i64)v1 * mb_cols(dd.ny, dd.nz) + u / 30) * 2 + (u % 30 - 28)) * nx
                         : 0;
    const i64 grow_in = g_in ? ((i64)(v1 / W) * NU + u) * nx : 0;
    const i64 grow_out = g_out ? ((i64)((v1 + 1) / W) * NU + u) * nx : 0;
    const T* Qin = a.Qin + dd.off;
    const T* B = a.b + dd.off;
    T* Xo = a.x + dd.off;
    T* Qo = a.Qout ? a.Qout + dd.off : nullptr;
    // this problem's mailboxes.  Within a row, x1 is at row + x1 in a forward
    // sweep and at row + nx - 1 - x1 in a backward one (the direction of the
    // arrays), so a lane's mailbox index is its array index p plus a
    // constant: the pointers below are offset by that constant once.
    const i64 wpv = sizeof(T) == 8 ? 2 : 1;
    const i64 rx = rev ? nx - 1 : 0;
    u64* const mbox = a.mbox + a.mboff[2 * un.z] * wpv;
    u64* const mbg = a.mbg + a.mboff[2 * un.z + 1] * wpv;
    u64* const mbox_p = mbox + (mrow + rx - L1) * wpv;     // index p
    u64* const mbg_p = mbg + (grow_in + rx - L1) * wpv;    // index p
    const i64 Gu = grow_out + rx;                           // + step_dir * x
    // the fused r.z partial is used by the FP64 PCG only; compiling it out of
    // the FP32 sweep keeps float->double conversions off the FP64 pipe
    const bool want_rz = sizeof(T) == 8 && a.rz != nullptr;

    // row state: the last two x values and the sums passed to the lane above
    T xm1 = 0, xm2 = 0, h1 = 0, h2 = 0, s21 = 0, s22 = 0;
    // prefetch ring: Q and b (computing lanes) or the mailbox bits of the
    // replayed row (halo lanes); the mailbox bits of G (warp 0)
    T rq[D], rb[D], ra0[D], rb0[D];

    const int S = nx + 2 * 31 + 3;
    // fetch the inputs of step s (x1 = s - 2 lane - 2) into slot k
    auto fetch = [&](int k, int x1) {
        T q = 0, bv = 0, m0 = 0, m1 = 0;
        if (rv1 && (unsigned)x1 < (unsigned)nx) {
            const i64 p = L1 + step_dir * x1;
            if (!halo) {
                q = __ldg(Qin + p);
                bv = __ldg(B + p);
                // once per 128-byte line of the row, ask L2 for the line one
                // line ahead (256^3 FP64 sweep 1.58 -> 1.55 ms; no change in
                // FP32)
                constexpr int kLine = 128 / (int)sizeof(T);
                if ((x1 & (kLine - 1)) == 0 && x1 + kLine < nx) {
                    prefetch_l2(Qin + p + step_dir * kLine);
                    prefetch_l2(B + p + step_dir * kLine);
                }
                if (g_in) tw_to_regs(mb_load<T>(mbg_p, p), &m0, &m1);
            } else {
                tw_to_regs(mb_load<T>(mbox_p, p), &q, &bv);
            }
        }
        rq[k] = q;
        rb[k] = bv;
        ra0[k] = m0;
        rb0[k] = m1;
    };
#pragma unroll
    for (int k = 0; k < D; ++k) fetch(k, k - 2 * lane - 2);

    double rz = 0.0;
    bool ok = true;
    int cachedC = -(1 << 30);
    // FP32 reads the ring entry of step s + 1 at the end of step s (the wait
    // at step s + 1 then checks a tag already in registers): 256^3 FP32 sweep
    // 1.21 -> 1.18 ms; FP64 measured no faster and reads it at its step.
    constexpr bool kEarlyRing = sizeof(T) == 4;
    TW pre = Tagged<T>::zero();
    if (kEarlyRing && ring_in) pre = ring_load(&sh.ring[w - 1][(tbase - 1) & (RING - 1)][lane]);
    auto fail = [&]() -> bool {  // abort check / timeout for the slow paths
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
        const int x1 = s - 2 * lane - 2;
        const int tnow = s + tbase;
        const T q = rq[k], bv = rb[k], m0 = ra0[k], m1 = rb0[k];
        fetch(k, x1 + D);
        const bool in1 = rv1 && (unsigned)x1 < (unsigned)nx;
        const bool comp = in1 && !halo;
        const bool in0 = comp && g_in;  // G of the plane below from the mailbox
        // replayed values: mailbox (halo lanes: x of the row; warp 0: G of
        // the plane below at this point) and ring (G, warps above 0)
        T X1 = 0, gin = 0;
        bool good = true;
        if (in1 && halo) good = Tagged<T>::unpack(regs_to_tw(q, bv), tag, &X1);
        if (in0) good = Tagged<T>::unpack(regs_to_tw(m0, m1), tag, &gin) && good;
        // The lane shuffles and the first add of N need only the previous
        // step: issued before the wait, they overlap its ring load and vote
        // (isolated 4-warp FP64 unit 684 -> 585 ns per step; 256^3 FP64
        // sweep -4 %).
        const T hu1 = __shfl_up_sync(FULL, h1, 1);
        const T hu2 = __shfl_up_sync(FULL, h2, 1);
        const T su2 = __shfl_up_sync(FULL, s22, 1);
        const T xh = xm1 + hu1;
        const T x2 = xm2 + xm1;  // the first add of the row sum H
        const TW* re = ring_in ? &sh.ring[w - 1][(tnow - 1) & (RING - 1)][lane] : nullptr;
        const unsigned gtag = (unsigned)(tnow - 1 + BIAS);
        // The warp below writes a ring entry at each of its steps; this warp's
        // step s reads the entry of its step s + 1 (all but the last), so the
        // wait needs no vote.  A poll reloads only what is missing and reads
        // the abort word and the clock once every 32 polls, so that it costs
        // one load: a consumer sees its producer's value within a few dozen
        // cycles of its arrival (FP32 measured 1.15 -> 1.11 ms per 256^3
        // sweep against a poll that rereads every source, the abort word and
        // the clock each time).
        bool okx = good, okg = true;
        if (ring_in && s + 1 < S) okg = Tagged<T>::unpack(kEarlyRing ? pre : ring_load(re), gtag, &gin);
        if (!__all_sync(FULL, okx && okg)) {
            bool ok1 = !(in1 && halo), ok0 = !in0;
            if (!ok1) ok1 = Tagged<T>::unpack(regs_to_tw(q, bv), tag, &X1);
            if (!ok0) ok0 = Tagged<T>::unpack(regs_to_tw(m0, m1), tag, &gin);
            unsigned long long t0 = 0;
            for (int it = 1;; ++it) {
                if (!okg) okg = Tagged<T>::unpack(ring_load(re), gtag, &gin);
                if (!ok1) ok1 = Tagged<T>::unpack(mb_load<T>(mbox_p, L1 + step_dir * x1), tag, &X1);
                if (!ok0) ok0 = Tagged<T>::unpack(mb_load<T>(mbg_p, L1 + step_dir * x1), tag, &gin);
                if (__all_sync(FULL, ok1 && ok0 && okg)) break;
                if ((it & 31) == 0) {
                    const unsigned long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    if (fail()) { ok = false; return; }
                    if ((long long)(now - t0) > a.spin_ns) { timeout(); ok = false; return; }
                }
            }
        }
        // computed plane
        if (comp) {
            const T N = xh + gin;
            X1 = fma(N, inv26, q);
            const i64 p = L1 + step_dir * x1;
            Xo[p] = X1;
            if (Qo) Qo[p] = fma(N, inv26, bv);
            if constexpr (sizeof(T) == 8) {
                if (want_rz) rz = fma((double)bv, (double)X1, rz);
            }
            if (mb_out) mb_store<T>(mbox_p, p, X1, tag);
        }
        const T H = x2 + X1;
        xm2 = xm1;
        xm1 = X1;
        h2 = h1;
        h1 = H;
        const T S2 = hu2 + H;
        const T G = su2 + H;  // centred at x1 - 1
        s22 = s21;
        s21 = S2;
        if (ring_out) {
            // back-pressure: the ring entry of step tnow - RING must have been
            // read by the warp above (first read: entry tbase + 1)
            const int old_entry = tnow - RING;
            if (old_entry >= tbase + 1 && old_entry + 1 > cachedC) {
                int c = 0, okk = 1;
                if (lane == 0) {
                    const unsigned long long t0 = global_ns();
                    for (;;) {
                        c = sh.prog[w + 1];
                        if (c >= old_entry + 1) break;
                        if (ld_relaxed_gpu(&a.status->abort) ||
                            (long long)(global_ns() - t0) > a.spin_ns) {
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
            sh.ring[w][tnow & (RING - 1)][lane] = Tagged<T>::pack(G, (unsigned)(tnow + BIAS));
        }
        // the top warp publishes G for warp 0 of the unit above, at the point
        // of the row above that consumes it
        if (g_out && (unsigned)(x1 - 1) < (unsigned)nx) mb_store<T>(mbg, Gu + step_dir * (x1 - 1), G, tag);
        if (kEarlyRing && ring_in) pre = ring_load(&sh.ring[w - 1][tnow & (RING - 1)][lane]);
        __syncwarp();
        if (lane == 0) sh.prog[w] = tnow;
    };
    for (int s0 = 0; ok && s0 < S; s0 += D) {
#pragma unroll
        for (int k = 0; k < D; ++k)
            if (ok) step(s0 + k, k);
    }
    __syncwarp();
    if (lane == 0) sh.prog[w] = INT_MAX;
    if (want_rz) {
        for (int o = 16; o > 0; o >>= 1) rz += __shfl_down_sync(FULL, rz, o);
        if (lane == 0) a.rz[(i64)un.w + w] = ok ? rz : 0.0;
    }
}

// Warps run a copy of the step compiled for their role (bottom warp:
// mailbox in, ring out; middle: ring in and out; top: ring in, mailbox out),
// which drops the role tests from the step: FP64 isolated 4-warp unit 584 ->
// 539 ns per step, 256^3 sweep 1.56 -> 1.52 ms, 512^3 with 8-warp units
// 4.29 -> 4.21 ms; FP32 (at prefetch depth 4) 256^3 sweep 1.03 -> 1.00 ms,
// 128^3 0.42 -> 0.38 ms.
template <typename T, int W>
constexpr bool kRoles = true;

template <typename T, int K, int W, int D, int RD>
__global__ void __launch_bounds__(W * 32, 1) gs27_cta_kernel(CtaArgs<T> a) {
    static_assert(K == 2, "one halo plane and one computed plane per warp");
    __shared__ int s_ticket;
    __shared__ unsigned s_tag;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    CtaShared<T, W>& sh = *reinterpret_cast<CtaShared<T, W>*>(dyn_smem);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tag = (unsigned)ld_relaxed_gpu(&a.ctrl[2]) + 1u;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&a.ctrl[0], 1);
        // ring tags from an earlier unit of this CTA could match a step of
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
            if constexpr (kRoles<T, W>) {
                if (warp == 0)
                    compute_warp<T, W, D, RD, 0>(a, t, warp, sh, s_tag);
                else if (warp == W - 1)
                    compute_warp<T, W, D, RD, 2>(a, t, warp, sh, s_tag);
                else
                    compute_warp<T, W, D, RD, 1>(a, t, warp, sh, s_tag);
            } else {
                compute_warp<T, W, D, RD, -1>(a, t, warp, sh, s_tag);
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

}  // namespace

// Shapes of the CTA wavefront per element type: K register slots per lane
// (one halo plane + K-1 computed planes) and the depth D of the input
// prefetch ring in steps, which is also the unrolling of the step loop.  The
// number W of compute warps per CTA is chosen at run time (4 or 8); D2 is
// the depth of levels above 128^3 points.  Measured on a GB300: FP64 runs
// fastest with D = 2 at every level size (a shorter unrolled loop, 1.79 vs
// 1.93 ms at 256^3).  FP32, whose warps run role-compiled copies of the
// step, with D = 4 at every size (256^3: 1.00 ms against 1.54 ms with
// D = 6, whose three copies no longer fit the instruction cache; without
// the copies D = 8 had measured 1.03 ms and D = 4 1.75 ms there).
template <typename T> struct CtaShape;
template <> struct CtaShape<double> { static constexpr int K = 2, D = 2, D2 = 2; };
template <> struct CtaShape<float> { static constexpr int K = 2, D = 4, D2 = 4; };

// Prefetch depth of a level: CtaShape::D, or CtaShape::D2 for FP32 levels of
// more than 128^3 points.
template <typename T>
int cta_depth(Dims d) {
    return (sizeof(T) == 4 && d.n > (i64)128 * 128 * 128) ? CtaShape<T>::D2 : CtaShape<T>::D;
}

template <typename T, int W>
size_t cta_smem_bytes() {
    return sizeof(CtaShared<T, W>);
}

template <typename T, int W, int D>
int cta_occupancy() {
    constexpr int K = CtaShape<T>::K;
    const size_t smem = cta_smem_bytes<T, W>();
    constexpr int R0 = sizeof(T) == 8 ? -1 : 0, R1 = sizeof(T) == 8 ? -1 : 1;
    cudaFuncSetAttribute(gs27_cta_kernel<T, K, W, D, R0>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(gs27_cta_kernel<T, K, W, D, R1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0, per_sm_rev = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gs27_cta_kernel<T, K, W, D, R0>,
                                                  W * 32, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_rev, gs27_cta_kernel<T, K, W, D, R1>,
                                                  W * 32, smem);
    per_sm = std::min(per_sm, per_sm_rev);
    return per_sm;
}

bool cta_warps_supported(int warps) { return warps == 4 || warps == 8; }

// The most units of W planes that the wavefront keeps busy at once on a
// level's problems (their units share one schedule, all starting at key 0):
// unit (U, V) of a problem has rows u in [30 U, 30 U + 30) and planes v in
// [W V, W V + W), computes when some row y = u - v lies in [0, ny), starts at
// the step 60 U + 2 W V of its schedule key and runs nx + 65 steps.
int cta_peak_units(const std::vector<Dims>& dims, int W) {
    std::vector<int> delta;
    for (const Dims& d : dims) {
        if (d.nx < 1 || d.ny < 1 || d.nz < 1) continue;
        const int NU = d.ny + d.nz - 1, NUc = (NU + 29) / 30, NVc = (d.nz + W - 1) / W;
        const int S = d.nx + 65;
        const long long kmax = 60LL * (NUc - 1) + 2LL * W * (NVc - 1);
        if (delta.size() < (size_t)(kmax + S + 1)) delta.resize((size_t)(kmax + S + 1), 0);
        for (int U = 0; U < NUc; ++U) {
            const int umin = 30 * U, umax = std::min(30 * U + 29, NU - 1);
            for (int V = 0; V < NVc; ++V) {
                const int vmin = W * V, vmax = std::min(W * V + W - 1, d.nz - 1);
                if (umax - vmin < 0 || umin - vmax > d.ny - 1) continue;
                const long long k = 60LL * U + 2LL * W * V;
                ++delta[(size_t)k];
                --delta[(size_t)(k + S)];
            }
        }
    }
    int run = 0, peak = 0;
    for (int v : delta) peak = std::max(peak, run += v);
    return peak;
}

// Default warps per unit (m2s_autotune_sweeps measures instead), one CTA per
// SM.  A lone warp on its sub-partition steps faster (FP64 unit-step 0.58 us
// with 4 warps, 0.76 us with 8 when no other unit feeds it), so 4-warp units
// win while the wavefront keeps the SMs short of work, and 8-warp units,
// which finish twice the points per SM and step, win once it has more ready
// units than SMs.  Measured FP64 sweeps on a GB300 (4 vs 8 warps): 256^3
// 1.57 vs 1.59 ms (peak of 197 busy 4-warp units), 320^3 2.18 vs 2.09 ms
// (285), 512^3 5.96 vs 4.33 ms, 1024^3 39.5 vs 25.0 ms; so FP64 levels take
// 4-warp units while their peak stays within 1.5 x the SMs.  FP32 levels
// take 8-warp units (256^3: 1.11 vs 1.30 ms).
int cta_default_warps(int dtype_is_f64, const std::vector<Dims>& dims) {
    if (!dtype_is_f64) return 8;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 8;
    return 2 * cta_peak_units(dims, 4) <= 3 * sms ? 4 : 8;
}

// Ghost units: warp 0 of unit (U, V) reads the plane sums G of the top plane
// of unit (U, V-1), published by that unit's top warp.  Where (U, V-1) has no
// valid row, the sums over the rows u0-2, u0-1 (the halo rows of the unit)
// can still be non-zero, so the unit is added: its rows compute nothing,
// its halo lanes and sums run and its top warp publishes G.
void add_ghost_units(int lanes, int planes, std::vector<int2>& org) {
    int NU = 0, NV = 0;
    for (const int2& o : org) {
        NU = std::max(NU, o.x / lanes + 1);
        NV = std::max(NV, o.y / planes + 1);
    }
    std::vector<char> has((size_t)NU * NV, 0);
    for (const int2& o : org) has[(size_t)(o.y / planes) * NU + o.x / lanes] = 1;
    const size_t n0 = org.size();
    for (size_t k = 0; k < n0; ++k) {
        const int U = org[k].x / lanes, V = org[k].y / planes;
        if (V >= 1 && !has[(size_t)(V - 1) * NU + U]) {
            has[(size_t)(V - 1) * NU + U] = 1;
            org.push_back(make_int2(U * lanes, (V - 1) * planes));
        }
    }
}

int cta_rz_partials_max(const std::vector<Dims>& dims) {
    int m = 0;
    for (int W : {4, 8}) {
        int tot = 0;
        for (const Dims& d : dims) {
            std::vector<int2> org;
            std::vector<int4> prod;
            build_units_host(30, 1, 1, W + 1, d, org, prod);
            add_ghost_units(30, W, org);
            tot += (int)org.size() * W;
        }
        m = std::max(m, tot);
    }
    return m;
}

// Unit table of one level for all problems of a grid (one launch per level).
// Within a problem the units are ordered by the step at which they can start
// on an idle GPU (the unit to the right lags 2*lanes steps, the unit above
// 2*planes); every producer (left, below, below-left) has a smaller key, so
// the order stays topological: a unit waits only on units with smaller
// tickets, which have started, and the sweep cannot deadlock.  Problems are
// independent, so their lists are merged by the same key and all problems
// advance together.
template <typename T>
cudaError_t build_cta_units(const std::vector<Dims>& dims, int W, WaveUnits* out) {
    constexpr int K = CtaShape<T>::K;
    if (!cta_warps_supported(W)) return cudaErrorInvalidValue;
    const int lanes = 30, planes = W * (K - 1);
    struct Item {
        long long key;
        int v0, problem, local;
        int2 org;
    };
    std::vector<Item> items;
    std::vector<int> rzpre(dims.size() + 1, 0);
    // per problem the first value of its slice of each mailbox
    std::vector<long long> mboff(2 * std::max<size_t>(dims.size(), 1), 0);
    i64 nbox = 0, ng = 0;
    for (size_t i = 0; i < dims.size(); ++i) {
        std::vector<int2> org;
        std::vector<int4> prod;
        build_units_host(lanes, 1, 1, planes + 1, dims[i], org, prod);
        add_ghost_units(lanes, planes, org);
        std::vector<Item> mine;
        for (const int2& o : org)
            mine.push_back(Item{2LL * lanes * (o.x / lanes) + 2LL * planes * (o.y / planes), o.y,
                                (int)i, 0, o});
        std::stable_sort(mine.begin(), mine.end(), [](const Item& a, const Item& b) {
            return a.key != b.key ? a.key < b.key : a.v0 < b.v0;
        });
        for (size_t k = 0; k < mine.size(); ++k) {
            mine[k].local = (int)k;
            items.push_back(mine[k]);
        }
        rzpre[i + 1] = rzpre[i] + (int)mine.size() * W;
        mboff[2 * i] = nbox;
        mboff[2 * i + 1] = ng;
        nbox += mbox_values(dims[i]);
        ng += mbg_values(dims[i], W);
    }
    const i64 wpv = sizeof(T) == 8 ? 2 : 1;  // mailbox words per value
    const i64 box_words = std::max<i64>(nbox, 1) * wpv;
    const i64 words = box_words + std::max<i64>(ng, 1) * wpv;
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) {
        if (a.key != b.key) return a.key < b.key;
        return a.problem != b.problem ? a.problem < b.problem : a.v0 < b.v0;
    });
    std::vector<int4> units(items.size());
    for (size_t k = 0; k < items.size(); ++k) {
        const Item& it = items[k];
        units[k] = make_int4(it.org.x, it.org.y, it.problem, rzpre[it.problem] + it.local * W);
    }
    WaveUnits u{};
    u.n_units = (int)units.size();
    u.W = W;
    u.stencil = 27;
    u.np = (int)dims.size();
    u.n_rz = rzpre.back();
    cudaError_t e;
    const size_t nu = std::max<size_t>(units.size(), 1);
    if ((e = cudaMalloc(&u.d_units, nu * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_dims, std::max<size_t>(dims.size(), 1) * sizeof(Dims))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_rzpre, rzpre.size() * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_ctrl, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_mboff, mboff.size() * sizeof(long long))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_mbox, (size_t)words * sizeof(u64))) != cudaSuccess) {
        free_wave_units(&u);
        return e;
    }
    if ((!units.empty() && (e = cudaMemcpy(u.d_units, units.data(), units.size() * sizeof(int4),
                                           cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (!dims.empty() && (e = cudaMemcpy(u.d_dims, dims.data(), dims.size() * sizeof(Dims),
                                          cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(u.d_rzpre, rzpre.data(), rzpre.size() * sizeof(int),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(u.d_mboff, mboff.data(), mboff.size() * sizeof(long long),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(u.d_ctrl, 0, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(u.d_mbox, 0, (size_t)words * sizeof(u64))) != cudaSuccess) {
        free_wave_units(&u);
        return e;
    }
    u.mb_words = box_words;
    // the prefetch depth follows the largest problem of the level
    Dims big{};
    for (const Dims& d : dims)
        if (d.n > big.n) big = d;
    u.K = K;
    u.depth = cta_depth<T>(big);
    constexpr int D1 = CtaShape<T>::D, D2 = CtaShape<T>::D2;
    const int per_sm = W == 4 ? (u.depth == D1 ? cta_occupancy<T, 4, D1>() : cta_occupancy<T, 4, D2>())
                              : (u.depth == D1 ? cta_occupancy<T, 8, D1>() : cta_occupancy<T, 8, D2>());
    // One CTA per SM: units that share an SM share its FP64 pipes and issue
    // slots, and the unit on the critical path then steps slower (256^3 FP64
    // with 4-warp units: 1.69 ms at one CTA per SM, 2.14 ms at two).
    u.grid = per_sm > 0 ? wave_grid(u.n_units, 1) : 0;
    if (u.grid == 0) {
        free_wave_units(&u);
        return cudaErrorInvalidConfiguration;
    }
    *out = u;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gs27_cta(const WaveUnits& u, const WaveCall& c, const T* Qin, T* Qout,
                            const T* b, T* x, cudaStream_t st) {
    constexpr int K = CtaShape<T>::K, D1 = CtaShape<T>::D, D2 = CtaShape<T>::D2;
    if (u.n_units == 0) return cudaSuccess;
    CtaArgs<T> a;
    a.rev = c.rev;
    a.spin_ns = c.spin_ns;
    a.Qin = Qin;
    a.Qout = Qout;
    a.b = b;
    a.x = x;
    a.units = u.d_units;
    a.dims = u.d_dims;
    a.n_units = u.n_units;
    a.ctrl = u.d_ctrl;
    a.status = c.status;
    a.rz = c.rz_partials;
    a.stall_unit = c.stall_unit;
    a.mbox = u.d_mbox;
    a.mbg = u.d_mbox + u.mb_words;
    a.mboff = u.d_mboff;
    const bool d1 = u.depth == D1;
    if (u.W != 4 && u.W != 8) return cudaErrorInvalidValue;
    // FP64: one kernel for both directions; FP32: one per direction
    constexpr int R0 = sizeof(T) == 8 ? -1 : 0, R1 = sizeof(T) == 8 ? -1 : 1;
#define M2S_GS27(Wv, Dv)                                                                      \
    (c.rev ? gs27_cta_kernel<T, K, Wv, Dv, R1><<<u.grid, Wv * 32, cta_smem_bytes<T, Wv>(), st>>>(a) \
           : gs27_cta_kernel<T, K, Wv, Dv, R0><<<u.grid, Wv * 32, cta_smem_bytes<T, Wv>(), st>>>(a))
    if (u.W == 4 && d1)
        M2S_GS27(4, D1);
    else if (u.W == 4)
        M2S_GS27(4, D2);
    else if (d1)
        M2S_GS27(8, D1);
    else
        M2S_GS27(8, D2);
#undef M2S_GS27
    return cudaGetLastError();
}

template cudaError_t build_cta_units<double>(const std::vector<Dims>&, int, WaveUnits*);
template cudaError_t build_cta_units<float>(const std::vector<Dims>&, int, WaveUnits*);
template cudaError_t launch_gs27_cta<double>(const WaveUnits&, const WaveCall&, const double*,
                                             double*, const double*, double*, cudaStream_t);
template cudaError_t launch_gs27_cta<float>(const WaveUnits&, const WaveCall&, const float*,
                                            float*, const float*, float*, cudaStream_t);

}  // namespace m2s
