// Application of the ILU(0) factors of the 27-point HPCG matrix (the
// incomplete LU preconditioner of paper Sec. 1; the ILU micro-benchmark of
// Sec. 7.2.1) as two persistent wavefront launches.
//
// The forward substitution y_p = r_p - sum_{q lower} l_pq y_q and the
// backward one z_p = (y_p - sum_{q upper} u_pq z_q) / u_pp have the
// dependence of the lexicographic Gauss-Seidel sweep, so they run on the
// CTA wavefront of k_wave2.cu: the same units (30 rows u = y + z by W planes
// v = z, tickets in topological order), the same tagged mailboxes and
// shared-memory rings, the same bounded waits.  The backward substitution
// is a forward one in the reflected index space (point p <-> n - 1 - p),
// with the upper factors stored at the reflected offsets: one kernel serves
// both triangles, each point scaling its sum by a per-point factor (1, or
// the pivot's rounded reciprocal).
//
// What differs from the sweep: the weights are per point, so no separable
// sum applies.  A lane keeps windows of the last three values of the row
// below it (x - 1, x, x + 1: one shuffle per step) and of the three rows of
// the plane below (rows u - 2, u - 1, u of the warp below, from its ring, or
// for warp 0 from the top plane of the unit underneath, read from a
// mailbox of full rows), and forms the 13-term sum in two chains.  Each
// point's 13 weights and its scale sit in one 128-byte record (seven 16-byte
// loads into registers two steps ahead, asked of L2 six steps ahead).
#include <algorithm>
#include <climits>
#include <vector>

#include "m2s_cta.cuh"
#include "m2s_internal.cuh"
#include "m2s_wave_sync.cuh"

namespace m2s {

namespace {

using namespace wave;
using namespace cta;

constexpr int kW = 4;  // warps (planes) per unit
constexpr int kD = 2;  // prefetch depth in steps (the unroll of the step loop)
constexpr int kRec = 16;  // doubles per weight record: 13 weights, the scale, 2 pad
constexpr int kUsed = 14;  // record entries read
constexpr int kL2 = 6;     // steps ahead that a lane asks L2 for its record and input

// Mailbox row geometry of build_cta_units (k_wave2.cu): rows u = y + z of a
// plane, 30 per unit column; the row mailbox holds the rows u mod 30 = 28, 29
// of every plane, the plane mailbox full rows of the planes v = W m - 1.
__device__ __forceinline__ int mb_rows_u(int ny, int nz) { return ny + nz - 1; }
__device__ __forceinline__ int mb_cols(int ny, int nz) { return (mb_rows_u(ny, nz) - 1) / 30 + 1; }

struct IluArgs {
    int rev;
    long long spin_ns;
    const double* Wt;  // [n][16] weight records (packed over problems)
    const double* in;  // forward: r; backward: y (held in out)
    double* out;       // y, then z
    const int4* units;
    const Dims* dims;
    int n_units;
    int* ctrl;
    DevStatus* status;
    u64* mbox;  // tagged x of the rows the unit to the right replays
    u64* mbt;   // tagged x of the top plane of every unit, full rows
    const long long* mboff;
    int stall_unit;  // test hook: this unit neither computes nor publishes (-1: none)
};

template <int W, int ROLE>
__device__ __forceinline__ void ilu_warp(const IluArgs& a, int t, int w, CtaShared<double, W>& sh,
                                         unsigned tag) {
    typedef Tagged<double>::W TW;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int4 un = a.units[t];
    const Dims dd = a.dims[un.z];
    const int v1 = un.y + w;
    const int u = un.x - 2 + lane;
    const int tbase = 2 * (un.x - 2) + 2 * (v1 - 1);
    const bool halo = lane < 2;
    // ROLE (compile time): 0 the bottom warp, 1 a middle one, 2 the top one
    const bool ring_in = ROLE != 0;
    const bool ring_out = ROLE != 2;
    const bool mb_out = !halo && lane >= 30;
    const int nx = dd.nx;
    const int y1 = u - v1;
    const bool rv1 = v1 < dd.nz && y1 >= 0 && y1 < dd.ny;
    const i64 dir = a.rev ? -1 : 1;
    const i64 r1 = ((i64)v1 * dd.ny + y1) * nx;
    const i64 L1 = a.rev ? dd.n - 1 - r1 : r1;  // problem-local point of x = 0
    const i64 rx = a.rev ? nx - 1 : 0;           // mailbox position of x = 0
    const int NU = mb_rows_u(dd.ny, dd.nz);
    const i64 mrow = (u >= 0 && (halo || mb_out))
                         ? (((i64)v1 * mb_cols(dd.ny, dd.nz) + u / 30) * 2 + (u % 30 - 28)) * nx
                         : 0;
    u64* const mbox = a.mbox + a.mboff[2 * un.z] * 2;
    u64* const mbt = a.mbt + a.mboff[2 * un.z + 1] * 2;
    u64* const mbox_p = mbox + (mrow + rx - L1) * 2;  // tagged words of point p at [2p], [2p+1]
    // the top warp publishes its rows for warp 0 of the unit above
    const bool t_out = ROLE == 2 && !halo && rv1 && v1 + 1 < dd.nz;
    u64* const tout = mbt + (t_out ? ((i64)((v1 + 1) / W) * NU + u) * nx + rx : 0) * 2;
    // warp 0 reads rows u - 2 + j (j = 0, 1, 2) of plane v1 - 1 there
    bool pj[3];
    const u64* tin[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int uj = u - 2 + j, yj = uj - (v1 - 1);
        pj[j] = !ring_in && !halo && rv1 && v1 >= 1 && yj >= 0 && yj < dd.ny;
        tin[j] = mbt + (pj[j] ? ((i64)(v1 / W) * NU + uj) * nx + rx : 0) * 2;
    }
    const double* Wt = a.Wt + dd.off * kRec;
    const double* In = a.in + dd.off;
    double* Out = a.out + dd.off;
    const int S = nx + 2 * 31 + 3;

    // prefetch ring: the weight record and input of the lane's point
    // (computing lanes), the replayed row's words (halo lanes), the plane
    // below's words at x + 1 (warp 0)
    double rw[kD][kUsed], rin[kD];
    u64 rh[kD][2], rt[kD][3][2];
    auto fetch = [&](int k, int x1) {
        const bool in = rv1 && (unsigned)x1 < (unsigned)nx;
        const i64 p = L1 + dir * x1;
        if (in && !halo) {
            const double2* rec = reinterpret_cast<const double2*>(Wt + p * kRec);
#pragma unroll
            for (int q = 0; q < kUsed / 2; ++q) {
                const double2 v = __ldg(rec + q);
                rw[k][2 * q] = v.x;
                rw[k][2 * q + 1] = v.y;
            }
            rin[k] = In[p];
        } else {
#pragma unroll
            for (int q = 0; q < kUsed; ++q) rw[k][q] = 0.0;
            rin[k] = 0.0;
        }
        rh[k][0] = rh[k][1] = 0;
        if (in && halo) {
            rh[k][0] = ld_relaxed_u64(mbox_p + 2 * p);
            rh[k][1] = ld_relaxed_u64(mbox_p + 2 * p + 1);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            rt[k][j][0] = rt[k][j][1] = 0;
            if (pj[j] && (unsigned)(x1 + 1) < (unsigned)nx) {
                const u64* q = tin[j] + 2 * dir * (x1 + 1);
                rt[k][j][0] = ld_relaxed_u64(q);
                rt[k][j][1] = ld_relaxed_u64(q + 1);
            }
        }
    };
#pragma unroll
    for (int k = 0; k < kD; ++k) fetch(k, k - 2 * lane - 2);

    // windows: the row below at x - 1, x, x + 1, the plane below's rows at
    // x - 1, x, x + 1, and this row's previous value
    double B0 = 0, B1 = 0, B2 = 0, P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, xm1 = 0;
    bool ok = true;
    int cachedC = -(1 << 30);
    auto step = [&](int s, int k) {
        const int x1 = s - 2 * lane - 2;
        const int tnow = s + tbase;
        const double* wt = rw[k];
        const double inv = rin[k];
        const TW hw{rh[k][0], rh[k][1]};
        TW tw[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) tw[j] = TW{rt[k][j][0], rt[k][j][1]};
        const bool in1 = rv1 && (unsigned)x1 < (unsigned)nx;
        const bool comp = in1 && !halo;
        // the newest values of the plane below (x + 1 of rows u - 2 + j),
        // needed wherever x + 1 is in the row (also at x = -1, whose window
        // feeds x = 0), and the replayed x of the halo lanes
        const bool needp = rv1 && !halo && (unsigned)(x1 + 1) < (unsigned)nx;
        double pn[3] = {0.0, 0.0, 0.0}, xmb = 0.0;
        bool okj[3] = {true, true, true}, okh = true;
        // Everything that needs only earlier steps is issued before the wait
        // and overlaps it: the row below at x + 1 (what the lane below
        // computed last step), the window shifts, and the ten terms of the
        // sum over values already held (the two older columns of the plane
        // below, the row below, x - 1).  After the wait only the plane
        // below's newest column (three FMAs) remains.  Record offsets
        // k = (dz+1) 9 + (dy+1) 3 + (dx+1) in the sweep's space.
        const double bn = __shfl_up_sync(FULL, xm1, 1);
        B0 = B1;
        B1 = B2;
        B2 = bn;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            P[j][0] = P[j][1];
            P[j][1] = P[j][2];
        }
        double t0 = fma(-wt[0], P[0][0], inv);
        t0 = fma(-wt[1], P[0][1], t0);
        t0 = fma(-wt[3], P[1][0], t0);
        t0 = fma(-wt[4], P[1][1], t0);
        double t1 = -wt[6] * P[2][0];
        t1 = fma(-wt[7], P[2][1], t1);
        t1 = fma(-wt[9], B0, t1);
        t1 = fma(-wt[10], B1, t1);
        t1 = fma(-wt[11], B2, t1);
        t1 = fma(-wt[12], xm1, t1);
        const TW* re[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            re[j] = ring_in ? &sh.ring[w - 1][(tnow - 5 + 2 * j) & (RING - 1)][lane - 2 + j] : nullptr;
            if (ring_in) {
                if (needp)
                    okj[j] = Tagged<double>::unpack(*(volatile const TW*)re[j],
                                                    (unsigned)(tnow - 5 + 2 * j + BIAS), &pn[j]);
            } else if (needp && pj[j]) {
                okj[j] = Tagged<double>::unpack(tw[j], tag, &pn[j]);
            }
        }
        if (in1 && halo) okh = Tagged<double>::unpack(hw, tag, &xmb);
        if (!__all_sync(FULL, okh && okj[0] && okj[1] && okj[2])) {
            // poll: reload only what is missing; the abort word and the clock
            // once every 32 polls
            const i64 p = L1 + dir * x1;
            unsigned long long t0 = 0;
            for (int it = 1;; ++it) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (okj[j]) continue;
                    if (ring_in)
                        okj[j] = Tagged<double>::unpack(*(volatile const TW*)re[j],
                                                        (unsigned)(tnow - 5 + 2 * j + BIAS), &pn[j]);
                    else
                        okj[j] = Tagged<double>::unpack(
                            mb_load<double>(tin[j] + 2 * dir * (x1 + 1), 0), tag, &pn[j]);
                }
                if (!okh) okh = Tagged<double>::unpack(mb_load<double>(mbox_p, p), tag, &xmb);
                if (__all_sync(FULL, okh && okj[0] && okj[1] && okj[2])) break;
                if ((it & 31) == 0) {
                    const unsigned long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    int ab = 0;
                    if (lane == 0) ab = ld_relaxed_gpu(&a.status->abort);
                    if (__shfl_sync(FULL, ab, 0)) { ok = false; return; }
                    if ((long long)(now - t0) > a.spin_ns) {
                        if (lane == 0) {
                            atomicCAS(&a.status->err, 0, (int)M2S_ERR_TIMEOUT);
                            atomicExch(&a.status->abort, 1);
                        }
                        ok = false;
                        return;
                    }
                }
            }
        }
        // the plane below's newest column, then in - sum of the 13 weighted
        // lower neighbours, times the point's scale
#pragma unroll
        for (int j = 0; j < 3; ++j) P[j][2] = pn[j];
        t0 = fma(-wt[2], P[0][2], t0);
        t0 = fma(-wt[5], P[1][2], t0);
        t1 = fma(-wt[8], P[2][2], t1);
        const double acc = (t0 + t1) * wt[13];
        const double X = comp ? acc : (in1 && halo ? xmb : 0.0);
        // the slot's inputs are used: refill it for step s + kD (from L2,
        // where the record and input of step s + kL2 are asked for now)
        fetch(k, x1 + kD);
        if (rv1 && !halo && (unsigned)(x1 + kL2) < (unsigned)nx) {
            const i64 pf = L1 + dir * (x1 + kL2);
            prefetch_l2(Wt + pf * kRec);
            prefetch_l2(In + pf);
        }
        const i64 p = L1 + dir * x1;
        if (comp) {
            Out[p] = X;
            if (mb_out) mb_store<double>(mbox_p, p, X, tag);
            if (t_out) mb_store<double>(tout + 2 * dir * x1, 0, X, tag);
        }
        xm1 = X;
        if (ring_out) {
            // back-pressure: the warp above still reads entries down to its
            // step's tnow - 5; entry tnow - RING may be overwritten once the
            // warp above has finished the step with tnow >= that entry + 5
            const int old_entry = tnow - RING;
            if (old_entry >= tbase && old_entry + 5 > cachedC) {
                int c = 0, okk = 1;
                if (lane == 0) {
                    const unsigned long long tt = global_ns();
                    for (;;) {
                        c = sh.prog[w + 1];
                        if (c >= old_entry + 5) break;
                        if (ld_relaxed_gpu(&a.status->abort) ||
                            (long long)(global_ns() - tt) > a.spin_ns) {
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
            sh.ring[w][tnow & (RING - 1)][lane] = Tagged<double>::pack(X, (unsigned)(tnow + BIAS));
        }
        __syncwarp();
        if (lane == 0) sh.prog[w] = tnow;
    };
    for (int s0 = 0; ok && s0 < S; s0 += kD) {
#pragma unroll
        for (int k = 0; k < kD; ++k)
            if (ok) step(s0 + k, k);
    }
    __syncwarp();
    if (lane == 0) sh.prog[w] = INT_MAX;
}

template <int W>
__global__ void __launch_bounds__(W * 32, 1) ilu_cta_kernel(IluArgs a) {
    __shared__ int s_ticket;
    __shared__ unsigned s_tag;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    CtaShared<double, W>& sh = *reinterpret_cast<CtaShared<double, W>*>(dyn_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_tag = (unsigned)ld_relaxed_gpu(&a.ctrl[2]) + 1u;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&a.ctrl[0], 1);
        // ring tags of an earlier unit of this CTA could match: clear
        for (int i = threadIdx.x; i < W * RING * 32; i += blockDim.x)
            (&sh.ring[0][0][0])[i] = Tagged<double>::zero();
        if (threadIdx.x < W) sh.prog[threadIdx.x] = -(1 << 30);
        __syncthreads();
        const int t = s_ticket;
        if (t >= a.n_units) break;
        // a unit without a computing row (a ghost unit of the sweep's table)
        // produces nothing anyone reads: skip it
        const int4 un = a.units[t];
        const Dims dd = a.dims[un.z];
        const int v1 = un.y + warp, y1 = un.x - 2 + lane - v1;
        const int mine = lane >= 2 && v1 < dd.nz && y1 >= 0 && y1 < dd.ny;
        int ab = 0;
        if (threadIdx.x == 0) ab = ld_relaxed_gpu(&a.status->abort) || t == a.stall_unit;
        const int any = __syncthreads_or(mine);
        ab = __syncthreads_or(ab);
        // each warp runs a copy of the step compiled for its role
        if (any && !ab) {
            if (warp == 0)
                ilu_warp<W, 0>(a, t, warp, sh, s_tag);
            else if (warp == W - 1)
                ilu_warp<W, 2>(a, t, warp, sh, s_tag);
            else
                ilu_warp<W, 1>(a, t, warp, sh, s_tag);
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

// Weight records from the factors F[p][27] (box offsets o; o < 13 L, 13 the
// pivot, o > 13 U) and the pivots' reciprocals: forward record k = o (k <
// 13), scale 1; backward record k = 26 - o (the upper offsets reflected),
// scale 1 / u_pp.
__global__ void ilu_records_kernel(i64 n, const double* __restrict__ F,
                                   const double* __restrict__ Finv, double* __restrict__ Lw,
                                   double* __restrict__ Uw) {
    const i64 p = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double* f = F + 27 * p;
    double* l = Lw + kRec * p;
    double* uu = Uw + kRec * p;
    for (int k = 0; k < 13; ++k) {
        l[k] = f[k];
        uu[k] = f[26 - k];
    }
    l[13] = 1.0;
    uu[13] = Finv[p];
    l[14] = l[15] = uu[14] = uu[15] = 0.0;
}

// One unit per SM: a unit's 4 warps then have an FP64 pipe each (a GB300
// sub-partition issues one FP64 warp instruction per ~32 ns, and a step
// issues 15); co-resident units would share the pipes and slow every unit
// on the critical path.  The launch asks for more shared memory than half an
// SM holds so that no second CTA fits.
constexpr size_t kIluSmem = 120 * 1024;
static_assert(sizeof(CtaShared<double, kW>) <= kIluSmem, "ring fits the padded allocation");

int ilu_grid(int n_units) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(ilu_cta_kernel<kW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kIluSmem);
        attr = true;
    }
    return wave_grid(n_units, 1);
}

}  // namespace

cudaError_t ilu_wave_setup(const std::vector<Dims>& dims, i64 n, const double* F,
                           const double* Finv, double* Lw, double* Uw, WaveUnits* units,
                           cudaStream_t st) {
    if (n > 0) {
        ilu_records_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, F, Finv, Lw, Uw);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (units->d_units) return cudaSuccess;
    cudaError_t e = build_cta_units<double>(dims, kW, units);
    if (e != cudaSuccess) return e;
    units->grid = ilu_grid(units->n_units);
    return cudaSuccess;
}

cudaError_t launch_ilu_wave(const WaveUnits& u, int rev, long long spin_ns, DevStatus* status,
                            const double* Wt, const double* in, double* out, int stall_unit,
                            cudaStream_t st) {
    if (u.n_units == 0) return cudaSuccess;
    IluArgs a;
    a.rev = rev;
    a.spin_ns = spin_ns;
    a.Wt = Wt;
    a.in = in;
    a.out = out;
    a.units = u.d_units;
    a.dims = u.d_dims;
    a.n_units = u.n_units;
    a.ctrl = u.d_ctrl;
    a.status = status;
    a.mbox = u.d_mbox;
    a.mbt = u.d_mbox + u.mb_words;
    a.mboff = u.d_mboff;
    a.stall_unit = stall_unit;
    ilu_cta_kernel<kW><<<u.grid, kW * 32, kIluSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace m2s
