// 5x5-block 7-point operator in the shape of NPB-LU and its SSOR step
// (paper Sec. 1 and Sec. 4.3.3: SSOR among the routines with spatial
// dependence; Sec. 4.2.3: inner values are 5-vectors and 5x5 blocks).
//
// One SSOR step from u (Saad, Iterative Methods, Sec. 4.1.2):
//   s = D^-1 (b - A u)                       Jacobi-style, fully parallel
//   lower, p increasing:  v_p = s_p - sum_d M_{p,d} v_{p-e_d},  M = w D^-1 L
//   upper, p decreasing:  w_p = v_p - sum_d N_{p,d} w_{p+e_d},  N = w D^-1 U
//   u += w(2-w) w_p      (fused into the upper sweep)
// which is (D + wL) v = r and (D + wU) w = D v with D^-1 applied once per
// point per step instead of one 5x5 elimination per point per sweep: the
// products w D^-1 L and w D^-1 U are formed once per omega at set-up.
// Where the blocks are formed from u every step (op BLOCK7_JAC, below), the
// products are not formed at all: the sweeps apply w D^-1 themselves.
//
// The sweeps run on the wavefront machinery of k_wave.cu (hyperplane
// x + y + z, one progress counter per unit, ticketed units), with FIVE lanes
// per grid point -- lane c computes component c -- so that a wavefront step
// costs 15 FMAs per lane instead of 75 (the FP64 pipe of a GB300 SM
// sub-partition retires one warp instruction per ~32 ns whatever the
// number of active lanes).  A warp holds 6 point rows in y (group 0 is the
// halo row replayed from the producer) and K register slots in z.
#include <algorithm>

#include <climits>

#include "m2s_block.cuh"
#include "m2s_bounds.cuh"
#include "m2s_cta.cuh"
#include "m2s_wave_sync.cuh"

namespace m2s {

namespace {

using namespace wave;


__device__ __forceinline__ void coords(i64 i, int nx, int ny, int* x, int* y, int* z) {
    *x = (int)(i % nx);
    const i64 r = i / nx;
    *y = (int)(r % ny);
    *z = (int)(r / ny);
}

// In-place inverse of a 5x5 matrix by Gauss-Jordan elimination without
// pivoting (the blocks are diagonally dominant).
__device__ void inv5(const double* a, double* out) {
    double m[5][10];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            m[i][j] = a[i * 5 + j];
            m[i][5 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int k = 0; k < 5; ++k) {
        const double piv = 1.0 / m[k][k];
        for (int j = 0; j < 10; ++j) m[k][j] *= piv;
        for (int i = 0; i < 5; ++i) {
            if (i == k) continue;
            const double f = m[i][k];
            for (int j = 0; j < 10; ++j) m[i][j] -= f * m[k][j];
        }
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) out[i * 5 + j] = m[i][5 + j];
}

// The stored blocks of op BLOCK7_5x5 are kept entry-major ("structure of
// arrays"): entry k of the blocks of point p at [k][npts] (D, D^-1: k < 25;
// L, U: k = d * 25 + r * 5 + c < 75), so that one thread per point reads
// every entry with one coalesced warp access (32 consecutive points, 256 B)
// instead of 8-byte words 200-600 B apart.  block_to_soa_kernel makes the
// copies from the caller's point-major arrays at creation.
__global__ void block_to_soa_kernel(i64 n, i64 npts, i64 off, int nent,
                                    const double* __restrict__ src, double* __restrict__ dst) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < nent; ++k) dst[(i64)k * npts + off + i] = src[i * nent + k];
}

// D^-1 (entry-major, for the residual) and the products M = w D^-1 L,
// N = w D^-1 U (point-major, for the sweeps' five lanes per point).
__global__ void block_setup_kernel(Dims d, i64 npts, const double* __restrict__ D,
                                   const double* __restrict__ L, const double* __restrict__ U,
                                   double omega, double* __restrict__ Dinv,
                                   double* __restrict__ M, double* __restrict__ N) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 p = d.off + i;
    double dp[25], di[25];
    for (int k = 0; k < 25; ++k) dp[k] = D[(i64)k * npts + p];
    inv5(dp, di);
    for (int k = 0; k < 25; ++k) Dinv[(i64)k * npts + p] = di[k];
    const bool lo[3] = {x > 0, y > 0, z > 0};
    const bool hi[3] = {x < d.nx - 1, y < d.ny - 1, z < d.nz - 1};
    for (int dd = 0; dd < 3; ++dd) {
        const double* Lb = L + (i64)(dd * 25) * npts + p;
        const double* Ub = U + (i64)(dd * 25) * npts + p;
        for (int r = 0; r < 5; ++r)
            for (int c = 0; c < 5; ++c) {
                double sl = 0.0, su = 0.0;
                for (int k = 0; k < 5; ++k) {
                    sl = fma(di[r * 5 + k], Lb[(i64)(k * 5 + c) * npts], sl);
                    su = fma(di[r * 5 + k], Ub[(i64)(k * 5 + c) * npts], su);
                }
                M[(p * 3 + dd) * 25 + r * 5 + c] = lo[dd] ? omega * sl : 0.0;
                N[(p * 3 + dd) * 25 + r * 5 + c] = hi[dd] ? omega * su : 0.0;
            }
    }
}

// y = A u, or (resid) s = D^-1 (b - A u).  One thread per point, the blocks
// entry-major (coalesced across the warp); the 5-vectors of u point-major.
template <bool RESID>
__global__ void __launch_bounds__(128) block_apply_kernel(
    Dims d, i64 npts, const double* __restrict__ D, const double* __restrict__ L,
    const double* __restrict__ U, const double* __restrict__ Dinv, const double* __restrict__ b,
    const double* __restrict__ u, double* __restrict__ out) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 p = d.off + i;
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    double acc[5] = {0, 0, 0, 0, 0};
    // B: entry 0 of the block at this point; entry k at B[k * npts]
    auto mv = [&](const double* B, i64 q) {
        if (!M2S_IN(q - d.off, d.n)) return;
        const double* uq = u + q * 5;
        double v[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c] = uq[c];
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[r] = fma(B[(i64)(r * 5 + c) * npts], v[c], acc[r]);
    };
    if (z > 0) mv(L + (i64)50 * npts + p, p - sz);
    if (y > 0) mv(L + (i64)25 * npts + p, p - sy);
    if (x > 0) mv(L + p, p - 1);
    mv(D + p, p);
    if (x < d.nx - 1) mv(U + p, p + 1);
    if (y < d.ny - 1) mv(U + (i64)25 * npts + p, p + sy);
    if (z < d.nz - 1) mv(U + (i64)50 * npts + p, p + sz);
    if constexpr (!RESID) {
#pragma unroll
        for (int r = 0; r < 5; ++r) out[p * 5 + r] = acc[r];
        return;
    } else {
        double rr[5];
#pragma unroll
        for (int r = 0; r < 5; ++r) rr[r] = b[p * 5 + r] - acc[r];
        const double* Di = Dinv + p;
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < 5; ++c) s = fma(Di[(i64)(r * 5 + c) * npts], rr[c], s);
            out[p * 5 + r] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Blocks formed from the state (the NPB-LU situation of paper Sec. 1 and
// Sec. 4.2.3: the 5x5 blocks of an SSOR step are Jacobians evaluated at the
// current u and change every step).  Parameters, per problem, JP doubles:
// sigma, nu, then for k = 0..3 (point term, x, y, z) C_k (5x5), E_k (5x5),
// g_k (5).  With J_k(q) = C_k + (g_k . q) E_k + (E_k q) g_k^T, the Jacobian
// of the flux F_k(q) = C_k q + (g_k . q) E_k q:
//   D_p = sigma I + J_0(u_p),  L_{p,d} = -nu I - J_{d+1}(u_{p-e_d}) / 2,
//   U_{p,d} = -nu I + J_{d+1}(u_{p+e_d}) / 2   (0 where they leave the grid).
// Each Jacobian J_d(u_q) (d = x, y, z) serves two blocks, L_{q+e_d,d} and
// U_{q-e_d,d}, so the forming pass scatters: the thread of point q forms
// J_0(u_q) and its three J_d(u_q) once, writes the two blocks of each into
// the slots of q + e_d and q - e_d (zero where no neighbour writes a slot),
// w D_q^-1, the flux products h_d(q) = J_d(u_q) u_q and b_q - D_q u_q.  A
// second, memory-bound pass assembles the residual from them,
//   r_p = b_p - D_p u_p + sum_d [nu (u_{p-e_d} + u_{p+e_d})
//                                + h_d(p-e_d) / 2 - h_d(p+e_d) / 2],
// since L_{p,d} u_{p-e_d} = -nu u_{p-e_d} - h_d(p-e_d) / 2 (and U likewise).
// The sweeps then apply w D^-1 to their neighbour sums (the DI form of
// block_warp): forming the products w D^-1 L and w D^-1 U here would cost
// 750 more FP64 operations per point in a pass bound by the FP64 pipe.  No
// block outlives its step.  The operator apply y = A(u) u (block_jac_apply
// kernel) gathers instead: one thread forms the seven blocks of its point.
// ---------------------------------------------------------------------------
constexpr int JB = 128;  // threads per CTA of the block-forming kernel

// B = sj * J_k(q) + dj I, Pk = the 55 parameters of flux k (shared memory)
__device__ __forceinline__ void jac_form(const double* Pk, const double* q, double sj, double dj,
                                         double* B) {
    const double* C = Pk;
    const double* E = Pk + 25;
    const double* g = Pk + 50;
    double gq = 0.0;
#pragma unroll
    for (int j = 0; j < 5; ++j) gq = fma(g[j], q[j], gq);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        double eq = 0.0;
#pragma unroll
        for (int j = 0; j < 5; ++j) eq = fma(E[i * 5 + j], q[j], eq);
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const double J = fma(eq, g[j], fma(gq, E[i * 5 + j], C[i * 5 + j]));
            B[i * 5 + j] = i == j ? fma(sj, J, dj) : sj * J;
        }
    }
}

// In-place inverse of a 5x5 matrix, Gauss-Jordan without pivoting (the
// diagonal blocks are diagonally dominant): 125 FMAs and 5 reciprocals.
__device__ __forceinline__ void inv5_inplace(double* a) {
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double piv = 1.0 / a[k * 5 + k];
        a[k * 5 + k] = 1.0;
#pragma unroll
        for (int j = 0; j < 5; ++j) a[k * 5 + j] *= piv;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (i == k) continue;
            const double f = a[i * 5 + k];
            a[i * 5 + k] = 0.0;
#pragma unroll
            for (int j = 0; j < 5; ++j) a[i * 5 + j] = fma(-f, a[k * 5 + j], a[i * 5 + j]);
        }
    }
}

// y = A(u) u, the blocks of point p formed from u_p and its neighbours
__global__ void __launch_bounds__(JB) block_jac_apply_kernel(Dims d, const double* __restrict__ Pg,
                                                             const double* __restrict__ u,
                                                             double* __restrict__ out) {
    __shared__ double P[JP];
    for (int k = threadIdx.x; k < JP; k += blockDim.x) P[k] = Pg[k];
    __syncthreads();
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 p = d.off + i;
    const i64 st[3] = {1, d.nx, (i64)d.nx * d.ny};
    const bool lo[3] = {x > 0, y > 0, z > 0};
    const bool hi[3] = {x < d.nx - 1, y < d.ny - 1, z < d.nz - 1};
    double q[5], B[25], acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    auto add = [&](const double* Pk, i64 qi, double sj, double dj) {
        if (!M2S_IN(qi - d.off, d.n)) return;
#pragma unroll
        for (int c = 0; c < 5; ++c) q[c] = u[qi * 5 + c];
        jac_form(Pk, q, sj, dj, B);
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[r] = fma(B[r * 5 + c], q[c], acc[r]);
    };
    add(P + 2, p, 1.0, P[0]);
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        if (lo[dd]) add(P + 2 + 55 * (dd + 1), p - st[dd], -0.5, -P[1]);
        if (hi[dd]) add(P + 2 + 55 * (dd + 1), p + st[dd], 0.5, -P[1]);
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) out[p * 5 + r] = acc[r];
}

// Warp-wide store of W values per lane, staged in shared memory: each lane
// has put its values at sb[lane * W + k]; the lane's values go to
// dst[target + 0..W-1] (target < 0: nowhere).  The warp copies in runs of
// 32 consecutive values, so a store request covers a few contiguous runs
// instead of 32 scattered 8-byte words.
template <int W>
__device__ __forceinline__ void warp_flush(const double* __restrict__ sb, i64* __restrict__ tg,
                                           int lane, i64 target, double* __restrict__ dst) {
    tg[lane] = target;
    __syncwarp();
#pragma unroll
    for (int it = 0; it < W; ++it) {
        const int idx = it * 32 + lane;  // = pt * W + k
        const int pt = idx / W;
        const i64 t = tg[pt];
        if (t >= 0) dst[t + (idx - pt * W)] = sb[idx];
    }
    __syncwarp();
}

// The forming pass of an SSOR step (scatter form, see above).  Outputs:
// Lo/Up [n][3][25] the blocks L, U; Dinv [n][25] w D^-1; h [3][n][5] the
// flux products (one array per direction, so that the residual pass reads
// its neighbours' contiguously); w0 [n][5] b - D u.  Every lane of a warp
// takes part in its staged stores (lanes past the last point store nothing).
__global__ void __launch_bounds__(JB, 3) block_jac_form_kernel(Dims d, const double* __restrict__ Pg,
                                                               double omega,
                                                               const double* __restrict__ b,
                                                               const double* __restrict__ u,
                                                               double* __restrict__ Lo,
                                                               double* __restrict__ Up,
                                                               double* __restrict__ Dinv,
                                                               double* __restrict__ h, i64 nall,
                                                               double* __restrict__ w0) {
    __shared__ double P[JP];
    __shared__ double sbuf[JB / 32][32 * 25];
    __shared__ double hbuf[JB / 32][3][32 * 5];
    __shared__ i64 stgt[JB / 32][32];
    for (int k = threadIdx.x; k < JP; k += blockDim.x) P[k] = Pg[k];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    double* sb = sbuf[threadIdx.x >> 5];
    double(*hb)[32 * 5] = hbuf[threadIdx.x >> 5];
    i64* tg = stgt[threadIdx.x >> 5];
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    const bool valid = i < d.n;
    int x = 0, y = 0, z = 0;
    if (valid) coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 p = d.off + (valid ? i : 0);
    const i64 st[3] = {1, d.nx, (i64)d.nx * d.ny};
    const bool lo[3] = {x > 0, y > 0, z > 0};
    const bool hi[3] = {x < d.nx - 1, y < d.ny - 1, z < d.nz - 1};
    const double nu = P[1];
    double q[5], B[25];
#pragma unroll
    for (int c = 0; c < 5; ++c) q[c] = valid ? u[p * 5 + c] : 0.0;
    jac_form(P + 2, q, 1.0, P[0], B);  // D_p
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 5; ++c) s = fma(B[r * 5 + c], q[c], s);
        sb[lane * 5 + r] = (valid ? b[p * 5 + r] : 0.0) - s;
    }
    warp_flush<5>(sb, tg, lane, valid ? p * 5 : -1, w0);
    inv5_inplace(B);
#pragma unroll
    for (int k = 0; k < 25; ++k) sb[lane * 25 + k] = omega * B[k];
    warp_flush<25>(sb, tg, lane, valid ? p * 25 : -1, Dinv);
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        jac_form(P + 2 + 55 * (dd + 1), q, 1.0, 0.0, B);  // J_d(u_p)
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < 5; ++c) s = fma(B[r * 5 + c], q[c], s);
            hb[dd][lane * 5 + r] = s;
        }
        // L of the point above in d reads u_p; so does U of the point below
        // (each slot has exactly one writer)
#pragma unroll
        for (int k = 0; k < 25; ++k) sb[lane * 25 + k] = fma(-0.5, B[k], k % 6 == 0 ? -nu : 0.0);
        const bool lo_ok = valid && lo[dd] && M2S_IN(p - st[dd] - d.off, d.n);
        const bool hi_ok = valid && hi[dd] && M2S_IN(p + st[dd] - d.off, d.n);
        warp_flush<25>(sb, tg, lane, hi_ok ? ((p + st[dd]) * 3 + dd) * 25 : -1, Lo);
#pragma unroll
        for (int k = 0; k < 25; ++k) sb[lane * 25 + k] = fma(0.5, B[k], k % 6 == 0 ? -nu : 0.0);
        warp_flush<25>(sb, tg, lane, lo_ok ? ((p - st[dd]) * 3 + dd) * 25 : -1, Up);
        // the slots no neighbour writes: this point's own L (U) where the
        // grid ends below (above) it in d
        if (valid && !lo[dd]) {
            double* Zb = Lo + (p * 3 + dd) * 25;
#pragma unroll
            for (int k = 0; k < 25; ++k) Zb[k] = 0.0;
        }
        if (valid && !hi[dd]) {
            double* Zb = Up + (p * 3 + dd) * 25;
#pragma unroll
            for (int k = 0; k < 25; ++k) Zb[k] = 0.0;
        }
    }
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) warp_flush<5>(hb[dd], tg, lane, valid ? p * 5 : -1, h + dd * nall * 5);
}

// r / w at every point from the forming pass's outputs (memory-bound)
__global__ void block_jac_resid_kernel(Dims d, const double* __restrict__ u,
                                       const double* __restrict__ h, i64 nall,
                                       const double* __restrict__ w0, double nu, double iw,
                                       double* __restrict__ out) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 p = d.off + i;
    const i64 st[3] = {1, d.nx, (i64)d.nx * d.ny};
    const bool lo[3] = {x > 0, y > 0, z > 0};
    const bool hi[3] = {x < d.nx - 1, y < d.ny - 1, z < d.nz - 1};
    double acc[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) acc[r] = w0[p * 5 + r];
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        if (lo[dd] && M2S_IN(p - st[dd] - d.off, d.n)) {
            const i64 q = p - st[dd];
#pragma unroll
            for (int r = 0; r < 5; ++r)
                acc[r] = fma(0.5, h[(dd * nall + q) * 5 + r], fma(nu, u[q * 5 + r], acc[r]));
        }
        if (hi[dd] && M2S_IN(p + st[dd] - d.off, d.n)) {
            const i64 q = p + st[dd];
#pragma unroll
            for (int r = 0; r < 5; ++r)
                acc[r] = fma(-0.5, h[(dd * nall + q) * 5 + r], fma(nu, u[q * 5 + r], acc[r]));
        }
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) out[p * 5 + r] = acc[r] * iw;
}

// ---------------------------------------------------------------------------
// Block sweeps as a CTA wavefront (the design of the 7-point sweep in
// k_wave7.cu, with a group of five lanes per grid point).  A unit is a CTA of
// BW warps, warp w owning plane z = z0 + w; lane 5g + c of a warp holds
// component c of the point in row y = y0 - 1 + g (group 0 replays row y0 - 1
// of the unit to the left from its mailbox, groups 1-5 compute, lanes 30-31
// idle).  At local step s group g of warp w is at x = s - g - w: the whole
// CTA is on one hyperplane x + y + z.  The x - 1 neighbour is the group's own
// previous 5-vector, the y - 1 neighbour the group below one step earlier
// (shuffles), the z - 1 neighbour the warp below one step earlier (a tagged
// shared-memory ring) or, for warp 0, the top warp of the unit underneath
// (tagged mailbox).  Each lane then does 15 FMAs: its row of the three 5x5
// coupling blocks against the three neighbour vectors.  The backward sweep
// is the forward sweep in reflected index space with N in place of M.
// ---------------------------------------------------------------------------
constexpr int BW = 8;      // warps (planes) per unit
constexpr int BROWS = 5;   // computing rows (groups 1-5) per unit
constexpr int BD = 2;      // prefetch depth in steps
constexpr int BD_DI = 1;   // the same with D^-1 applied in the sweep

struct BlockCtaArgs {
    int rev;
    long long spin_ns;
    const double* coup;  // [n][3][25]: M (forward) or N (backward)
    const double* rhs;   // [n][5]: s (forward) or v (backward)
    double* out;         // [n][5]: v or w
    double* u;           // backward only: u += cu * w  (may be NULL)
    double cu;
    const int4* units;   // (y0, z0, problem, 0) in ticket order
    const Dims* dims;
    int n_units;
    int* ctrl;
    DevStatus* status;
    int stall_unit;
    cta::u64* mbox;      // per point and component one tagged value (2 words)
    const double* dinv;  // DI form only: [n][25] w D^-1 (coup then holds L or U)
};

struct BlockShared {
    cta::Tagged<double>::W ring[BW][cta::RING][32];
    volatile int prog[BW];
};

// DI = false: coup holds M = w D^-1 L (N = w D^-1 U) and a step is
//   v_p = s_p - sum_d M_{p,d} v_{p-e_d}   (w_p = v_p - sum_d N_{p,d} w_{p+e_d}).
// DI = true (blocks formed every step, so the products are not formed):
// coup holds L (U) itself, dinv holds w D^-1, the lower rhs r / w, and a
// step applies w D^-1 to the neighbour sum,
//   v_p = w D_p^-1 (r_p / w - sum_d L_{p,d} v_{p-e_d})
//   w_p = v_p - w D_p^-1 sum_d U_{p,d} w_{p+e_d},
// lane c taking row c of w D_p^-1 and the group's five sums by shuffles:
// 20 FP64 instructions per step against 15 for the product form.
template <bool DI, int PD, int ROLE>
__device__ __forceinline__ void block_warp(const BlockCtaArgs& a, int t, int w, BlockShared& sh,
                                           unsigned tag) {
    using namespace cta;
    typedef Tagged<double>::W TW;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int g = lane / 5, c = lane - 5 * (lane / 5);
    const int gb = 5 * (g < 6 ? g : 0);  // first lane of the group
    const int4 un = a.units[t];
    const Dims dm = a.dims[un.z];
    const int y = un.x - 1 + g;
    const int z = un.y + w;
    const bool lane_ok = g < 6;
    const bool halo = g == 0;
    const bool rv = lane_ok && y >= 0 && y < dm.ny && z < dm.nz;
    // ROLE: -1 read from w; 0 the bottom warp, 1 a middle one, 2 the top one
    const bool bottom = ROLE < 0 ? w == 0 : ROLE == 0;
    const bool topw = ROLE < 0 ? w == BW - 1 : ROLE == 2;
    const bool ring_in = !bottom, ring_out = !topw;
    const bool mb_out = lane_ok && !halo && (g == BROWS || topw);
    const bool zmb = bottom && z >= 1;
    const int nx = dm.nx;
    const i64 dir = a.rev ? -1 : 1;
    const i64 r = rv ? ((i64)z * dm.ny + y) * nx : 0;
    const i64 L = a.rev ? dm.n - 1 - r : r;  // problem-local point of x = 0
    const i64 szd = dir * (i64)nx * dm.ny;
    const double* C = a.coup + dm.off * 75;
    const double* R = a.rhs + dm.off * 5;
    double* O = a.out + dm.off * 5;
    double* U = a.u ? a.u + dm.off * 5 : nullptr;
    const double* Dv = DI ? a.dinv + dm.off * 25 : nullptr;
    u64* const mbox = a.mbox + dm.off * 10;  // 5 components x 2 words per point
    const int S = nx + BROWS + 1 + BW;

    // prefetch: the lane's rows of the three coupling blocks, its rhs
    // component and (backward sweep) its component of u (computing lanes),
    // its component of the replayed row (group 0), its component of the
    // plane below (warp 0).  u[p] is written only by this lane's own step at
    // p, so the value fetched PD steps ahead is the one the update needs.
    double pc[PD][15], pr[PD], pu[PD], pm0[PD], pm1[PD], pd[PD][DI ? 5 : 1];
    auto fetch = [&](int k, int s) {
        const int xx = s - g - w;
        const bool in = rv && (unsigned)xx < (unsigned)nx && M2S_IN(L + dir * xx, dm.n);
        const i64 p = L + dir * xx;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int j = 0; j < 5; ++j)
                pc[k][5 * d + j] = (in && !halo) ? __ldg(C + p * 75 + d * 25 + c * 5 + j) : 0.0;
        double m0 = 0.0, m1 = 0.0;
        if (in && halo) tw_to_regs(mb_load<double>(mbox, p * 5 + c), &m0, &m1);
        if (in && !halo && zmb && M2S_IN(p - szd, dm.n))
            tw_to_regs(mb_load<double>(mbox, (p - szd) * 5 + c), &m0, &m1);
        pr[k] = (in && !halo) ? __ldg(R + p * 5 + c) : 0.0;
        pu[k] = (in && !halo && U) ? U[p * 5 + c] : 0.0;
        if constexpr (DI) {
#pragma unroll
            for (int j = 0; j < 5; ++j) pd[k][j] = (in && !halo) ? __ldg(Dv + p * 25 + c * 5 + j) : 0.0;
        }
        pm0[k] = m0;
        pm1[k] = m1;
    };
#pragma unroll
    for (int k = 0; k < PD; ++k) fetch(k, k);

    double xprev = 0.0;  // this lane's component at the previous step
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
        const int xx = s - g - w;
        double cf[15];
#pragma unroll
        for (int j = 0; j < 15; ++j) cf[j] = pc[k][j];
        const double rh = pr[k], uo = pu[k], m0 = pm0[k], m1 = pm1[k];
        double di[DI ? 5 : 1];
#pragma unroll
        for (int j = 0; j < (DI ? 5 : 1); ++j) di[j] = pd[k][j];
        fetch(k, s + PD);
        const bool in = rv && (unsigned)xx < (unsigned)nx && M2S_IN(L + dir * xx, dm.n);
        const bool comp = in && !halo;
        double X = 0.0, zc = 0.0;
        bool okx = true, okz = true, okr = true;
        if (in && halo) okx = Tagged<double>::unpack(regs_to_tw(m0, m1), tag, &X);
        if (comp && zmb) okz = Tagged<double>::unpack(regs_to_tw(m0, m1), tag, &zc);
        // The x - 1 and y - 1 neighbours (the own group and the group below,
        // both from the previous step) need no wait: their ten FMAs are
        // issued before it and overlap it, and only the five of the z - 1
        // neighbour follow the wait.
        const int gy = g >= 1 && g < 6 ? gb - 5 : 0;
        double acc = DI && a.rev ? 0.0 : rh;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const double vx = __shfl_sync(FULL, xprev, gb + j);
            const double vy = __shfl_sync(FULL, xprev, gy + j);
            acc = fma(-cf[j], vx, acc);
            acc = fma(-cf[5 + j], vy, acc);
        }
        const TW* re = ring_in ? &sh.ring[w - 1][(s - 1) & (RING - 1)][lane] : nullptr;
        const unsigned rtag = (unsigned)(s - 1 + BIAS);
        if (ring_in && s >= 1) okr = Tagged<double>::unpack(*(volatile const TW*)re, rtag, &zc);
        if (!__all_sync(FULL, okx && okz && okr)) {
            const i64 p = L + dir * xx;
            unsigned long long t0 = 0;
            for (int it = 1;; ++it) {
                if (!okr) okr = Tagged<double>::unpack(*(volatile const TW*)re, rtag, &zc);
                if (!okx) okx = Tagged<double>::unpack(mb_load<double>(mbox, p * 5 + c), tag, &X);
                if (!okz && M2S_IN(p - szd, dm.n))
                    okz = Tagged<double>::unpack(mb_load<double>(mbox, (p - szd) * 5 + c), tag, &zc);
                if (__all_sync(FULL, okx && okz && okr)) break;
                if ((it & 31) == 0) {
                    const unsigned long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    if (fail()) { ok = false; return; }
                    if ((long long)(now - t0) > a.spin_ns) { timeout(); ok = false; return; }
                }
            }
        }
        // the z - 1 neighbour (warp below / unit underneath), continuing the
        // one chain (the sweep is bound by the FP64 instructions it issues,
        // so no extra partial sums)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const double vz = __shfl_sync(FULL, zc, gb + j);
            acc = fma(-cf[10 + j], vz, acc);
        }
        if constexpr (DI) {
            // dinv holds w D^-1 and the lower rhs r / w: lower
            // X = w D^-1 (r / w - L v); upper X = v + w D^-1 (-U w)
            double e = a.rev ? rh : 0.0;
#pragma unroll
            for (int j = 0; j < 5; ++j) e = fma(di[j], __shfl_sync(FULL, acc, gb + j), e);
            acc = e;
        }
        if (comp) {
            X = acc;
            const i64 p = L + dir * xx;
            O[p * 5 + c] = X;
            if (U) U[p * 5 + c] = fma(a.cu, X, uo);
            if (mb_out) mb_store<double>(mbox, p * 5 + c, X, tag);
        } else if (!in) {
            X = 0.0;
        }
        xprev = X;
        if (ring_out) {
            const int old = s - RING;
            if (old >= 0 && old + 1 > cachedC) {
                int cc2 = 0, okk = 1;
                if (lane == 0) {
                    unsigned long long t0 = 0;
                    for (int it = 1;; ++it) {
                        cc2 = sh.prog[w + 1];
                        if (cc2 >= old + 1) break;
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
                cachedC = __shfl_sync(FULL, cc2, 0);
                if (!okk) { ok = false; return; }
            }
            sh.ring[w][s & (RING - 1)][lane] = Tagged<double>::pack(X, (unsigned)(s + BIAS));
        }
        __syncwarp();
        if (lane == 0) sh.prog[w] = s;
    };
    for (int s0 = 0; ok && s0 < S; s0 += PD) {
#pragma unroll
        for (int k = 0; k < PD; ++k)
            if (ok) step(s0 + k, k);
    }
    __syncwarp();
    if (lane == 0) sh.prog[w] = INT_MAX;
}

template <bool DI>
__global__ void __launch_bounds__(BW * 32, 1) block_cta_kernel(BlockCtaArgs a) {
    __shared__ int s_ticket;
    __shared__ unsigned s_tag;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    BlockShared& sh = *reinterpret_cast<BlockShared*>(dyn_smem);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tag = (unsigned)ld_relaxed_gpu(&a.ctrl[2]) + 1u;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&a.ctrl[0], 1);
        for (int i = threadIdx.x; i < BW * cta::RING * 32; i += blockDim.x)
            (&sh.ring[0][0][0])[i] = cta::Tagged<double>::zero();
        if (threadIdx.x < BW) sh.prog[threadIdx.x] = -(1 << 30);
        __syncthreads();
        const int t = s_ticket;
        if (t >= a.n_units) break;
        int ab = 0;
        if (threadIdx.x == 0) ab = ld_relaxed_gpu(&a.status->abort) || t == a.stall_unit;
        ab = __syncthreads_or(ab);
        // with stored blocks each warp runs a copy of the step compiled for
        // its role, which drops the role tests from the step (162^3 x 5 SSOR
        // iteration 4.30 -> 4.24 ms); the form that applies w D^-1 keeps one
        // copy (its step measured 1 % slower with three)
        if (!ab) {
            constexpr int PD = DI ? BD_DI : BD;
            if (DI)
                block_warp<DI, PD, -1>(a, t, warp, sh, s_tag);
            else if (warp == 0)
                block_warp<DI, PD, 0>(a, t, warp, sh, s_tag);
            else if (warp == BW - 1)
                block_warp<DI, PD, 2>(a, t, warp, sh, s_tag);
            else
                block_warp<DI, PD, 1>(a, t, warp, sh, s_tag);
        }
        __syncthreads();
    }
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

unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

M2S_BOUNDS_READER(bounds_read_block)

cudaError_t block_create(BlockOp* b, const m2s_grid_desc* descs, int n_problems,
                         const std::vector<std::vector<Dims>>& dims, cudaStream_t st,
                         BlockAlloc alloc) {
    b->np = n_problems;
    b->dims.resize(n_problems);
    b->npts = 0;
    for (int i = 0; i < n_problems; ++i) {
        b->dims[i] = dims[i][0];
        b->npts += b->dims[i].n;
    }
    const size_t n = (size_t)std::max<i64>(b->npts, 1);
    cudaError_t e;
    b->jac = descs[0].op == M2S_OP_BLOCK7_JAC;
    if (b->jac) {
        if ((e = alloc((void**)&b->P, (size_t)n_problems * JP * 8)) != cudaSuccess) return e;
        if ((e = alloc((void**)&b->Dinv, n * 25 * 8)) != cudaSuccess) return e;
        if ((e = alloc((void**)&b->h, n * 15 * 8)) != cudaSuccess) return e;
        b->nu.resize(n_problems);
        for (int i = 0; i < n_problems; ++i) b->nu[i] = descs[i].jac[1];
        for (int i = 0; i < n_problems; ++i)
            if ((e = cudaMemcpyAsync(b->P + (size_t)i * JP, descs[i].jac, JP * 8,
                                     cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return e;
    } else {
        if ((e = alloc((void**)&b->D, n * 25 * 8)) != cudaSuccess) return e;
        if ((e = alloc((void**)&b->L, n * 75 * 8)) != cudaSuccess) return e;
        if ((e = alloc((void**)&b->U, n * 75 * 8)) != cudaSuccess) return e;
        if ((e = alloc((void**)&b->Dinv, n * 25 * 8)) != cudaSuccess) return e;
    }
    if ((e = alloc((void**)&b->M, n * 75 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->N, n * 75 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->s, n * 5 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->v, n * 5 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->w, n * 5 * 8)) != cudaSuccess) return e;
    for (int i = 0; i < n_problems && !b->jac; ++i) {
        const Dims& d = b->dims[i];
        if (d.n == 0) continue;
        const unsigned nb = (unsigned)nblk(d.n, 128);
        block_to_soa_kernel<<<nb, 128, 0, st>>>(d.n, b->npts, d.off, 25, descs[i].D, b->D);
        block_to_soa_kernel<<<nb, 128, 0, st>>>(d.n, b->npts, d.off, 75, descs[i].L, b->L);
        block_to_soa_kernel<<<nb, 128, 0, st>>>(d.n, b->npts, d.off, 75, descs[i].U, b->U);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // sweep units of all problems: 5 rows x BW planes, ordered by the step
    // at which they could start on an idle GPU (the unit to the right lags
    // BROWS steps, the unit above BW; producers have smaller keys), problems
    // merged by the same key
    struct Item {
        long long key;
        int z0, problem, y0;
    };
    std::vector<Item> items;
    for (int i = 0; i < n_problems; ++i) {
        const Dims& d = b->dims[i];
        for (int Z = 0; Z < (d.nz + BW - 1) / BW; ++Z)
            for (int Y = 0; Y < (d.ny + BROWS - 1) / BROWS; ++Y)
                items.push_back(Item{(long long)Y * BROWS + (long long)Z * BW, Z * BW, i, Y * BROWS});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
        if (x.key != y.key) return x.key < y.key;
        return x.problem != y.problem ? x.problem < y.problem : x.z0 < y.z0;
    });
    std::vector<int4> units(items.size());
    for (size_t k = 0; k < items.size(); ++k)
        units[k] = make_int4(items[k].y0, items[k].z0, items[k].problem, 0);
    WaveUnits& u = b->sweep;
    u = WaveUnits{};
    u.n_units = (int)units.size();
    u.np = n_problems;
    u.W = BW;
    if ((e = cudaMalloc(&u.d_units, std::max<size_t>(units.size(), 1) * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_dims, n_problems * sizeof(Dims))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_ctrl, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&u.d_mbox, n * 10 * sizeof(unsigned long long))) != cudaSuccess)
        return e;
    if ((!units.empty() && (e = cudaMemcpy(u.d_units, units.data(), units.size() * sizeof(int4),
                                           cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(u.d_dims, b->dims.data(), n_problems * sizeof(Dims),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(u.d_ctrl, 0, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(u.d_mbox, 0, n * 10 * sizeof(unsigned long long))) != cudaSuccess)
        return e;
    const int smem = (int)sizeof(BlockShared);
    auto sweep = b->jac ? block_cta_kernel<true> : block_cta_kernel<false>;
    cudaFuncSetAttribute(sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep, BW * 32,
                                                           smem)) != cudaSuccess)
        return e;
    u.grid = wave_grid(u.n_units, per_sm);
    b->omega = -1.0;
    return cudaSuccess;
}

void block_free_units(BlockOp* b) { free_wave_units(&b->sweep); }

cudaError_t block_apply(BlockOp* b, const double* u, double* y, cudaStream_t st) {
    for (int i = 0; i < b->np; ++i) {
        const Dims& d = b->dims[i];
        if (d.n == 0) continue;
        if (b->jac)
            block_jac_apply_kernel<<<nblk(d.n, JB), JB, 0, st>>>(d, b->P + (size_t)i * JP, u, y);
        else
            block_apply_kernel<false><<<nblk(d.n, 128), 128, 0, st>>>(d, b->npts, b->D, b->L, b->U,
                                                                      nullptr, nullptr, u, y);
    }
    return cudaGetLastError();
}

cudaError_t block_ssor_iter(BlockOp* b, const double* rhs, double* u, double omega,
                            DevStatus* status, long long spin_ns, cudaStream_t st) {
    cudaError_t e;
    if (b->jac) {
        // blocks of this step from the u it starts from: L, U (in M, N),
        // w D^-1, then s = r / w (b - D u parked in v until the lower sweep)
        for (int i = 0; i < b->np; ++i) {
            const Dims& d = b->dims[i];
            if (d.n == 0) continue;
            block_jac_form_kernel<<<nblk(d.n, JB), JB, 0, st>>>(d, b->P + (size_t)i * JP, omega,
                                                                rhs, u, b->M, b->N, b->Dinv, b->h,
                                                                b->npts, b->v);
        }
        for (int i = 0; i < b->np; ++i) {
            const Dims& d = b->dims[i];
            if (d.n == 0) continue;
            block_jac_resid_kernel<<<nblk(d.n, 256), 256, 0, st>>>(d, u, b->h, b->npts, b->v,
                                                                   b->nu[i], 1.0 / omega, b->s);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else if (omega != b->omega) {
        for (int i = 0; i < b->np; ++i) {
            const Dims& d = b->dims[i];
            if (d.n == 0) continue;
            block_setup_kernel<<<nblk(d.n, 64), 64, 0, st>>>(d, b->npts, b->D, b->L, b->U, omega,
                                                             b->Dinv, b->M, b->N);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        b->omega = omega;
    }
    const double cu = omega * (2.0 - omega);
    for (int i = 0; i < b->np && !b->jac; ++i) {
        const Dims& d = b->dims[i];
        if (d.n == 0) continue;
        block_apply_kernel<true><<<nblk(d.n, 128), 128, 0, st>>>(d, b->npts, b->D, b->L, b->U,
                                                                 b->Dinv, rhs, u, b->s);
    }
    const WaveUnits& un = b->sweep;
    if (un.n_units == 0) return cudaGetLastError();
    BlockCtaArgs a;
    a.spin_ns = spin_ns;
    a.units = un.d_units;
    a.dims = un.d_dims;
    a.n_units = un.n_units;
    a.ctrl = un.d_ctrl;
    a.status = status;
    a.stall_unit = -1;
    a.mbox = un.d_mbox;
    a.dinv = b->Dinv;
    auto sweep = b->jac ? block_cta_kernel<true> : block_cta_kernel<false>;
    // lower sweep: v = s - M v (increasing p), or v = D^-1 (r - w L v)
    a.rev = 0;
    a.coup = b->M;
    a.rhs = b->s;
    a.out = b->v;
    a.u = nullptr;
    a.cu = 0.0;
    sweep<<<un.grid, BW * 32, sizeof(BlockShared), st>>>(a);
    // upper sweep: w = v - N w (decreasing p), u += w(2-w) w
    a.rev = 1;
    a.coup = b->N;
    a.rhs = b->v;
    a.out = b->w;
    a.u = u;
    a.cu = cu;
    sweep<<<un.grid, BW * 32, sizeof(BlockShared), st>>>(a);
    return cudaGetLastError();
}

}  // namespace m2s
