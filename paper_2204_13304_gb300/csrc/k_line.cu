// Direct solves of pentadiagonal systems along the grid lines of one axis:
// the "direct solving of multi-diagonal matrices" of NPB-SP (paper Sec. 1;
// Sec. 7.2.2: along each axis every line is swept forward and backward, and
// fusing the two sweeps per line shrinks the intermediates to one line).
//
// Point p at position i of its line holds the equation
//   a v_{i-2} + b v_{i-1} + c v_i + d v_{i+1} + e v_{i+2} = r_i
// (coef[p] = (a, b, c, d, e), terms outside the line dropped) and K
// right-hand sides rhs[p][0..K-1], overwritten with the solutions.
//
// One thread owns one line and runs both sweeps of the LU factorisation
// without pivoting.  Forward, row i is reduced by rows i-2 and i-1:
//   l2 = a / u_{i-2},  l1 = (b - l2 u1_{i-2}) / u_{i-1},
//   u_i = c - l2 e_{i-2} - l1 u1_{i-1},  u1_i = d - l1 e_{i-1},
//   y_i = r_i - l2 y_{i-2} - l1 y_{i-1},
// with the two previous rows' (1/u, u1, e, y) in registers; backward,
//   v_i = (y_i - u1_i v_{i+1} - e_i v_{i+2}) / u_i.
// The forward sweep leaves y in rhs and (1/u, u1, e) in a work array read
// back by the backward sweep of the same thread.  Lines of the y and z axes
// map neighbouring threads to neighbouring x, so every access of a warp is
// one contiguous run; x lines walk their own contiguous records.
//
// On GB300 this is bound by FP64 issue (7 + 5K FP64 operations per point
// against ~215 bytes of DRAM traffic; 162^3 with K = 5: the FP64 pipe is
// ~65 % busy on y and z lines), not by HBM.  The coefficients and
// right-hand sides of the next LD points are loaded ahead of the one being
// eliminated, which hides the load latency of the few warps per SM.
#include "m2s_bounds.cuh"
#include "m2s_internal.cuh"

namespace m2s {

namespace {

// threads per CTA: one warp, so that the ~n^2 lines spread evenly over the
// SMs (the kernel is FP64-bound per SM; 128-thread CTAs left 2 on some SMs
// and 1 on others)
constexpr int LB = 32;
constexpr int LD = 4;    // points of a line in flight ahead of the one computed

struct LineArgs {
    int nx, ny, nz, axis;
    i64 n;
    const double* coef;  // pentadiagonal: [n][5]; block-tridiagonal: [n][3][25]
    double* rhs;         // [n][K]
    double* work;        // pentadiagonal: [3][n] (1/u, u1, e); block: [n][25] (C^)
};

// Line t of the launch: its first point, the point stride along it and its
// length.  Lines of the y and z axes are numbered with x fastest, so that
// neighbouring threads hold neighbouring x.
__device__ __forceinline__ bool line_of(const LineArgs& a, i64 t, i64* base, i64* stride, int* m) {
    if (a.axis == 0) {  // lines along x: one per (y, z)
        if (t >= (i64)a.ny * a.nz) return false;
        *base = t * a.nx;
        *stride = 1;
        *m = a.nx;
    } else if (a.axis == 1) {  // along y: one per (x, z)
        if (t >= (i64)a.nx * a.nz) return false;
        const i64 z = t / a.nx, x = t - z * a.nx;
        *base = z * a.nx * a.ny + x;
        *stride = a.nx;
        *m = a.ny;
    } else {  // along z: one per (x, y)
        if (t >= (i64)a.nx * a.ny) return false;
        *base = t;
        *stride = (i64)a.nx * a.ny;
        *m = a.nz;
    }
    return true;
}

template <int K>
__global__ void __launch_bounds__(LB) line_penta_kernel(LineArgs a) {
    i64 base, stride;
    int m;
    if (!line_of(a, blockIdx.x * (i64)LB + threadIdx.x, &base, &stride, &m)) return;
    // the line's points are affine in i: its two ends bound every access
    if (!(M2S_IN(base, a.n) && M2S_IN(base + (i64)(m - 1) * stride, a.n))) return;
    const double* __restrict__ coef = a.coef;
    double* __restrict__ rhs = a.rhs;
    double* __restrict__ w_inv = a.work;
    double* __restrict__ w_u1 = a.work + a.n;
    double* __restrict__ w_e = a.work + 2 * a.n;

    // forward: rows i-1 (suffix 1) and i-2 (suffix 2); the coefficients and
    // right-hand sides of the next LD points are in flight in a register
    // ring (the loop is unrolled by LD so the ring is statically indexed)
    double inv1 = 0.0, inv2 = 0.0, u11 = 0.0, u12 = 0.0, e1 = 0.0, e2 = 0.0;
    double y1[K], y2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) y1[k] = y2[k] = 0.0;
    double fc[LD][5], fr[LD][K];
    auto fetch_f = [&](int slot, int i) {
        if (i < m) {
            const i64 q = base + (i64)i * stride;
            const double* cp = coef + 5 * q;
            fc[slot][0] = i >= 2 ? __ldg(cp + 0) : 0.0;
            fc[slot][1] = i >= 1 ? __ldg(cp + 1) : 0.0;
            fc[slot][2] = __ldg(cp + 2);
            fc[slot][3] = i + 1 < m ? __ldg(cp + 3) : 0.0;
            fc[slot][4] = i + 2 < m ? __ldg(cp + 4) : 0.0;
            const double* rp = rhs + (i64)K * q;
#pragma unroll
            for (int k = 0; k < K; ++k) fr[slot][k] = rp[k];
        }
    };
#pragma unroll
    for (int s = 0; s < LD; ++s) fetch_f(s, s);
    for (int i0 = 0; i0 < m; i0 += LD) {
#pragma unroll
        for (int s = 0; s < LD; ++s) {
            const int i = i0 + s;
            if (i < m) {
                const double ca = fc[s][0], cb = fc[s][1], cc = fc[s][2], cd = fc[s][3],
                             ce = fc[s][4];
                double r[K];
#pragma unroll
                for (int k = 0; k < K; ++k) r[k] = fr[s][k];
                fetch_f(s, i + LD);
                const double l2 = ca * inv2;
                const double l1 = fma(-l2, u12, cb) * inv1;
                const double u = fma(-l1, u11, fma(-l2, e2, cc));
                const double u1 = fma(-l1, e1, cd);
                const double inv = __drcp_rn(u);
                const i64 p = base + (i64)i * stride;
                double* rp = rhs + (i64)K * p;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const double y = fma(-l1, y1[k], fma(-l2, y2[k], r[k]));
                    rp[k] = y;
                    y2[k] = y1[k];
                    y1[k] = y;
                }
                w_inv[p] = inv;
                w_u1[p] = u1;
                w_e[p] = ce;
                inv2 = inv1;
                inv1 = inv;
                u12 = u11;
                u11 = u1;
                e2 = e1;
                e1 = ce;
            }
        }
    }
    // backward: v_{i+1} (suffix 1) and v_{i+2} (suffix 2), with the next LD
    // points' (1/u, u1, e, y) in flight (written above by this thread)
    double v1[K], v2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v1[k] = v2[k] = 0.0;
    double bw[LD][3], by[LD][K];
    auto fetch_b = [&](int slot, int i) {
        if (i >= 0) {
            const i64 q = base + (i64)i * stride;
            bw[slot][0] = w_inv[q];
            bw[slot][1] = w_u1[q];
            bw[slot][2] = w_e[q];
            const double* rp = rhs + (i64)K * q;
#pragma unroll
            for (int k = 0; k < K; ++k) by[slot][k] = rp[k];
        }
    };
#pragma unroll
    for (int s = 0; s < LD; ++s) fetch_b(s, m - 1 - s);
    for (int i0 = m - 1; i0 >= 0; i0 -= LD) {
#pragma unroll
        for (int s = 0; s < LD; ++s) {
            const int i = i0 - s;
            if (i >= 0) {
                const double inv = bw[s][0], u1 = bw[s][1], e = bw[s][2];
                double y[K];
#pragma unroll
                for (int k = 0; k < K; ++k) y[k] = by[s][k];
                fetch_b(s, i - LD);
                double* rp = rhs + (i64)K * (base + (i64)i * stride);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const double v = fma(-e, v2[k], fma(-u1, v1[k], y[k])) * inv;
                    rp[k] = v;
                    v2[k] = v1[k];
                    v1[k] = v;
                }
            }
        }
    }
}

// Block-tridiagonal lines (NPB-BT shape): A v_{i-1} + B v_i + C v_{i+1} = r_i
// with 5x5 blocks.  One thread per line runs block elimination without
// pivoting, forward
//   B'_i = B_i - A_i C^_{i-1},  r'_i = r_i - A_i r^_{i-1},
//   [C^_i | r^_i] = B'_i^{-1} [C_i | r'_i]   (Gaussian elimination of B'_i),
// with C^_{i-1} and r^_{i-1} in registers, C^_i stored to the work array and
// r^_i to rhs; backward v_i = r^_i - C^_i v_{i+1}.  About 375 FP64
// operations per point against ~1.2 KB: FP64-bound on GB300.
__global__ void __launch_bounds__(LB) line_btri_kernel(LineArgs a) {
    i64 base, stride;
    int m;
    if (!line_of(a, blockIdx.x * (i64)LB + threadIdx.x, &base, &stride, &m)) return;
    if (!(M2S_IN(base, a.n) && M2S_IN(base + (i64)(m - 1) * stride, a.n))) return;
    const double* __restrict__ blk = a.coef;
    double* __restrict__ rhs = a.rhs;
    double* __restrict__ ch = a.work;
    double cp[25], rp[5];  // C^ and r^ of the previous point
#pragma unroll
    for (int j = 0; j < 25; ++j) cp[j] = 0.0;
#pragma unroll
    for (int j = 0; j < 5; ++j) rp[j] = 0.0;
    i64 p = base;
    for (int i = 0; i < m; ++i, p += stride) {
        const double* bp = blk + 75 * p;
        double B[25], r[5];
#pragma unroll
        for (int j = 0; j < 25; ++j) B[j] = __ldg(bp + 25 + j);
#pragma unroll
        for (int j = 0; j < 5; ++j) r[j] = rhs[5 * p + j];
        if (i > 0) {
            double A[25];
#pragma unroll
            for (int j = 0; j < 25; ++j) A[j] = __ldg(bp + j);
#pragma unroll
            for (int j = 0; j < 5; ++j) {
#pragma unroll
                for (int l = 0; l < 5; ++l) {
                    const double ajl = A[5 * j + l];
#pragma unroll
                    for (int c = 0; c < 5; ++c) B[5 * j + c] = fma(-ajl, cp[5 * l + c], B[5 * j + c]);
                    r[j] = fma(-ajl, rp[l], r[j]);
                }
            }
        }
        // X = [C | r'], eliminated with B' below
        double X[30];
        const bool last = i + 1 == m;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
#pragma unroll
            for (int c = 0; c < 5; ++c) X[6 * j + c] = last ? 0.0 : __ldg(bp + 50 + 5 * j + c);
            X[6 * j + 5] = r[j];
        }
        double piv[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            piv[k] = __drcp_rn(B[5 * k + k]);
#pragma unroll
            for (int j = k + 1; j < 5; ++j) {
                const double f = B[5 * j + k] * piv[k];
#pragma unroll
                for (int c = k + 1; c < 5; ++c) B[5 * j + c] = fma(-f, B[5 * k + c], B[5 * j + c]);
#pragma unroll
                for (int c = 0; c < 6; ++c) X[6 * j + c] = fma(-f, X[6 * k + c], X[6 * j + c]);
            }
        }
#pragma unroll
        for (int k = 4; k >= 0; --k) {
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                double sum = X[6 * k + c];
#pragma unroll
                for (int l = k + 1; l < 5; ++l) sum = fma(-B[5 * k + l], X[6 * l + c], sum);
                X[6 * k + c] = sum * piv[k];
            }
        }
        double* cw = ch + 25 * p;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                cp[5 * j + c] = X[6 * j + c];
                cw[5 * j + c] = X[6 * j + c];
            }
            rp[j] = X[6 * j + 5];
            rhs[5 * p + j] = rp[j];
        }
    }
    // backward
    double v[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) v[j] = 0.0;
    p = base + (i64)(m - 1) * stride;
    for (int i = m - 1; i >= 0; --i, p -= stride) {
        const double* cw = ch + 25 * p;
        double nv[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            double sum = rhs[5 * p + j];
#pragma unroll
            for (int l = 0; l < 5; ++l) sum = fma(-cw[5 * j + l], v[l], sum);
            nv[j] = sum;
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            v[j] = nv[j];
            rhs[5 * p + j] = nv[j];
        }
    }
}

template <int K>
void launch_k(const LineArgs& a, i64 lines, cudaStream_t st) {
    const unsigned grid = (unsigned)((lines + LB - 1) / LB);
    line_penta_kernel<K><<<grid, LB, 0, st>>>(a);
}

}  // namespace

i64 line_penta_work_doubles(int nx, int ny, int nz) { return 3LL * nx * ny * nz; }
i64 line_btri_work_doubles(int nx, int ny, int nz) { return 25LL * nx * ny * nz; }

cudaError_t launch_line_btri(int nx, int ny, int nz, int axis, const double* blk, double* rhs,
                             double* work, cudaStream_t st) {
    LineArgs a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.axis = axis;
    a.n = (i64)nx * ny * nz;
    a.coef = blk;
    a.rhs = rhs;
    a.work = work;
    const i64 lines = axis == 0 ? (i64)ny * nz : axis == 1 ? (i64)nx * nz : (i64)nx * ny;
    if (lines == 0) return cudaSuccess;
    line_btri_kernel<<<(unsigned)((lines + LB - 1) / LB), LB, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_line_penta(int nx, int ny, int nz, int axis, const double* coef, double* rhs,
                              int k, double* work, cudaStream_t st) {
    LineArgs a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.axis = axis;
    a.n = (i64)nx * ny * nz;
    a.coef = coef;
    a.rhs = rhs;
    a.work = work;
    const i64 lines = axis == 0 ? (i64)ny * nz : axis == 1 ? (i64)nx * nz : (i64)nx * ny;
    if (lines == 0) return cudaSuccess;
    switch (k) {
        case 1: launch_k<1>(a, lines, st); break;
        case 2: launch_k<2>(a, lines, st); break;
        case 3: launch_k<3>(a, lines, st); break;
        case 4: launch_k<4>(a, lines, st); break;
        case 5: launch_k<5>(a, lines, st); break;
        case 6: launch_k<6>(a, lines, st); break;
        case 7: launch_k<7>(a, lines, st); break;
        case 8: launch_k<8>(a, lines, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

M2S_BOUNDS_READER(bounds_read_line)

}  // namespace m2s
