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
    const double* coef;  // [n][5]
    double* rhs;         // [n][K]
    double* work;        // [3][n]: 1/u, u1, e
};

template <int K>
__global__ void __launch_bounds__(LB) line_penta_kernel(LineArgs a) {
    const i64 t = blockIdx.x * (i64)LB + threadIdx.x;
    i64 base, stride;
    int m;
    if (a.axis == 0) {  // lines along x: one per (y, z)
        if (t >= (i64)a.ny * a.nz) return;
        base = t * a.nx;
        stride = 1;
        m = a.nx;
    } else if (a.axis == 1) {  // along y: one per (x, z)
        if (t >= (i64)a.nx * a.nz) return;
        const i64 z = t / a.nx, x = t - z * a.nx;
        base = z * a.nx * a.ny + x;
        stride = a.nx;
        m = a.ny;
    } else {  // along z: one per (x, y)
        if (t >= (i64)a.nx * a.ny) return;
        base = t;
        stride = (i64)a.nx * a.ny;
        m = a.nz;
    }
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

template <int K>
void launch_k(const LineArgs& a, i64 lines, cudaStream_t st) {
    const unsigned grid = (unsigned)((lines + LB - 1) / LB);
    line_penta_kernel<K><<<grid, LB, 0, st>>>(a);
}

}  // namespace

i64 line_penta_work_doubles(int nx, int ny, int nz) { return 3LL * nx * ny * nz; }

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

}  // namespace m2s
