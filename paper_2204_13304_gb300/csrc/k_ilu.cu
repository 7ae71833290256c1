// ILU(0) of the HPCG 27-point matrix and its application (the incomplete LU
// preconditioner of paper Sec. 1; the ILU micro-benchmark of Sec. 7.2.1 on
// the 27-point stencil).
//
// Factors on the matrix's own pattern, 27 values per point over the 3x3x3
// box offsets o = (dz+1)*9 + (dy+1)*3 + (dx+1): o < 13 the unit-lower factor
// L, o = 13 the pivot u_pp, o > 13 the strict upper part of U, 0 where the
// neighbour is off the domain.  Row p of the IKJ elimination needs the
// finished rows of its lower neighbours, and so do the forward and backward
// substitutions: the same dependence as the lexicographic Gauss-Seidel
// sweep, so every point of a hyperplane t = x + 2y + 4z depends only on
// earlier hyperplanes.  Each launch here processes one hyperplane (one
// thread per point), and stream order between the launches carries every
// dependence: no kernel waits on another, nothing can hang.  The
// application replays its 2 (T + 1) launches from a CUDA graph.
#include "m2s_internal.cuh"

namespace m2s {

namespace {

constexpr int IB = 128;  // threads per CTA

__host__ __device__ constexpr int odx(int o) { return o % 3 - 1; }
__host__ __device__ constexpr int ody(int o) { return (o / 3) % 3 - 1; }
__host__ __device__ constexpr int odz(int o) { return o / 9 - 1; }
__host__ __device__ constexpr int box_index(int dx, int dy, int dz) {
    return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
}
__host__ __device__ constexpr bool in_box(int dx, int dy, int dz) {
    return dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
}

// The point of hyperplane t handled by this thread: y from the thread index
// within the window of y whose x = t - 2y - 4z lies in [0, nx), z from
// blockIdx.y.
__device__ __forceinline__ bool hyperplane_point(const Dims& d, int t, int* x, int* y, int* z) {
    *z = blockIdx.y;
    const int rem = t - 4 * *z;  // x + 2y
    if (rem < 0) return false;
    // smallest y with x = rem - 2y <= nx - 1
    int ylo = rem - (d.nx - 1) > 0 ? (rem - (d.nx - 1) + 1) / 2 : 0;
    *y = ylo + (int)(blockIdx.x * IB + threadIdx.x);
    *x = rem - 2 * *y;
    return *y < d.ny && *x >= 0 && *x < d.nx;
}

// in-domain flags of the 27 neighbours, from the 6 boundary tests
struct Inside {
    bool xm, xp, ym, yp, zm, zp;
    __device__ __forceinline__ bool operator()(int dx, int dy, int dz) const {
        return (dx < 0 ? xm : dx > 0 ? xp : true) && (dy < 0 ? ym : dy > 0 ? yp : true) &&
               (dz < 0 ? zm : dz > 0 ? zp : true);
    }
};

__device__ __forceinline__ Inside inside_of(const Dims& d, int x, int y, int z) {
    return Inside{x > 0, x < d.nx - 1, y > 0, y < d.ny - 1, z > 0, z < d.nz - 1};
}

__device__ __forceinline__ i64 nbr(const Dims& d, i64 p, int dx, int dy, int dz) {
    return p + ((i64)dz * d.ny + dy) * d.nx + dx;
}

__global__ void __launch_bounds__(IB) ilu_factor_kernel(Dims d, int t, double* __restrict__ F) {
    int x, y, z;
    if (!hyperplane_point(d, t, &x, &y, &z)) return;
    const Inside in = inside_of(d, x, y, z);
    const i64 p = ((i64)z * d.ny + y) * d.nx + x;  // problem-local
    double* Fb = F + 27 * d.off;
    double f[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) f[o] = in(odx(o), ody(o), odz(o)) ? (o == 13 ? 26.0 : -1.0) : 0.0;
#pragma unroll
    for (int ok = 0; ok < 13; ++ok) {
        if (!in(odx(ok), ody(ok), odz(ok))) continue;
        const double* Fk = Fb + 27 * nbr(d, p, odx(ok), ody(ok), odz(ok));
        const double l = f[ok] / Fk[13];
        f[ok] = l;
#pragma unroll
        for (int oj = ok + 1; oj < 27; ++oj) {
            const int rx = odx(oj) - odx(ok), ry = ody(oj) - ody(ok), rz = odz(oj) - odz(ok);
            if (!in_box(rx, ry, rz)) continue;  // folds at compile time
            if (!in(odx(oj), ody(oj), odz(oj))) continue;
            f[oj] = fma(-l, Fk[box_index(rx, ry, rz)], f[oj]);
        }
    }
    double* Fp = Fb + 27 * p;
#pragma unroll
    for (int o = 0; o < 27; ++o) Fp[o] = f[o];
}

// forward: y_p = r_p - sum_{o < 13} F[p][o] y_q, y kept in z
__global__ void __launch_bounds__(IB) ilu_lower_kernel(Dims d, int t, const double* __restrict__ F,
                                                       const double* r, double* z) {
    int x, y, zz;
    if (!hyperplane_point(d, t, &x, &y, &zz)) return;
    const Inside in = inside_of(d, x, y, zz);
    const i64 p = ((i64)zz * d.ny + y) * d.nx + x;
    const double* Fp = F + 27 * (d.off + p);
    const double* zb = z + d.off;
    double s = r[d.off + p];
#pragma unroll
    for (int o = 0; o < 13; ++o)
        if (in(odx(o), ody(o), odz(o))) s = fma(-__ldg(Fp + o), zb[nbr(d, p, odx(o), ody(o), odz(o))], s);
    z[d.off + p] = s;
}

// backward: z_p = (y_p - sum_{o > 13} F[p][o] z_q) / F[p][13]
__global__ void __launch_bounds__(IB) ilu_upper_kernel(Dims d, int t, const double* __restrict__ F,
                                                       double* z) {
    int x, y, zz;
    if (!hyperplane_point(d, t, &x, &y, &zz)) return;
    const Inside in = inside_of(d, x, y, zz);
    const i64 p = ((i64)zz * d.ny + y) * d.nx + x;
    const double* Fp = F + 27 * (d.off + p);
    const double* zb = z + d.off;
    double s = zb[p];
#pragma unroll
    for (int o = 14; o < 27; ++o)
        if (in(odx(o), ody(o), odz(o))) s = fma(-__ldg(Fp + o), zb[nbr(d, p, odx(o), ody(o), odz(o))], s);
    z[d.off + p] = s / __ldg(Fp + 13);
}

dim3 hyperplane_grid(const Dims& d) {
    // at most ceil(nx / 2) + 1 values of y per z on one hyperplane
    const int win = d.nx / 2 + 2;
    return dim3((unsigned)((win + IB - 1) / IB), (unsigned)d.nz);
}

}  // namespace

int ilu_hyperplanes(const Dims& d) { return (d.nx - 1) + 2 * (d.ny - 1) + 4 * (d.nz - 1) + 1; }

cudaError_t launch_ilu_factor(const Dims& d, double* F, cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    const dim3 g = hyperplane_grid(d);
    const int T = ilu_hyperplanes(d);
    for (int t = 0; t < T; ++t) {
        ilu_factor_kernel<<<g, IB, 0, st>>>(d, t, F);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_ilu_apply(const Dims& d, const double* F, const double* r, double* z,
                             cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    const dim3 g = hyperplane_grid(d);
    const int T = ilu_hyperplanes(d);
    for (int t = 0; t < T; ++t) {
        ilu_lower_kernel<<<g, IB, 0, st>>>(d, t, F, r, z);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int t = T - 1; t >= 0; --t) {
        ilu_upper_kernel<<<g, IB, 0, st>>>(d, t, F, z);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace m2s
