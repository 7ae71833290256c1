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
// earlier hyperplanes.  Each factorisation launch here processes one
// hyperplane (one thread per point), and stream order between the launches
// carries every dependence: no kernel waits on another.  The application
// (k_ilu_wave.cu) runs each triangle as one persistent wavefront launch.
#include <algorithm>

#include "m2s_bounds.cuh"
#include "m2s_internal.cuh"

namespace m2s {

namespace {

constexpr int IB = 256;  // largest CTA of a hyperplane launch

__host__ __device__ constexpr int odx(int o) { return o % 3 - 1; }
__host__ __device__ constexpr int ody(int o) { return (o / 3) % 3 - 1; }
__host__ __device__ constexpr int odz(int o) { return o / 9 - 1; }
__host__ __device__ constexpr int box_index(int dx, int dy, int dz) {
    return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
}
__host__ __device__ constexpr bool in_box(int dx, int dy, int dz) {
    return dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1;
}

// The point of hyperplane t handled by this thread: z = z0 + blockIdx.y
// (the launch covers the z that meet the hyperplane), y from the thread
// index within the window of y whose x = t - 2y - 4z lies in [0, nx).
__device__ __forceinline__ bool hyperplane_point(const Dims& d, int t, int z0, int* x, int* y,
                                                 int* z) {
    *z = z0 + (int)blockIdx.y;
    const int rem = t - 4 * *z;  // x + 2y
    if (rem < 0) return false;
    // smallest y with x = rem - 2y <= nx - 1
    int ylo = rem - (d.nx - 1) > 0 ? (rem - (d.nx - 1) + 1) / 2 : 0;
    *y = ylo + (int)(blockIdx.x * blockDim.x + threadIdx.x);
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

__global__ void __launch_bounds__(IB) ilu_factor_kernel(Dims d, int t, int z0,
                                                        double* __restrict__ F,
                                                        double* __restrict__ Finv) {
    int x, y, z;
    if (!hyperplane_point(d, t, z0, &x, &y, &z)) return;
    const Inside in = inside_of(d, x, y, z);
    const i64 p = ((i64)z * d.ny + y) * d.nx + x;  // problem-local
    if (!M2S_IN(p, d.n)) return;
    double* Fb = F + 27 * d.off;
    double* Ib = Finv + d.off;
    double f[27];
#pragma unroll
    for (int o = 0; o < 27; ++o) f[o] = in(odx(o), ody(o), odz(o)) ? (o == 13 ? 26.0 : -1.0) : 0.0;
#pragma unroll
    for (int ok = 0; ok < 13; ++ok) {
        if (!in(odx(ok), ody(ok), odz(ok))) continue;
        const i64 k = nbr(d, p, odx(ok), ody(ok), odz(ok));
        if (!M2S_IN(k, d.n)) continue;
        const double* Fk = Fb + 27 * k;
        const double l = f[ok] * Ib[k];  // the pivot's rounded reciprocal
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
    Ib[p] = 1.0 / f[13];
}

// Launch shape of hyperplane t: the z that meet it (0 <= t - 4z <= (nx-1) +
// 2(ny-1)), one CTA row each; the window of at most nx/2 + 2 values of y
// per z in CTAs of up to IB threads (a warp multiple).
struct HpLaunch {
    dim3 grid, block;
    int z0;
};
HpLaunch hyperplane_launch(const Dims& d, int t) {
    const int reach = (d.nx - 1) + 2 * (d.ny - 1);
    const int zlo = std::max(0, (t - reach + 3) / 4);
    const int zhi = std::min(d.nz - 1, t / 4);
    const int win = d.nx / 2 + 2;
    const int bs = std::min(IB, (win + 31) / 32 * 32);
    HpLaunch h;
    h.z0 = zlo;
    h.block = dim3((unsigned)bs);
    h.grid = dim3((unsigned)((win + bs - 1) / bs), (unsigned)std::max(0, zhi - zlo + 1));
    return h;
}

}  // namespace

int ilu_hyperplanes(const Dims& d) { return (d.nx - 1) + 2 * (d.ny - 1) + 4 * (d.nz - 1) + 1; }

cudaError_t launch_ilu_factor(const Dims& d, double* F, double* Finv, cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    const int T = ilu_hyperplanes(d);
    for (int t = 0; t < T; ++t) {
        const HpLaunch h = hyperplane_launch(d, t);
        if (h.grid.y == 0) continue;
        ilu_factor_kernel<<<h.grid, h.block, 0, st>>>(d, t, h.z0, F, Finv);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

M2S_BOUNDS_READER(bounds_read_ilu)

}  // namespace m2s
