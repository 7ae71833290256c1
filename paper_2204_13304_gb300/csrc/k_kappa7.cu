// Variable-coefficient 7-point diffusion operator (face-averaged kappa) --
// set-up, SpMV, old-neighbour sums, residual restriction, kappa coarsening
// and the kappa gradient of the adjoint.
//
// Operator: (A u)_p = sum over the 6 faces of cell p of k_f (u_p - u_q);
// an interior face between p and q has k_f = (k_p + k_q)/2 (the averaging
// matrix A = [1/2 1/2] of paper Sec. 4.1), a boundary face has k_f = k_p and
// a zero ghost value.  In matrix form a_pp = sum_f k_f and a_pq = -k_f.
//
// The face coefficients, the diagonal and its inverse are formed once per
// level at set-up (kf[d][p] couples p and p - e_d, kr[d][p] couples p and
// p + e_d, 0 on the boundary), so the
// SpMV costs 1 multiply + 6 FMAs per point: on GB300 FP64 issue, not HBM, is
// the scarce resource.
#include "m2s_internal.cuh"
#include "m2s_pcg.cuh"

namespace m2s {

namespace {

constexpr int B = 256;

__device__ __forceinline__ void coords(i64 i, int nx, int ny, int* x, int* y, int* z) {
    *x = (int)(i % nx);
    const i64 r = i / nx;
    *y = (int)(r % ny);
    *z = (int)(r / ny);
}

// Coarse kappa: mean over the fine cells {2i, 2i+1}^3 inside the grid, in
// the order dz, dy, dx.
__global__ void kappa_coarsen_kernel(Dims f, Dims c, const double* __restrict__ kf,
                                     double* __restrict__ kc) {
    const i64 i = blockIdx.x * (i64)B + threadIdx.x;
    if (i >= c.n) return;
    int cx, cy, cz;
    coords(i, c.nx, c.ny, &cx, &cy, &cz);
    double s = 0.0;
    int cnt = 0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const int x = 2 * cx + dx, y = 2 * cy + dy, z = 2 * cz + dz;
                if (x >= f.nx || y >= f.ny || z >= f.nz) continue;
                s += kf[f.off + ((i64)z * f.ny + y) * f.nx + x];
                ++cnt;
            }
    kc[c.off + i] = s / (double)cnt;
}

// Face coefficients and diagonal in precision T from the FP64 kappa of the
// level (rounded to T first, so the FP32 hierarchy is the FP32 operator of
// the FP32-rounded kappa).  Diagonal faces summed in the order
// -z, -y, -x, +x, +y, +z.
template <typename T>
__global__ void kappa_setup_kernel(Dims d, const double* __restrict__ kappa, KappaLevel<T> k) {
    const i64 i = blockIdx.x * (i64)B + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const double* K = kappa + d.off;
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    const T kp = (T)K[i];
    const T half = T(0.5);
    const T fzm = z > 0 ? half * (kp + (T)K[i - sz]) : T(0);
    const T fym = y > 0 ? half * (kp + (T)K[i - sy]) : T(0);
    const T fxm = x > 0 ? half * (kp + (T)K[i - 1]) : T(0);
    const T fxp = x < d.nx - 1 ? half * (kp + (T)K[i + 1]) : T(0);
    const T fyp = y < d.ny - 1 ? half * (kp + (T)K[i + sy]) : T(0);
    const T fzp = z < d.nz - 1 ? half * (kp + (T)K[i + sz]) : T(0);
    T dg = T(0);
    dg += z > 0 ? fzm : kp;
    dg += y > 0 ? fym : kp;
    dg += x > 0 ? fxm : kp;
    dg += x < d.nx - 1 ? fxp : kp;
    dg += y < d.ny - 1 ? fyp : kp;
    dg += z < d.nz - 1 ? fzp : kp;
    const i64 p = d.off + i;
    k.kf[0][p] = fxm;
    k.kf[1][p] = fym;
    k.kf[2][p] = fzm;
    k.kr[0][p] = fxp;
    k.kr[1][p] = fyp;
    k.kr[2][p] = fzp;
    k.diag[p] = dg;
    const T id = T(1) / dg;
    k.invdiag[p] = id;
    T* f = k.pack[0] + 4 * p;
    T* r = k.pack[1] + 4 * p;
    f[0] = fxm, f[1] = fym, f[2] = fzm, f[3] = id;
    r[0] = fxp, r[1] = fyp, r[2] = fzp, r[3] = id;
}

// (A x)_p at point i (local index) of level d.
template <typename T>
__device__ __forceinline__ T apply7_at(Dims d, const KappaLevel<T>& k, const T* __restrict__ xv,
                                       i64 i, int x, int y, int z) {
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    const i64 p = d.off + i;
    T s = T(0);
    if (z > 0) s = fma(k.kf[2][p], xv[p - sz], s);
    if (y > 0) s = fma(k.kf[1][p], xv[p - sy], s);
    if (x > 0) s = fma(k.kf[0][p], xv[p - 1], s);
    if (x < d.nx - 1) s = fma(k.kf[0][p + 1], xv[p + 1], s);
    if (y < d.ny - 1) s = fma(k.kf[1][p + sy], xv[p + sy], s);
    if (z < d.nz - 1) s = fma(k.kf[2][p + sz], xv[p + sz], s);
    return fma(k.diag[p], xv[p], -s);
}

template <typename T>
__global__ void spmv7_kernel(Dims d, KappaLevel<T> k, const T* __restrict__ xv,
                             T* __restrict__ yv) {
    const i64 i = blockIdx.x * (i64)B + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    yv[d.off + i] = apply7_at(d, k, xv, i, x, y, z);
}

// value of (x + P xc) at fine point p with coordinates (x, y, z)
template <typename T>
__device__ __forceinline__ T prolonged(const T* __restrict__ xv, const T* __restrict__ xc, Dims dc,
                                       i64 p, int x, int y, int z) {
    T v = xv[p];
    if (xc && ((x | y | z) & 1) == 0)
        v += xc[dc.off + ((i64)(z >> 1) * dc.ny + (y >> 1)) * dc.nx + (x >> 1)];
    return v;
}

template <typename T>
__global__ void qinit7_kernel(Dims d, Dims dc, KappaLevel<T> k, int up, const T* __restrict__ xv,
                              const T* __restrict__ xc, const T* __restrict__ b,
                              T* __restrict__ Q) {
    const i64 i = blockIdx.x * (i64)B + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    const i64 p = d.off + i;
    T s = b[p];
    if (up) {
        if (x < d.nx - 1) s = fma(k.kf[0][p + 1], prolonged(xv, xc, dc, p + 1, x + 1, y, z), s);
        if (y < d.ny - 1) s = fma(k.kf[1][p + sy], prolonged(xv, xc, dc, p + sy, x, y + 1, z), s);
        if (z < d.nz - 1) s = fma(k.kf[2][p + sz], prolonged(xv, xc, dc, p + sz, x, y, z + 1), s);
    } else {
        if (x > 0) s = fma(k.kf[0][p], prolonged(xv, xc, dc, p - 1, x - 1, y, z), s);
        if (y > 0) s = fma(k.kf[1][p], prolonged(xv, xc, dc, p - sy, x, y - 1, z), s);
        if (z > 0) s = fma(k.kf[2][p], prolonged(xv, xc, dc, p - sz, x, y, z - 1), s);
    }
    Q[p] = s;
}

template <typename T>
__global__ void restrict7_kernel(Dims f, Dims c, KappaLevel<T> k, const T* __restrict__ r,
                                 const T* __restrict__ zv, T* __restrict__ rc) {
    const i64 i = blockIdx.x * (i64)B + threadIdx.x;
    if (i >= c.n) return;
    int cx, cy, cz;
    coords(i, c.nx, c.ny, &cx, &cy, &cz);
    const int x = 2 * cx, y = 2 * cy, z = 2 * cz;
    const i64 fi = ((i64)z * f.ny + y) * f.nx + x;
    rc[c.off + i] = r[f.off + fi] - apply7_at(f, k, zv, fi, x, y, z);
}

// g_c = -[ sum_{interior faces} (1/2)(lam_c - lam_q)(u_c - u_q)
//          + (boundary faces of c) lam_c u_c ], faces -z, -y, -x, +x, +y, +z.
__global__ void kappa_grad_kernel(Dims d, const double* __restrict__ u,
                                  const double* __restrict__ lam, double* __restrict__ g) {
    const i64 i = blockIdx.x * (i64)B + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    const i64 p = d.off + i;
    const double uc = u[p], lc = lam[p];
    const double bnd = lc * uc;
    double s = 0.0;
    s += z > 0 ? 0.5 * (lc - lam[p - sz]) * (uc - u[p - sz]) : bnd;
    s += y > 0 ? 0.5 * (lc - lam[p - sy]) * (uc - u[p - sy]) : bnd;
    s += x > 0 ? 0.5 * (lc - lam[p - 1]) * (uc - u[p - 1]) : bnd;
    s += x < d.nx - 1 ? 0.5 * (lc - lam[p + 1]) * (uc - u[p + 1]) : bnd;
    s += y < d.ny - 1 ? 0.5 * (lc - lam[p + sy]) * (uc - u[p + sy]) : bnd;
    s += z < d.nz - 1 ? 0.5 * (lc - lam[p + sz]) * (uc - u[p + sz]) : bnd;
    g[p] = -s;
}

// Batched forms: one launch for all problems of a level, one CTA per chunk
// of one problem (see Batch).
template <typename T>
__global__ void __launch_bounds__(B) spmv7_b_kernel(Batch b, KappaLevel<T> k,
                                                    const T* __restrict__ xv, T* __restrict__ yv) {
    i64 lo, hi;
    const Dims d = b.dims[batch_locate(b, blockIdx.x, &lo, &hi)];
    for (i64 p = lo + threadIdx.x; p < hi; p += B) {
        const i64 i = p - d.off;
        int x, y, z;
        coords(i, d.nx, d.ny, &x, &y, &z);
        yv[p] = apply7_at(d, k, xv, i, x, y, z);
    }
}

template <typename T>
__global__ void __launch_bounds__(B) qinit7_b_kernel(Batch b, Batch c, int has_c, KappaLevel<T> k,
                                                     int up, const T* __restrict__ xv,
                                                     const T* __restrict__ xc,
                                                     const T* __restrict__ bv, T* __restrict__ Q) {
    i64 lo, hi;
    const int pb = batch_locate(b, blockIdx.x, &lo, &hi);
    const Dims d = b.dims[pb];
    const Dims dc = has_c ? c.dims[pb] : d;
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    for (i64 p = lo + threadIdx.x; p < hi; p += B) {
        int x, y, z;
        coords(p - d.off, d.nx, d.ny, &x, &y, &z);
        T s = bv[p];
        if (up) {
            if (x < d.nx - 1) s = fma(k.kf[0][p + 1], prolonged(xv, xc, dc, p + 1, x + 1, y, z), s);
            if (y < d.ny - 1) s = fma(k.kf[1][p + sy], prolonged(xv, xc, dc, p + sy, x, y + 1, z), s);
            if (z < d.nz - 1) s = fma(k.kf[2][p + sz], prolonged(xv, xc, dc, p + sz, x, y, z + 1), s);
        } else {
            if (x > 0) s = fma(k.kf[0][p], prolonged(xv, xc, dc, p - 1, x - 1, y, z), s);
            if (y > 0) s = fma(k.kf[1][p], prolonged(xv, xc, dc, p - sy, x, y - 1, z), s);
            if (z > 0) s = fma(k.kf[2][p], prolonged(xv, xc, dc, p - sz, x, y, z - 1), s);
        }
        Q[p] = s;
    }
}

// chunks of the coarse level's batch
template <typename T>
__global__ void __launch_bounds__(B) restrict7_b_kernel(Batch f, Batch c, KappaLevel<T> k,
                                                        const T* __restrict__ r,
                                                        const T* __restrict__ zv,
                                                        T* __restrict__ rc) {
    i64 lo, hi;
    const int pb = batch_locate(c, blockIdx.x, &lo, &hi);
    const Dims dc = c.dims[pb], df = f.dims[pb];
    for (i64 p = lo + threadIdx.x; p < hi; p += B) {
        int cx, cy, cz;
        coords(p - dc.off, dc.nx, dc.ny, &cx, &cy, &cz);
        const int x = 2 * cx, y = 2 * cy, z = 2 * cz;
        const i64 fi = ((i64)z * df.ny + y) * df.nx + x;
        rc[p] = r[df.off + fi] - apply7_at(df, k, zv, fi, x, y, z);
    }
}

__global__ void __launch_bounds__(B) kappa_grad_b_kernel(Batch b, const double* __restrict__ u,
                                                         const double* __restrict__ lam,
                                                         double* __restrict__ g) {
    i64 lo, hi;
    const Dims d = b.dims[batch_locate(b, blockIdx.x, &lo, &hi)];
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    for (i64 p = lo + threadIdx.x; p < hi; p += B) {
        int x, y, z;
        coords(p - d.off, d.nx, d.ny, &x, &y, &z);
        const double uc = u[p], lc = lam[p];
        const double bnd = lc * uc;
        double s = 0.0;
        s += z > 0 ? 0.5 * (lc - lam[p - sz]) * (uc - u[p - sz]) : bnd;
        s += y > 0 ? 0.5 * (lc - lam[p - sy]) * (uc - u[p - sy]) : bnd;
        s += x > 0 ? 0.5 * (lc - lam[p - 1]) * (uc - u[p - 1]) : bnd;
        s += x < d.nx - 1 ? 0.5 * (lc - lam[p + 1]) * (uc - u[p + 1]) : bnd;
        s += y < d.ny - 1 ? 0.5 * (lc - lam[p + sy]) * (uc - u[p + sy]) : bnd;
        s += z < d.nz - 1 ? 0.5 * (lc - lam[p + sz]) * (uc - u[p + sz]) : bnd;
        g[p] = -s;
    }
}

unsigned blocks_for(i64 n) { return (unsigned)((n + B - 1) / B); }

}  // namespace

cudaError_t launch_kappa_coarsen(Dims f, Dims c, const double* kf, double* kc, cudaStream_t st) {
    if (c.n == 0) return cudaSuccess;
    kappa_coarsen_kernel<<<blocks_for(c.n), B, 0, st>>>(f, c, kf, kc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kappa_setup(Dims d, const double* kappa, KappaLevel<T> k, cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    kappa_setup_kernel<T><<<blocks_for(d.n), B, 0, st>>>(d, kappa, k);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmv7(Dims d, const KappaLevel<T>& k, const T* x, T* y, cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    spmv7_kernel<T><<<blocks_for(d.n), B, 0, st>>>(d, k, x, y);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_qinit7(Dims d, Dims dc, const KappaLevel<T>& k, int up, const T* x, const T* xc,
                          const T* b, T* Q, cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    qinit7_kernel<T><<<blocks_for(d.n), B, 0, st>>>(d, dc, k, up, x, xc, b, Q);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict7(Dims f, Dims c, const KappaLevel<T>& k, const T* r, const T* z, T* rc,
                             cudaStream_t st) {
    if (c.n == 0) return cudaSuccess;
    restrict7_kernel<T><<<blocks_for(c.n), B, 0, st>>>(f, c, k, r, z, rc);
    return cudaGetLastError();
}

cudaError_t launch_kappa_grad(Dims d, const double* u, const double* lam, double* g,
                              cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    kappa_grad_kernel<<<blocks_for(d.n), B, 0, st>>>(d, u, lam, g);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spmv7_b(const Batch& b, const KappaLevel<T>& k, const T* x, T* y,
                           cudaStream_t st) {
    spmv7_b_kernel<T><<<b.nchunks, B, 0, st>>>(b, k, x, y);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_qinit7_b(const Batch& b, const Batch* c, const KappaLevel<T>& k, int up,
                            const T* x, const T* xc, const T* bv, T* Q, cudaStream_t st) {
    qinit7_b_kernel<T><<<b.nchunks, B, 0, st>>>(b, c ? *c : b, c != nullptr, k, up, x, xc, bv, Q);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict7_b(const Batch& f, const Batch& c, const KappaLevel<T>& k,
                               const T* r, const T* z, T* rc, cudaStream_t st) {
    restrict7_b_kernel<T><<<c.nchunks, B, 0, st>>>(f, c, k, r, z, rc);
    return cudaGetLastError();
}

cudaError_t launch_kappa_grad_b(const Batch& b, const double* u, const double* lam, double* g,
                                cudaStream_t st) {
    kappa_grad_b_kernel<<<b.nchunks, B, 0, st>>>(b, u, lam, g);
    return cudaGetLastError();
}

#define M2S_INST7(T)                                                                            \
    template cudaError_t launch_kappa_setup<T>(Dims, const double*, KappaLevel<T>, cudaStream_t); \
    template cudaError_t launch_spmv7<T>(Dims, const KappaLevel<T>&, const T*, T*, cudaStream_t); \
    template cudaError_t launch_qinit7<T>(Dims, Dims, const KappaLevel<T>&, int, const T*,        \
                                          const T*, const T*, T*, cudaStream_t);                  \
    template cudaError_t launch_restrict7<T>(Dims, Dims, const KappaLevel<T>&, const T*,          \
                                             const T*, T*, cudaStream_t);                         \
    template cudaError_t launch_spmv7_b<T>(const Batch&, const KappaLevel<T>&, const T*, T*,      \
                                           cudaStream_t);                                         \
    template cudaError_t launch_qinit7_b<T>(const Batch&, const Batch*, const KappaLevel<T>&, int,  \
                                            const T*, const T*, const T*, T*, cudaStream_t);      \
    template cudaError_t launch_restrict7_b<T>(const Batch&, const Batch&, const KappaLevel<T>&,   \
                                               const T*, const T*, T*, cudaStream_t);
M2S_INST7(double)
M2S_INST7(float)

}  // namespace m2s
