// 27-point (HPCG) Jacobi-style stencil kernels: SpMV, the fused p-update +
// SpMV + p.Ap of CG, the old-neighbour sums that seed a Gauss-Seidel sweep,
// residual restriction and prolongation.
//
// Operator (paper Sec. 7.1, HPCG; Sec. 4.3.1 SpMV): a_pp = 26, a_pq = -1 for
// the in-domain points of the 3x3x3 box, out-of-domain neighbours dropped.
// On GB300 FP64 arithmetic issues at 2 lanes/clk/SM, far below the HBM rate,
// so the sum over the box is evaluated separably -- row 3-sums H, plane 3x3
// sums S2 = H(y-1)+H(y)+H(y+1), box = S2(z-1)+S2(z)+S2(z+1) -- and
// y = 27 x_p - box (one FMA): about 7.5 FP64 operations per point instead of
// 27.  The re-association is exact for integer data (b = A*ones) and within
// a few ulps otherwise.
//
// Tiling: a CTA of 32 x 8 threads owns a 32 x 8 column of (x, y) and marches
// ZC planes in z; each plane (with a one-point halo) is staged in shared
// memory, its row sums computed once, and the per-plane 3x3 sums are carried
// in registers across the z march, so every input plane is read once per
// CTA (plus the two halo planes).
#include "m2s_internal.cuh"
#include "m2s_pcg.cuh"

namespace m2s {

namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int ZC = 8;

template <typename T>
struct St27Args {
    Dims d;      // this level
    Dims dc;     // coarse level (PROLONG_QUP)
    const T* x;  // input field (x, z or the fine correction)
    const T* xc; // coarse correction (PROLONG_QUP)
    const T* b;  // right-hand side (Q modes) / p_in (PSPMV_DOT)
    T* y;        // output (A x, q, or Q)
    T scale;     // Q modes: Q is written times this (1 or 1/26)
    T* bs;       // Q modes: b * scale is also written here when not NULL
    T* pout;     // PSPMV_DOT: updated search direction
    const double* beta;  // PSPMV_DOT: device beta, NULL => p = z
    double* partials;    // PSPMV_DOT: one p.q partial per CTA
};

template <typename T, int MODE>
__device__ __forceinline__ T load_pt(const St27Args<T>& a, i64 q, int qx, int qy, int qz, T beta) {
    if (MODE == ST27_PSPMV_DOT) {
        T z = a.x[q];
        if (a.beta == nullptr) return z;
        return z + beta * a.b[q];
    }
    if (MODE == ST27_PROLONG_QUP) {
        T v = a.x[q];
        if (((qx | qy | qz) & 1) == 0) {
            i64 c = a.dc.off + ((i64)(qz >> 1) * a.dc.ny + (qy >> 1)) * a.dc.nx + (qx >> 1);
            v += a.xc[c];
        }
        return v;
    }
    return a.x[q];
}

template <typename T, int MODE>
__global__ void __launch_bounds__(TX * TY) st27_kernel(St27Args<T> a) {
    __shared__ T sv[TY + 2][TX + 2];
    __shared__ T sh[TY + 2][TX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = a.d.nx, ny = a.d.ny, nz = a.d.nz;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * ZC;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    T beta = T(0);
    if (MODE == ST27_PSPMV_DOT && a.beta != nullptr) beta = (T)(*a.beta);

    // per-plane quantities of the two previous planes
    T s2_m2 = T(0), s2_m1 = T(0);            // 3x3 sums of planes zl-2, zl-1
    T c_m1 = T(0), hup_m1 = T(0), hdn_m1 = T(0), xl_m1 = T(0), xr_m1 = T(0);
    double part = 0.0;
    const int zend = min(z0 + ZC, nz);

    for (int zl = z0 - 1; zl <= zend; ++zl) {
        for (int i = tid; i < (TY + 2) * (TX + 2); i += TX * TY) {
            const int ly = i / (TX + 2), lx = i - ly * (TX + 2);
            const int qx = x0 + lx - 1, qy = y0 + ly - 1;
            T v = T(0);
            if (zl >= 0 && zl < nz && qx >= 0 && qx < nx && qy >= 0 && qy < ny) {
                const i64 q = a.d.off + ((i64)zl * ny + qy) * nx + qx;
                v = load_pt<T, MODE>(a, q, qx, qy, zl, beta);
            }
            sv[ly][lx] = v;
        }
        __syncthreads();
        for (int i = tid; i < (TY + 2) * TX; i += TX * TY) {
            const int ly = i / TX, lx = i - ly * TX;
            sh[ly][lx] = (sv[ly][lx] + sv[ly][lx + 1]) + sv[ly][lx + 2];
        }
        __syncthreads();
        const T hdn = sh[ty][tx], hc = sh[ty + 1][tx], hup = sh[ty + 2][tx];
        const T s2 = (hdn + hc) + hup;
        const T c = sv[ty + 1][tx + 1];
        const T xl = sv[ty + 1][tx], xr = sv[ty + 1][tx + 2];
        __syncthreads();

        const int zo = zl - 1;  // output plane
        if (zo >= z0 && zo < zend && own) {
            const i64 p = a.d.off + ((i64)zo * ny + gy) * nx + gx;
            if (MODE == ST27_SPMV || MODE == ST27_PSPMV_DOT) {
                const T box = (s2_m2 + s2_m1) + s2;
                const T yv = fma(T(27), c_m1, -box);
                a.y[p] = yv;
                if (MODE == ST27_PSPMV_DOT) {
                    a.pout[p] = c_m1;
                    part = fma((double)c_m1, (double)yv, part);
                }
            } else {
                const T bp = a.b[p];
                const T q = MODE == ST27_QLO ? ((bp + s2_m2) + hdn_m1) + xl_m1
                                             : ((bp + s2) + hup_m1) + xr_m1;  // QUP, PROLONG_QUP
                a.y[p] = q * a.scale;
                if (a.bs) a.bs[p] = bp * a.scale;
            }
        }
        s2_m2 = s2_m1;
        s2_m1 = s2;
        c_m1 = c;
        hup_m1 = hup;
        hdn_m1 = hdn;
        xl_m1 = xl;
        xr_m1 = xr;
    }

    if (MODE == ST27_PSPMV_DOT) {
        // fixed-shape reduction: warp tree, then the 8 warp sums in order
        __shared__ double wsum[TY];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (tx == 0) wsum[ty] = part;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < TY; ++w) s += wsum[w];
            const int bid = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            a.partials[bid] = s;
        }
    }
}

template <typename T>
__global__ void restrict27_kernel(Dims f, Dims c, const T* __restrict__ r,
                                  const T* __restrict__ z, T* __restrict__ rc,
                                  T* __restrict__ rcs) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const int cx = (int)(i % c.nx);
    const int cy = (int)((i / c.nx) % c.ny);
    const int cz = (int)(i / ((i64)c.nx * c.ny));
    const int fx = 2 * cx, fy = 2 * cy, fz = 2 * cz;
    T box = T(0);
    for (int dz = -1; dz <= 1; ++dz) {
        const int qz = fz + dz;
        if (qz < 0 || qz >= f.nz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int qy = fy + dy;
            if (qy < 0 || qy >= f.ny) continue;
            const T* row = z + f.off + ((i64)qz * f.ny + qy) * f.nx;
            T h = T(0);
            for (int dx = -1; dx <= 1; ++dx) {
                const int qx = fx + dx;
                if (qx >= 0 && qx < f.nx) h += row[qx];
            }
            box += h;
        }
    }
    const i64 p = f.off + ((i64)fz * f.ny + fy) * f.nx + fx;
    const T az = fma(T(27), z[p], -box);
    const T v = r[p] - az;
    rc[c.off + i] = v;
    if (rcs) rcs[c.off + i] = v * Lit<T>::inv26();
}

template <typename T>
__global__ void scale_kernel(i64 n, const T* __restrict__ x, T* __restrict__ y) {
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
        y[i] = x[i] * Lit<T>::inv26();
}

template <typename T>
__global__ void prolong_kernel(Dims f, Dims c, const T* __restrict__ zc, T* __restrict__ z) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    const int cx = (int)(i % c.nx);
    const int cy = (int)((i / c.nx) % c.ny);
    const int cz = (int)(i / ((i64)c.nx * c.ny));
    const i64 p = f.off + ((i64)(2 * cz) * f.ny + 2 * cy) * f.nx + 2 * cx;
    z[p] += zc[c.off + i];
}

dim3 st27_grid(Dims d) {
    return dim3((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, (d.nz + ZC - 1) / ZC);
}

}  // namespace

int st27_num_partials(Dims d) {
    if (st27_tma_shape_ok(d, sizeof(double))) return st27_tma_pcg_partials(d);
    dim3 g = st27_grid(d);
    return (int)(g.x * g.y * g.z);
}

template <typename T>
cudaError_t launch_spmv27(Dims d, const T* x, T* y, int* err, cudaStream_t st) {
    const cudaError_t e = launch_spmv27_tma<T>(d, x, y, err, st);
    if (e != cudaErrorNotSupported) return e;
    return launch_st27<T>(ST27_SPMV, d, d, x, nullptr, nullptr, y, st);
}

template <typename T>
cudaError_t st27_run(St27Mode mode, Dims d, Dims dc, const T* x, const T* xc, const T* b, T* y,
                     T scale, T* bs, cudaStream_t st) {
    St27Args<T> a;
    a.d = d;
    a.dc = dc;
    a.x = x;
    a.xc = xc;
    a.b = b;
    a.y = y;
    a.scale = scale;
    a.bs = bs;
    a.pout = nullptr;
    a.beta = nullptr;
    a.partials = nullptr;
    if (d.n == 0) return cudaSuccess;
    dim3 g = st27_grid(d), blk(TX, TY);
    switch (mode) {
        case ST27_SPMV: st27_kernel<T, ST27_SPMV><<<g, blk, 0, st>>>(a); break;
        case ST27_QUP: st27_kernel<T, ST27_QUP><<<g, blk, 0, st>>>(a); break;
        case ST27_QLO: st27_kernel<T, ST27_QLO><<<g, blk, 0, st>>>(a); break;
        case ST27_PROLONG_QUP: st27_kernel<T, ST27_PROLONG_QUP><<<g, blk, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_st27(St27Mode mode, Dims d, Dims dc, const T* x, const T* xc, const T* b, T* y,
                        cudaStream_t st) {
    return st27_run<T>(mode, d, dc, x, xc, b, y, T(1), nullptr, st);
}

template <typename T>
cudaError_t launch_st27_q26(St27Mode mode, Dims d, Dims dc, const T* x, const T* xc, const T* b,
                            T* Q, T* bs, cudaStream_t st) {
    if (mode == ST27_SPMV || mode == ST27_PSPMV_DOT) return cudaErrorInvalidValue;
    return st27_run<T>(mode, d, dc, x, xc, b, Q, T(1) / T(26), bs, st);
}

template <typename T>
cudaError_t launch_scale26(i64 n, const T* x, T* y, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    i64 g = (n + 256 * 8 - 1) / (256 * 8);
    g = g < 1 ? 1 : (g > 4096 ? 4096 : g);
    scale_kernel<T><<<(unsigned)g, 256, 0, st>>>(n, x, y);
    return cudaGetLastError();
}

// p-update + SpMV + dot: pout = z + beta*pin (beta NULL => pout = z),
// q = A pout, partials[cta] = sum pout.q over the CTA.
cudaError_t launch_pspmv_dot(Dims d, const double* z, const double* pin, double* pout,
                             double* q, const double* beta, double* partials, int* err,
                             cudaStream_t st) {
    // the partial count was fixed by st27_num_partials: no fallback from here
    if (st27_tma_shape_ok(d, sizeof(double)))
        return launch_pspmv_dot_tma(d, z, pin, pout, q, beta, partials, err, st);
    St27Args<double> a;
    a.d = d;
    a.dc = d;
    a.x = z;
    a.xc = nullptr;
    a.b = pin;
    a.y = q;
    a.scale = 1.0;
    a.bs = nullptr;
    a.pout = pout;
    a.beta = beta;
    a.partials = partials;
    if (d.n == 0) return cudaSuccess;
    st27_kernel<double, ST27_PSPMV_DOT><<<st27_grid(d), dim3(TX, TY), 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict27(Dims f, Dims c, const T* r, const T* z, T* rc, T* rcs,
                              cudaStream_t st) {
    if (c.n == 0) return cudaSuccess;
    const int bs = 256;
    restrict27_kernel<T><<<(unsigned)((c.n + bs - 1) / bs), bs, 0, st>>>(f, c, r, z, rc, rcs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(Dims f, Dims c, const T* zc, T* z, cudaStream_t st) {
    if (c.n == 0) return cudaSuccess;
    const int bs = 256;
    prolong_kernel<T><<<(unsigned)((c.n + bs - 1) / bs), bs, 0, st>>>(f, c, zc, z);
    return cudaGetLastError();
}

template cudaError_t launch_st27<double>(St27Mode, Dims, Dims, const double*, const double*,
                                         const double*, double*, cudaStream_t);
template cudaError_t launch_st27<float>(St27Mode, Dims, Dims, const float*, const float*,
                                        const float*, float*, cudaStream_t);
template cudaError_t launch_st27_q26<double>(St27Mode, Dims, Dims, const double*, const double*,
                                             const double*, double*, double*, cudaStream_t);
template cudaError_t launch_st27_q26<float>(St27Mode, Dims, Dims, const float*, const float*,
                                            const float*, float*, float*, cudaStream_t);
template cudaError_t launch_spmv27<double>(Dims, const double*, double*, int*, cudaStream_t);
template cudaError_t launch_spmv27<float>(Dims, const float*, float*, int*, cudaStream_t);
template cudaError_t launch_scale26<double>(i64, const double*, double*, cudaStream_t);
template cudaError_t launch_scale26<float>(i64, const float*, float*, cudaStream_t);
template cudaError_t launch_restrict27<double>(Dims, Dims, const double*, const double*, double*,
                                               double*, cudaStream_t);
template cudaError_t launch_restrict27<float>(Dims, Dims, const float*, const float*, float*,
                                              float*, cudaStream_t);
template cudaError_t launch_prolong<double>(Dims, Dims, const double*, double*, cudaStream_t);
template cudaError_t launch_prolong<float>(Dims, Dims, const float*, float*, cudaStream_t);

}  // namespace m2s
