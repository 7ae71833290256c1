// CG vector kernels (paper Sec. 6.2.1: pointwise operations are fused into
// their neighbours so that each vector is streamed as few times as possible).
//
// Reductions are deterministic: every kernel writes one partial per CTA with
// a fixed thread-to-element mapping and a fixed reduction tree, and a
// single-CTA finaliser sums the partials in a fixed order.  The CG scalars
// (rho, alpha, beta, |r|) live in device memory, so an iteration needs no
// host round trip and can be captured in a CUDA graph.
#include "m2s_internal.cuh"
#include "m2s_pcg.cuh"

namespace m2s {

namespace {

constexpr int VB = 256;  // threads per CTA of the streaming kernels

__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    __syncthreads();
    return s;  // valid in thread 0
}

template <typename T>
__global__ void __launch_bounds__(VB) dot_kernel(i64 n, const T* __restrict__ a,
                                                 const T* __restrict__ b, double* partials) {
    __shared__ double sh[VB / 32];
    double s = 0.0;
    for (i64 i = blockIdx.x * (i64)VB + threadIdx.x; i < n; i += (i64)gridDim.x * VB)
        s = fma((double)a[i], (double)b[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// z = double(z32); partial r.z and (if zold) r.zold
__global__ void __launch_bounds__(VB) cast_up_dots_kernel(i64 n, const float* __restrict__ z32,
                                                          const double* __restrict__ r,
                                                          const double* __restrict__ zold,
                                                          double* __restrict__ z,
                                                          double* part_rz, double* part_rzo) {
    __shared__ double sh[VB / 32];
    double s = 0.0, so = 0.0;
    for (i64 i = blockIdx.x * (i64)VB + threadIdx.x; i < n; i += (i64)gridDim.x * VB) {
        const double zi = (double)z32[i];
        const double ri = r[i];
        z[i] = zi;
        s = fma(ri, zi, s);
        if (zold) so = fma(ri, zold[i], so);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part_rz[blockIdx.x] = s;
    if (zold) {
        so = block_sum(so, sh);
        if (threadIdx.x == 0) part_rzo[blockIdx.x] = so;
    }
}

__global__ void __launch_bounds__(VB) cast_down_kernel(i64 n, const double* __restrict__ r,
                                                       float* __restrict__ r32) {
    for (i64 i = blockIdx.x * (i64)VB + threadIdx.x; i < n; i += (i64)gridDim.x * VB)
        r32[i] = (float)r[i];
}

// x += alpha p; r -= alpha q; partial r.r
__global__ void __launch_bounds__(VB) update_kernel(i64 n, const PcgDev* __restrict__ s,
                                                    const double* __restrict__ p,
                                                    const double* __restrict__ q,
                                                    double* __restrict__ x,
                                                    double* __restrict__ r, double* partials) {
    __shared__ double sh[VB / 32];
    const double alpha = s->alpha;
    double acc = 0.0;
    for (i64 i = blockIdx.x * (i64)VB + threadIdx.x; i < n; i += (i64)gridDim.x * VB) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Single-CTA reduction of `np` partials in a fixed order.
__device__ __forceinline__ double reduce_partials(const double* part, int np, double* sh) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[w] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;
}

__global__ void __launch_bounds__(1024) finalize_kernel(int kind, PcgDev* s, const double* part,
                                                        int np, const double* part2, int np2,
                                                        double* hist) {
    __shared__ double sh[32];
    const double v = reduce_partials(part, np, sh);
    __syncthreads();
    double v2 = 0.0;
    if (part2) v2 = reduce_partials(part2, np2, sh);
    if (threadIdx.x != 0) return;
    switch (kind) {
        case FIN_BB:
            s->bb = v;
            s->rr = v;
            s->iter = 0;
            s->status = 0;
            if (hist) hist[0] = sqrt(v);
            break;
        case FIN_RHO: {
            const bool first = s->iter == 0;
            s->rho = v;
            double beta = 0.0;
            if (!first) beta = part2 ? (v - v2) / s->rho_old : v / s->rho_old;
            s->beta = beta;
            if (!isfinite(v) || !isfinite(beta)) s->status = (int)M2S_ERR_BREAKDOWN;
            break;
        }
        case FIN_PQ: {
            s->pq = v;
            const bool bad = !(v > 0.0) || !isfinite(v) || s->status != 0;
            s->alpha = bad ? 0.0 : s->rho / v;
            if (bad) s->status = (int)M2S_ERR_BREAKDOWN;
            break;
        }
        case FIN_RR: {
            s->rr = v;
            s->rho_old = s->rho;
            s->iter += 1;
            if (hist) hist[s->iter] = sqrt(v);
            if (!isfinite(v)) s->status = (int)M2S_ERR_BREAKDOWN;
            break;
        }
        case FIN_DOT:
            s->scratch = v;
            break;
    }
}

int grid_for(i64 n) {
    i64 g = (n + (i64)VB * 8 - 1) / ((i64)VB * 8);
    if (g < 1) g = 1;
    if (g > 2048) g = 2048;
    return (int)g;
}

}  // namespace

int dot_num_partials(i64 n) { return grid_for(n); }

template <typename T>
cudaError_t launch_dot_partials(i64 n, const T* a, const T* b, double* partials, int nparts,
                                cudaStream_t st) {
    (void)nparts;
    dot_kernel<T><<<grid_for(n), VB, 0, st>>>(n, a, b, partials);
    return cudaGetLastError();
}

cudaError_t launch_cast_up_dots(i64 n, const float* z32, const double* r, const double* zold,
                                double* z, double* part_rz, double* part_rzo, cudaStream_t st) {
    cast_up_dots_kernel<<<grid_for(n), VB, 0, st>>>(n, z32, r, zold, z, part_rz, part_rzo);
    return cudaGetLastError();
}

cudaError_t launch_cast_down(i64 n, const double* r, float* r32, cudaStream_t st) {
    cast_down_kernel<<<grid_for(n), VB, 0, st>>>(n, r, r32);
    return cudaGetLastError();
}

cudaError_t launch_update(i64 n, const PcgDev* s, const double* p, const double* q, double* x,
                          double* r, double* partials, cudaStream_t st) {
    update_kernel<<<grid_for(n), VB, 0, st>>>(n, s, p, q, x, r, partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int kind, PcgDev* s, const double* part, int np, const double* part2,
                            int np2, double* hist, cudaStream_t st) {
    finalize_kernel<<<1, 1024, 0, st>>>(kind, s, part, np, part2, np2, hist);
    return cudaGetLastError();
}

template cudaError_t launch_dot_partials<double>(i64, const double*, const double*, double*, int,
                                                 cudaStream_t);
template cudaError_t launch_dot_partials<float>(i64, const float*, const float*, double*, int,
                                                cudaStream_t);

}  // namespace m2s

namespace m2s {
namespace {
// pout = z + beta * pin  (beta == NULL: pout = z)
__global__ void __launch_bounds__(256) paxpy_kernel(i64 n, const double* __restrict__ z,
                                                    const double* __restrict__ pin,
                                                    double* __restrict__ pout,
                                                    const double* __restrict__ beta) {
    const double b = beta ? *beta : 0.0;
    for (i64 i = blockIdx.x * (i64)256 + threadIdx.x; i < n; i += (i64)gridDim.x * 256)
        pout[i] = beta ? fma(b, pin[i], z[i]) : z[i];
}
}  // namespace

cudaError_t launch_paxpy(i64 n, const double* z, const double* pin, double* pout,
                         const double* beta, cudaStream_t st) {
    i64 g = (n + 2047) / 2048;
    if (g < 1) g = 1;
    if (g > 2048) g = 2048;
    paxpy_kernel<<<(unsigned)g, 256, 0, st>>>(n, z, pin, pout, beta);
    return cudaGetLastError();
}
}  // namespace m2s
