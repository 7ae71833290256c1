// CG vector kernels for every problem of a grid at once (paper Sec. 6.2.1:
// pointwise operations are fused into their neighbours so that each vector
// is streamed as few times as possible).
//
// The problems' vectors are packed back to back.  A batched launch gives
// each CTA one chunk (kChunk elements) of one problem, found from the chunk
// prefix by binary search, so one launch serves any number of problems and
// the partial sums of a problem form a contiguous range.  Reductions are
// deterministic: a fixed thread-to-element mapping and reduction tree per
// CTA, and a finaliser CTA per problem that sums its partials in a fixed
// order.  The CG scalars live in device memory: an iteration needs no host
// round trip and can be captured in a CUDA graph.
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
__global__ void __launch_bounds__(VB) dot_b_kernel(Batch b, const T* __restrict__ x,
                                                   const T* __restrict__ y, double* partials) {
    __shared__ double sh[VB / 32];
    i64 lo, hi;
    batch_locate(b, blockIdx.x, &lo, &hi);
    double s = 0.0;
    for (i64 i = lo + threadIdx.x; i < hi; i += VB) s = fma((double)x[i], (double)y[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// z = double(z32); partial r.z and (if zold) r.zold
__global__ void __launch_bounds__(VB) cast_up_dots_b_kernel(Batch b, const float* __restrict__ z32,
                                                            const double* __restrict__ r,
                                                            const double* __restrict__ zold,
                                                            double* __restrict__ z,
                                                            double* part_rz, double* part_rzo) {
    __shared__ double sh[VB / 32];
    i64 lo, hi;
    batch_locate(b, blockIdx.x, &lo, &hi);
    double s = 0.0, so = 0.0;
    for (i64 i = lo + threadIdx.x; i < hi; i += VB) {
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

// r32 = float(r); r32s = r32 / 26 when not NULL
__global__ void __launch_bounds__(VB) cast_down_kernel(i64 n, const double* __restrict__ r,
                                                       float* __restrict__ r32,
                                                       float* __restrict__ r32s) {
    for (i64 i = blockIdx.x * (i64)VB + threadIdx.x; i < n; i += (i64)gridDim.x * VB) {
        const float v = (float)r[i];
        r32[i] = v;
        if (r32s) r32s[i] = v * Lit<float>::inv26();
    }
}

// x += alpha p; r -= alpha q (alpha of the chunk's problem); partial r.r;
// rs = r / 26 when not NULL
__global__ void __launch_bounds__(VB) update_b_kernel(Batch b, const PcgDev* __restrict__ s,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ q,
                                                      double* __restrict__ x,
                                                      double* __restrict__ r,
                                                      double* __restrict__ rs, double* partials) {
    __shared__ double sh[VB / 32];
    i64 lo, hi;
    const int pb = batch_locate(b, blockIdx.x, &lo, &hi);
    const double alpha = s[pb].alpha;
    double acc = 0.0;
    for (i64 i = lo + threadIdx.x; i < hi; i += VB) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        if (rs) rs[i] = ri * Lit<double>::inv26();
        acc = fma(ri, ri, acc);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// pout = z + beta pin (beta of the chunk's problem); pout = z when first
__global__ void __launch_bounds__(VB) paxpy_b_kernel(Batch b, const PcgDev* __restrict__ s,
                                                     int first, const double* __restrict__ z,
                                                     const double* __restrict__ pin,
                                                     double* __restrict__ pout) {
    i64 lo, hi;
    const int pb = batch_locate(b, blockIdx.x, &lo, &hi);
    const double beta = first ? 0.0 : s[pb].beta;
    for (i64 i = lo + threadIdx.x; i < hi; i += VB) pout[i] = first ? z[i] : fma(beta, pin[i], z[i]);
}

// Sum of part[lo..hi) by one CTA in a fixed order.
__device__ __forceinline__ double reduce_range(const double* part, int lo, int hi, double* sh) {
    double s = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) s += part[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[w] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(1024) finalize_b_kernel(int kind, PcgDev* st, const double* part,
                                                          const int* pre, const double* part2,
                                                          const int* pre2, double* hist,
                                                          int hist_stride, double rtol2,
                                                          int fixed) {
    __shared__ double sh[32];
    const int pb = blockIdx.x;
    const double v = reduce_range(part, pre[pb], pre[pb + 1], sh);
    double v2 = 0.0;
    if (part2) v2 = reduce_range(part2, pre2[pb], pre2[pb + 1], sh);
    if (threadIdx.x != 0) return;
    PcgDev* s = st + pb;
    double* h = hist ? hist + (i64)pb * hist_stride : nullptr;
    switch (kind) {
        case FIN_BB:
            s->bb = v;
            s->rr = v;
            s->iter = 0;
            s->status = 0;
            s->done = 0;
            s->rtol2 = rtol2;
            s->fixed = fixed;
            if (h) h[0] = sqrt(v);
            break;
        case FIN_RHO: {
            if (s->done) break;
            const bool first = s->iter == 0;
            s->rho = v;
            double beta = 0.0;
            if (!first) beta = part2 ? (v - v2) / s->rho_old : v / s->rho_old;
            s->beta = beta;
            if (!isfinite(v) || !isfinite(beta)) s->status = (int)M2S_ERR_BREAKDOWN;
            break;
        }
        case FIN_PQ: {
            if (s->done) {
                s->alpha = 0.0;
                break;
            }
            s->pq = v;
            const bool bad = !(v > 0.0) || !isfinite(v) || s->status != 0;
            s->alpha = bad ? 0.0 : s->rho / v;
            if (bad) s->status = (int)M2S_ERR_BREAKDOWN;
            break;
        }
        case FIN_RR: {
            if (s->done) break;
            s->rr = v;
            s->rho_old = s->rho;
            s->iter += 1;
            if (h && s->iter < hist_stride) h[s->iter] = sqrt(v);
            if (!isfinite(v)) s->status = (int)M2S_ERR_BREAKDOWN;
            if (!s->fixed && v <= s->rtol2 * s->bb) s->done = 1;
            break;
        }
        case FIN_DOT:
            s->scratch = v;
            break;
    }
}

inline unsigned grid_of(const Batch& b) { return (unsigned)(b.nchunks > 0 ? b.nchunks : 1); }

}  // namespace

template <typename T>
cudaError_t launch_dot_b(const Batch& b, const T* x, const T* y, double* partials,
                         cudaStream_t st) {
    dot_b_kernel<T><<<grid_of(b), VB, 0, st>>>(b, x, y, partials);
    return cudaGetLastError();
}

cudaError_t launch_cast_up_dots_b(const Batch& b, const float* z32, const double* r,
                                  const double* zold, double* z, double* part_rz,
                                  double* part_rzo, cudaStream_t st) {
    cast_up_dots_b_kernel<<<grid_of(b), VB, 0, st>>>(b, z32, r, zold, z, part_rz, part_rzo);
    return cudaGetLastError();
}

cudaError_t launch_cast_down(i64 n, const double* r, float* r32, float* r32s, cudaStream_t st) {
    i64 g = (n + (i64)VB * 8 - 1) / ((i64)VB * 8);
    g = g < 1 ? 1 : (g > 4096 ? 4096 : g);
    cast_down_kernel<<<(unsigned)g, VB, 0, st>>>(n, r, r32, r32s);
    return cudaGetLastError();
}

cudaError_t launch_update_b(const Batch& b, const PcgDev* s, const double* p, const double* q,
                            double* x, double* r, double* rs, double* partials, cudaStream_t st) {
    update_b_kernel<<<grid_of(b), VB, 0, st>>>(b, s, p, q, x, r, rs, partials);
    return cudaGetLastError();
}

cudaError_t launch_paxpy_b(const Batch& b, const PcgDev* s, int first, const double* z,
                           const double* pin, double* pout, cudaStream_t st) {
    paxpy_b_kernel<<<grid_of(b), VB, 0, st>>>(b, s, first, z, pin, pout);
    return cudaGetLastError();
}

cudaError_t launch_finalize_b(int kind, PcgDev* s, int np, const double* part, const int* pre,
                              const double* part2, const int* pre2, double* hist,
                              int hist_stride, double rtol2, int fixed, cudaStream_t st) {
    finalize_b_kernel<<<np, 1024, 0, st>>>(kind, s, part, pre, part2, pre2, hist, hist_stride,
                                           rtol2, fixed);
    return cudaGetLastError();
}

template cudaError_t launch_dot_b<double>(const Batch&, const double*, const double*, double*,
                                          cudaStream_t);
template cudaError_t launch_dot_b<float>(const Batch&, const float*, const float*, double*,
                                         cudaStream_t);

}  // namespace m2s
