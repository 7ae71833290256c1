// Device-resident CG state of every problem of a grid and the launchers of
// the batched vector kernels.
#pragma once
#include "m2s_internal.cuh"

namespace m2s {

// CG scalars of one problem.  A problem whose residual reaches the tolerance
// is frozen (done = 1: alpha = 0, no further iteration counted) while the
// other problems of the batch go on, so each stops where a solve of its own
// would stop.
struct PcgDev {
    double rho;      // r.z of this iteration
    double rho_old;  // r.z of the previous iteration
    double pq;       // p.Ap
    double alpha;
    double beta;
    double rr;       // |r|^2 after the update
    double bb;       // |b|^2
    double scratch;  // result of a plain dot (FIN_DOT)
    double rtol2;    // stop when rr <= rtol2 * bb (unless fixed)
    int iter;        // completed iterations
    int status;      // 0 or M2S_ERR_BREAKDOWN
    int done;        // converged and frozen
    int fixed;       // run a fixed number of iterations (never freeze)
};

enum FinKind { FIN_BB = 0, FIN_RHO = 1, FIN_PQ = 2, FIN_RR = 3, FIN_DOT = 4 };

// The problems of one level, packed back to back; batched element kernels
// give each CTA one chunk of kChunk elements of one problem, so the partial
// sums of a problem are the contiguous range cstart[i] .. cstart[i+1].
constexpr int kChunk = 2048;
struct Batch {
    int np;
    const Dims* dims;   // device, np entries
    const int* cstart;  // device, np + 1 entries
    int nchunks;
};

// Problem of chunk `blk` of a batched launch and the packed element range
// [*lo, *hi) the chunk covers (binary search on the chunk prefix).
__device__ __forceinline__ int batch_locate(const Batch& b, int blk, i64* lo, i64* hi) {
    int a = 0, c = b.np - 1;
    while (a < c) {
        const int m = (a + c + 1) >> 1;
        if (b.cstart[m] <= blk) a = m;
        else c = m - 1;
    }
    const Dims d = b.dims[a];
    const i64 first = (i64)(blk - b.cstart[a]) * kChunk;
    *lo = d.off + first;
    *hi = d.off + (d.n < first + (i64)kChunk ? d.n : first + (i64)kChunk);
    return a;
}

template <typename T>
cudaError_t launch_dot_b(const Batch& b, const T* x, const T* y, double* partials,
                         cudaStream_t st);
cudaError_t launch_cast_up_dots_b(const Batch& b, const float* z32, const double* r,
                                  const double* zold, double* z, double* part_rz,
                                  double* part_rzo, cudaStream_t st);
// r32 = float(r), and r32s = r32 / 26 when r32s is not NULL
cudaError_t launch_cast_down(i64 n, const double* r, float* r32, float* r32s, cudaStream_t st);
// x += alpha p, r -= alpha q, partial r.r; rs = r / 26 when rs is not NULL
cudaError_t launch_update_b(const Batch& b, const PcgDev* s, const double* p, const double* q,
                            double* x, double* r, double* rs, double* partials, cudaStream_t st);
cudaError_t launch_paxpy_b(const Batch& b, const PcgDev* s, int first, const double* z,
                           const double* pin, double* pout, cudaStream_t st);
// One CTA per problem: sums the problem's partials (range pre[i]..pre[i+1],
// and pre2 for part2) in a fixed order and updates its scalars.  FIN_BB also
// sets the tolerance and the fixed-iterations flag.
cudaError_t launch_finalize_b(int kind, PcgDev* s, int np, const double* part, const int* pre,
                              const double* part2, const int* pre2, double* hist,
                              int hist_stride, double rtol2, int fixed, cudaStream_t st);
// Batched variable-kappa kernels (k_kappa7.cu): one launch for all problems
// of a level; `c` is the coarse level's batch (prolongation / restriction).
template <typename T>
cudaError_t launch_spmv7_b(const Batch& b, const KappaLevel<T>& k, const T* x, T* y,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_qinit7_b(const Batch& b, const Batch* c, const KappaLevel<T>& k, int up,
                            const T* x, const T* xc, const T* bv, T* Q, cudaStream_t st);
template <typename T>
cudaError_t launch_restrict7_b(const Batch& f, const Batch& c, const KappaLevel<T>& k,
                               const T* r, const T* z, T* rc, cudaStream_t st);
cudaError_t launch_kappa_grad_b(const Batch& b, const double* u, const double* lam, double* g,
                                cudaStream_t st);
// p = z + beta p_in, q = A p, p.q partials (st27_num_partials(d) of them):
// the TMA kernel where st27_tma_shape_ok(d, 8), st27_kernel otherwise; err is
// the grid's status word.
cudaError_t launch_pspmv_dot(Dims d, const double* z, const double* pin, double* pout, double* q,
                             const double* beta, double* partials, int* err, cudaStream_t st);

}  // namespace m2s
