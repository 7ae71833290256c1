// Device-resident CG state and the launchers of the vector kernels.
#pragma once
#include "m2s_internal.cuh"

namespace m2s {

struct PcgDev {
    double rho;      // r.z of this iteration
    double rho_old;  // r.z of the previous iteration
    double pq;       // p.Ap
    double alpha;
    double beta;
    double rr;       // |r|^2 after the update
    double bb;       // |b|^2
    double scratch;  // result of a plain dot (FIN_DOT)
    int iter;        // completed iterations
    int status;      // 0 or M2S_ERR_BREAKDOWN
};

enum FinKind { FIN_BB = 0, FIN_RHO = 1, FIN_PQ = 2, FIN_RR = 3, FIN_DOT = 4 };

cudaError_t launch_cast_up_dots(i64 n, const float* z32, const double* r, const double* zold,
                                double* z, double* part_rz, double* part_rzo, cudaStream_t st);
cudaError_t launch_cast_down(i64 n, const double* r, float* r32, cudaStream_t st);
cudaError_t launch_update(i64 n, const PcgDev* s, const double* p, const double* q, double* x,
                          double* r, double* partials, cudaStream_t st);
cudaError_t launch_finalize(int kind, PcgDev* s, const double* part, int np, const double* part2,
                            int np2, double* hist, cudaStream_t st);
cudaError_t launch_pspmv_dot(Dims d, const double* z, const double* pin, double* pout, double* q,
                             const double* beta, double* partials, cudaStream_t st);

}  // namespace m2s

namespace m2s {
cudaError_t launch_paxpy(i64 n, const double* z, const double* pin, double* pout,
                         const double* beta, cudaStream_t st);
}  // namespace m2s
