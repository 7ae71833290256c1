// 5x5-block 7-point operator (NPB-LU shape) and its SSOR step.
#pragma once
#include <functional>
#include <vector>

#include "m2s_internal.cuh"

namespace m2s {

constexpr int JP = 2 + 4 * 55;  // parameters of the blocks formed from the state

struct BlockOp {
    int np = 0;
    bool jac = false;           // blocks formed from u every step (op BLOCK7_JAC)
    double* P = nullptr;        // [np][JP] their parameters (op BLOCK7_JAC)
    double* h = nullptr;        // [3][npts][5] flux products J_d(u_q) u_q (op BLOCK7_JAC)
    std::vector<double> nu;     // per problem: nu of its parameters (op BLOCK7_JAC)
    std::vector<Dims> dims;     // per problem (points; vectors hold 5 per point)
    i64 npts = 0;               // total points
    // op BLOCK7_5x5: D, L, U and D^-1 entry-major, entry k of point p at
    // [k][npts] (L, U: k = d * 25 + r * 5 + c, couplings to p -/+ e_{x,y,z});
    // D, L, U are not allocated for BLOCK7_JAC
    double* D = nullptr;        // [25][npts]
    double* L = nullptr;        // [75][npts]
    double* U = nullptr;        // [75][npts]
    double* Dinv = nullptr;     // [25][npts] (BLOCK7_JAC: w D^-1 of the current step, [npts][25])
    double* M = nullptr;        // [npts][3][25]  omega D^-1 L (0 off the grid; BLOCK7_JAC: L)
    double* N = nullptr;        // [npts][3][25]  omega D^-1 U (0 off the grid; BLOCK7_JAC: U)
    double* s = nullptr;        // [npts][5] D^-1 (b - A u) (BLOCK7_JAC: (b - A(u) u) / w)
    double* v = nullptr;        // [npts][5] lower-sweep result (BLOCK7_JAC: b - D u until then)
    double* w = nullptr;        // [npts][5] upper-sweep result
    double omega = -1.0;        // omega that M and N were built for
    WaveUnits sweep;            // CTA wavefront units of all problems (one launch)
};

using BlockAlloc = std::function<cudaError_t(void**, size_t)>;

cudaError_t block_create(BlockOp* b, const m2s_grid_desc* descs, int n_problems,
                         const std::vector<std::vector<Dims>>& dims, cudaStream_t st,
                         BlockAlloc alloc);
cudaError_t block_apply(BlockOp* b, const double* u, double* y, cudaStream_t st);
cudaError_t block_ssor_iter(BlockOp* b, const double* rhs, double* u, double omega,
                            DevStatus* status, long long spin_ns, cudaStream_t st);
void block_free_units(BlockOp* b);

}  // namespace m2s
