// 5x5-block 7-point operator in the shape of NPB-LU and its SSOR step
// (paper Sec. 1 and Sec. 4.3.3: SSOR among the routines with spatial
// dependence; Sec. 4.2.3: inner values are 5-vectors and 5x5 blocks).
//
// One SSOR step from u (Saad, Iterative Methods, Sec. 4.1.2):
//   s = D^-1 (b - A u)                       Jacobi-style, fully parallel
//   lower, p increasing:  v_p = s_p - sum_d M_{p,d} v_{p-e_d},  M = w D^-1 L
//   upper, p decreasing:  w_p = v_p - sum_d N_{p,d} w_{p+e_d},  N = w D^-1 U
//   u += w(2-w) w_p      (fused into the upper sweep)
// which is (D + wL) v = r and (D + wU) w = D v with D^-1 applied once per
// point per step instead of one 5x5 elimination per point per sweep: the
// products w D^-1 L and w D^-1 U are formed once per omega at set-up.
//
// The sweeps run on the wavefront machinery of k_wave.cu (hyperplane
// x + y + z, one progress counter per unit, ticketed units), with FIVE lanes
// per grid point -- lane c computes component c -- so that a wavefront step
// costs 15 FMAs per lane instead of 75 (the FP64 pipe of a GB300 SM
// sub-partition retires one warp instruction per ~32 ns whatever the
// number of active lanes).  A warp holds 6 point rows in y (group 0 is the
// halo row replayed from the producer) and K register slots in z.
#include <algorithm>

#include "m2s_block.cuh"
#include "m2s_wave_sync.cuh"

namespace m2s {

namespace {

using namespace wave;

constexpr int KB = 3;  // slots per lane (incl. the halo slot)
constexpr int GROUPS = 6;

__device__ __forceinline__ void coords(i64 i, int nx, int ny, int* x, int* y, int* z) {
    *x = (int)(i % nx);
    const i64 r = i / nx;
    *y = (int)(r % ny);
    *z = (int)(r / ny);
}

// In-place inverse of a 5x5 matrix by Gauss-Jordan elimination without
// pivoting (the blocks are diagonally dominant).
__device__ void inv5(const double* a, double* out) {
    double m[5][10];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            m[i][j] = a[i * 5 + j];
            m[i][5 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int k = 0; k < 5; ++k) {
        const double piv = 1.0 / m[k][k];
        for (int j = 0; j < 10; ++j) m[k][j] *= piv;
        for (int i = 0; i < 5; ++i) {
            if (i == k) continue;
            const double f = m[i][k];
            for (int j = 0; j < 10; ++j) m[i][j] -= f * m[k][j];
        }
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) out[i * 5 + j] = m[i][5 + j];
}

__global__ void block_setup_kernel(Dims d, const double* __restrict__ D,
                                   const double* __restrict__ L, const double* __restrict__ U,
                                   double omega, double* __restrict__ Dinv,
                                   double* __restrict__ M, double* __restrict__ N) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 p = d.off + i;
    double di[25];
    inv5(D + p * 25, di);
    for (int k = 0; k < 25; ++k) Dinv[p * 25 + k] = di[k];
    const bool lo[3] = {x > 0, y > 0, z > 0};
    const bool hi[3] = {x < d.nx - 1, y < d.ny - 1, z < d.nz - 1};
    for (int dd = 0; dd < 3; ++dd) {
        const double* Lb = L + (p * 3 + dd) * 25;
        const double* Ub = U + (p * 3 + dd) * 25;
        for (int r = 0; r < 5; ++r)
            for (int c = 0; c < 5; ++c) {
                double sl = 0.0, su = 0.0;
                for (int k = 0; k < 5; ++k) {
                    sl = fma(di[r * 5 + k], Lb[k * 5 + c], sl);
                    su = fma(di[r * 5 + k], Ub[k * 5 + c], su);
                }
                M[(p * 3 + dd) * 25 + r * 5 + c] = lo[dd] ? omega * sl : 0.0;
                N[(p * 3 + dd) * 25 + r * 5 + c] = hi[dd] ? omega * su : 0.0;
            }
    }
}

// y = A u, or (resid) s = D^-1 (b - A u).  One thread per point.
template <bool RESID>
__global__ void block_apply_kernel(Dims d, const double* __restrict__ D,
                                   const double* __restrict__ L, const double* __restrict__ U,
                                   const double* __restrict__ Dinv, const double* __restrict__ b,
                                   const double* __restrict__ u, double* __restrict__ out) {
    const i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    int x, y, z;
    coords(i, d.nx, d.ny, &x, &y, &z);
    const i64 p = d.off + i;
    const i64 sy = d.nx, sz = (i64)d.nx * d.ny;
    double acc[5] = {0, 0, 0, 0, 0};
    auto mv = [&](const double* B, i64 q) {
        const double* uq = u + q * 5;
        double v[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) v[c] = uq[c];
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[r] = fma(B[r * 5 + c], v[c], acc[r]);
    };
    if (z > 0) mv(L + (p * 3 + 2) * 25, p - sz);
    if (y > 0) mv(L + (p * 3 + 1) * 25, p - sy);
    if (x > 0) mv(L + (p * 3 + 0) * 25, p - 1);
    mv(D + p * 25, p);
    if (x < d.nx - 1) mv(U + (p * 3 + 0) * 25, p + 1);
    if (y < d.ny - 1) mv(U + (p * 3 + 1) * 25, p + sy);
    if (z < d.nz - 1) mv(U + (p * 3 + 2) * 25, p + sz);
    if constexpr (!RESID) {
#pragma unroll
        for (int r = 0; r < 5; ++r) out[p * 5 + r] = acc[r];
        return;
    } else {
    double rr[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) rr[r] = b[p * 5 + r] - acc[r];
    const double* Di = Dinv + p * 25;
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 5; ++c) s = fma(Di[r * 5 + c], rr[c], s);
        out[p * 5 + r] = s;
    }
    }
}

struct BlockWaveArgs {
    int nx, ny, nz;
    i64 n, off;
    int rev, publish_every;
    long long spin_ns;
    const double* coup;  // [n][3][25]: M (forward) or N (backward)
    const double* rhs;   // [n][5]: s (forward) or v (backward)
    double* out;         // [n][5]: v or w
    double* u;           // backward only: u += cu * w  (may be NULL)
    double cu;
    const int2* origin;
    const int4* prod;
    int n_units;
    int* flags;
    int* ctrl;
    DevStatus* status;
};

__device__ __forceinline__ void unit_block(const BlockWaveArgs& a, int t) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int gi = lane / 5, ci = lane - 5 * (lane / 5);
    const int gbase = 5 * gi;
    const bool active = gi < GROUPS;
    const int2 org = a.origin[t];
    const int4 pr = a.prod[t];
    const int y = org.x - 1 + gi;
    const int tbase = (org.x - 1) + (org.y - 1);
    const bool has_prod = pr.x >= 0 || pr.y >= 0;

    bool rv[KB];
    i64 base[KB];
    const i64 dir = a.rev ? -1 : 1;
#pragma unroll
    for (int j = 0; j < KB; ++j) {
        const int z = org.y - 1 + j;
        rv[j] = active && z >= 0 && z < a.nz && y >= 0 && y < a.ny;
        const i64 rb = rv[j] ? ((i64)z * a.ny + y) * a.nx : 0;
        base[j] = a.rev ? a.off + a.n - 1 - rb : a.off + rb;
    }
    double w[KB];
#pragma unroll
    for (int j = 0; j < KB; ++j) w[j] = 0.0;
    int cached = 0;
    const int S = a.nx + (GROUPS - 1) + (KB - 1);
    const int src_self = active ? gbase : 0;
    const int src_below = active && gi > 0 ? gbase - 5 : 0;
    for (int s = 0; s < S; ++s) {
        const int tnow = s + tbase;
        if (has_prod && tnow + BIAS > cached) {
            if (!wait_producers(a.flags, pr, tnow + BIAS, &cached, a.status, a.spin_ns)) return;
        }
        double nv[KB];
#pragma unroll
        for (int j = KB - 1; j >= 0; --j) {
            // neighbour 5-vectors: own point at x-1, row y-1 at x, plane z-1 at x
            double vx[5], vy[5], vz[5];
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                vx[c] = __shfl_sync(FULL, w[j], src_self + c);
                vy[c] = __shfl_sync(FULL, w[j], src_below + c);
                vz[c] = (j > 0) ? __shfl_sync(FULL, w[j > 0 ? j - 1 : 0], src_self + c) : 0.0;
            }
            const int x = s - gi - j;
            const bool in = rv[j] && x >= 0 && x < a.nx;
            nv[j] = 0.0;
            if (!in) continue;
            const i64 p = base[j] + dir * x;
            if (gi == 0 || j == 0) {
                if (!(gi == 0 && j == 0)) nv[j] = __ldcg(a.out + p * 5 + ci);
            } else {
                const double* C = a.coup + p * 75 + ci * 5;
                double acc = a.rhs[p * 5 + ci];
#pragma unroll
                for (int c = 0; c < 5; ++c) acc = fma(-C[c], vx[c], acc);
#pragma unroll
                for (int c = 0; c < 5; ++c) acc = fma(-C[25 + c], vy[c], acc);
#pragma unroll
                for (int c = 0; c < 5; ++c) acc = fma(-C[50 + c], vz[c], acc);
                a.out[p * 5 + ci] = acc;
                if (a.u) a.u[p * 5 + ci] = fma(a.cu, acc, a.u[p * 5 + ci]);
                nv[j] = acc;
            }
        }
#pragma unroll
        for (int j = 0; j < KB; ++j) w[j] = nv[j];
        if ((s + 1) % a.publish_every == 0) publish(a.flags + t, tnow + BIAS);
    }
    publish(a.flags + t, DONE);
}

__global__ void __launch_bounds__(32) block_wave_kernel(BlockWaveArgs a) {
    run_units(a.n_units, a.flags, a.ctrl, a.status, [&](int t) { unit_block(a, t); });
}

unsigned nblk(i64 n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t block_create(BlockOp* b, const m2s_grid_desc* descs, int n_problems,
                         const std::vector<std::vector<Dims>>& dims, cudaStream_t st,
                         BlockAlloc alloc) {
    b->np = n_problems;
    b->dims.resize(n_problems);
    b->npts = 0;
    for (int i = 0; i < n_problems; ++i) {
        b->dims[i] = dims[i][0];
        b->npts += b->dims[i].n;
    }
    const size_t n = (size_t)std::max<i64>(b->npts, 1);
    cudaError_t e;
    if ((e = alloc((void**)&b->D, n * 25 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->L, n * 75 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->U, n * 75 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->Dinv, n * 25 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->M, n * 75 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->N, n * 75 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->s, n * 5 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->v, n * 5 * 8)) != cudaSuccess) return e;
    if ((e = alloc((void**)&b->w, n * 5 * 8)) != cudaSuccess) return e;
    for (int i = 0; i < n_problems; ++i) {
        const Dims& d = b->dims[i];
        if ((e = cudaMemcpyAsync(b->D + d.off * 25, descs[i].D, d.n * 25 * 8,
                                 cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpyAsync(b->L + d.off * 75, descs[i].L, d.n * 75 * 8,
                                 cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpyAsync(b->U + d.off * 75, descs[i].U, d.n * 75 * 8,
                                 cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
    }
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_wave_kernel, 32, 0)) !=
        cudaSuccess)
        return e;
    b->units.resize(n_problems);
    for (int i = 0; i < n_problems; ++i)
        if ((e = build_units(GROUPS - 1, 0, 0, KB, b->dims[i], per_sm, &b->units[i])) != cudaSuccess)
            return e;
    b->omega = -1.0;
    return cudaSuccess;
}

void block_free_units(BlockOp* b) {
    for (auto& u : b->units) free_wave_units(&u);
    b->units.clear();
}

cudaError_t block_apply(BlockOp* b, const double* u, double* y, cudaStream_t st) {
    for (int i = 0; i < b->np; ++i) {
        const Dims& d = b->dims[i];
        if (d.n == 0) continue;
        block_apply_kernel<false><<<nblk(d.n, 128), 128, 0, st>>>(d, b->D, b->L, b->U, nullptr,
                                                                  nullptr, u, y);
    }
    return cudaGetLastError();
}

cudaError_t block_ssor_iter(BlockOp* b, const double* rhs, double* u, double omega,
                            DevStatus* status, long long spin_ns, cudaStream_t st) {
    cudaError_t e;
    if (omega != b->omega) {
        for (int i = 0; i < b->np; ++i) {
            const Dims& d = b->dims[i];
            if (d.n == 0) continue;
            block_setup_kernel<<<nblk(d.n, 64), 64, 0, st>>>(d, b->D, b->L, b->U, omega, b->Dinv,
                                                             b->M, b->N);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        b->omega = omega;
    }
    const double cu = omega * (2.0 - omega);
    for (int i = 0; i < b->np; ++i) {
        const Dims& d = b->dims[i];
        if (d.n == 0) continue;
        block_apply_kernel<true><<<nblk(d.n, 128), 128, 0, st>>>(d, b->D, b->L, b->U, b->Dinv,
                                                                 rhs, u, b->s);
        const WaveUnits& un = b->units[i];
        BlockWaveArgs a;
        a.nx = d.nx;
        a.ny = d.ny;
        a.nz = d.nz;
        a.n = d.n;
        a.off = d.off;
        a.publish_every = 4;
        a.spin_ns = spin_ns;
        a.origin = un.d_origin;
        a.prod = un.d_prod;
        a.n_units = un.n_units;
        a.flags = un.d_flags;
        a.ctrl = un.d_ctrl;
        a.status = status;
        // lower sweep: v = s - M v (increasing p)
        a.rev = 0;
        a.coup = b->M;
        a.rhs = b->s;
        a.out = b->v;
        a.u = nullptr;
        a.cu = 0.0;
        block_wave_kernel<<<un.grid, 32, 0, st>>>(a);
        // upper sweep: w = v - N w (decreasing p), u += w(2-w) w
        a.rev = 1;
        a.coup = b->N;
        a.rhs = b->v;
        a.out = b->w;
        a.u = u;
        a.cu = cu;
        block_wave_kernel<<<un.grid, 32, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace m2s
