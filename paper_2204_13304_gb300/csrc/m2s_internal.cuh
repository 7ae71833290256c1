// Internal declarations of the m2s CUDA library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "m2s.h"

namespace m2s {

typedef long long i64;

// Extents of one grid level of one problem and where its arrays start in the
// packed batch vectors.
struct Dims {
    int nx, ny, nz;
    i64 n;        // nx*ny*nz
    i64 off;      // element offset of this problem in packed vectors
};

// Device-side status words of a grid (one allocation).
struct DevStatus {
    int err;        // first error code raised by a kernel (0 = none)
    int abort;      // set together with err: every waiting unit stops
    int pad[14];
};

// ---------------------------------------------------------------------------
// Memory-model helpers (PTX ISA: release/acquire at gpu scope).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T> struct Lit;
template <> struct Lit<double> {
    static __device__ __forceinline__ double inv26() { return 1.0 / 26.0; }
};
template <> struct Lit<float> {
    static __device__ __forceinline__ float inv26() { return 1.0f / 26.0f; }
};

// ---------------------------------------------------------------------------
// Launchers (defined in the kernel translation units).
// ---------------------------------------------------------------------------

// 27-point stencil tile kernels (k_stencil27.cu).
enum St27Mode {
    ST27_SPMV = 0,        // y = A x
    ST27_PSPMV_DOT = 1,   // p = z + beta p (stored), q = A p, partial p.q
    ST27_QUP = 2,         // Q = b + sum of the 13 upper neighbours of x
    ST27_QLO = 3,         // Q = b + sum of the 13 lower neighbours of x
    ST27_PROLONG_QUP = 4  // Q = b + upper sums of (x + P xc)  (x not written)
};
template <typename T>
cudaError_t launch_st27(St27Mode mode, Dims d, Dims dc, const T* x, const T* xc, const T* b, T* y,
                        cudaStream_t st);
// The Q modes with Q written pre-scaled, Q/26 (the input of the CTA sweep
// kernel), and b/26 also written to bs when bs is not NULL.
template <typename T>
cudaError_t launch_st27_q26(St27Mode mode, Dims d, Dims dc, const T* x, const T* xc, const T* b,
                            T* Q, T* bs, cudaStream_t st);
// y = x / 26 (as x * fl(1/26)), n elements
template <typename T>
cudaError_t launch_scale26(i64 n, const T* x, T* y, cudaStream_t st);
// p.q partials the fused CG step writes for one problem (one per CTA).
int st27_num_partials(Dims d);

// TMA-staged forms (k_st27_tma.cu) for rows that are 16-byte aligned:
// st27_tma_shape_ok(d, sizeof(T)) tells whether d qualifies.
bool st27_tma_shape_ok(const Dims& d, size_t elem);
int st27_tma_pcg_partials(const Dims& d);
template <typename T>
cudaError_t launch_spmv27_tma(const Dims& d, const T* x, T* y, int* err, cudaStream_t st);
cudaError_t launch_pspmv_dot_tma(const Dims& d, const double* z, const double* pin, double* pout,
                                 double* q, const double* beta, double* partials, int* err,
                                 cudaStream_t st);
// y = A x of the 27-point operator on one problem's level: the TMA kernel
// where the shape and the vectors allow it, st27_kernel otherwise.  err is
// the grid's status word (an expired stage wait records M2S_ERR_TIMEOUT).
template <typename T>
cudaError_t launch_spmv27(Dims d, const T* x, T* y, int* err, cudaStream_t st);

// rc = injection of r - A z; rc/26 also written to rcs when rcs is not NULL
template <typename T>
cudaError_t launch_restrict27(Dims f, Dims c, const T* r, const T* z, T* rc, T* rcs,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_prolong(Dims f, Dims c, const T* zc, T* z, cudaStream_t st);

// Wavefront Gauss-Seidel (k_wave.cu).
struct WaveUnits {
    int n_units;      // units in ticket (topological) order
    int2* d_origin;   // (u0, v0) of each unit
    int4* d_prod;     // producer unit indices (left, below, below-left, -1)
    int* d_flags;     // progress word per unit (0 at rest)
    int* d_ctrl;      // [0] ticket, [1] exited CTAs, [2] launch tag (CTA kernel)
    unsigned long long* d_mbox = nullptr;  // CTA kernel: tagged boundary rows
    int grid;         // CTAs launched
    int K;            // slots per lane (incl. the halo slot)
    int stencil;      // 27 or 7
    int W = 1;        // CTA kernel: compute warps (planes) per unit
    int depth = 0;    // CTA kernel: prefetch depth (steps) of the launch
    // CTA kernels, all problems of a level in one launch: per unit (u0, v0,
    // problem, first b.x partial), per problem its dims and the prefix of
    // its b.x partials (np + 1 entries)
    int4* d_units = nullptr;
    Dims* d_dims = nullptr;
    int* d_rzpre = nullptr;
    int np = 0;
    int n_rz = 0;     // b.x partials of one launch (units x W)
    i64 mb_words = 0; // 27-point: words of the row mailbox (the plane-sum mailbox follows)
    long long* d_mboff = nullptr;  // 27-point: per problem its first mailbox values (2 each)
};
struct WaveCall {
    int rev;              // 0 forward, 1 backward (reflected index space)
    int publish_every;    // steps between progress publications
    long long spin_ns;    // bound of every spin-wait
    DevStatus* status;
    double* rz_partials;  // per unit b.x partials of the new x, or NULL
    int stall_unit;       // test hook: this unit neither computes nor
                          // publishes (-1 = none), so its consumers' bounded
                          // waits expire and the sweep reports a timeout
};
template <typename T>
cudaError_t launch_gs27_wave(const WaveUnits& u, const WaveCall& c, Dims d,
                             const T* Qin, T* Qout, const T* b, T* x,
                             cudaStream_t st);
// Face coefficients of the variable-kappa operator of one level: kf[d][p] is
// the coefficient of the face between p and p - e_d (0 on the boundary).
template <typename T>
struct KappaLevel {
    T* kf[3];  // kf[d][p]: face between p and p - e_d (0 on the boundary)
    T* kr[3];  // kr[d][p]: face between p and p + e_d (0 on the boundary)
    T* diag;
    T* invdiag;
    // the sweeps' coefficients packed per point, 4 values each: (kf x, y, z,
    // 1/a_pp) for the forward sweep, (kr x, y, z, 1/a_pp) for the backward
    T* pack[2];
};
// 7-point CTA wavefront sweep (k_wave7.cu): units of 31 rows x W planes.
template <typename T>
cudaError_t build_cta7_units(const std::vector<Dims>& dims, WaveUnits* out);
template <typename T>
cudaError_t launch_gs7_cta(const WaveUnits& u, const WaveCall& c, const KappaLevel<T>& k,
                           const T* Qin, T* Qout, const T* b, T* x, cudaStream_t st);

// Variable-kappa 7-point kernels (k_kappa7.cu).
cudaError_t launch_kappa_coarsen(Dims f, Dims c, const double* kf, double* kc,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_kappa_setup(Dims d, const double* kappa, KappaLevel<T> k,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_spmv7(Dims d, const KappaLevel<T>& k, const T* x, T* y,
                         cudaStream_t st);
// Q = b + sum over upper (up=1) or lower (up=0) faces of k_f x_q, with
// x = x + P xc when xc != NULL (prolongation fused; x is not written).
template <typename T>
cudaError_t launch_qinit7(Dims d, Dims dc, const KappaLevel<T>& k, int up,
                          const T* x, const T* xc, const T* b, T* Q,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_restrict7(Dims f, Dims c, const KappaLevel<T>& k,
                             const T* r, const T* z, T* rc, cudaStream_t st);
cudaError_t launch_kappa_grad(Dims d, const double* u, const double* lam,
                              double* g, cudaStream_t st);
cudaError_t build_units(int lanes, int skew, int corner, int K, Dims d, int per_sm,
                        WaveUnits* out);
void build_units_host(int lanes, int skew, int corner, int K, Dims d, std::vector<int2>& org,
                      std::vector<int4>& prod);
int wave_grid(int n_units, int per_sm);
int wave_blocks_per_sm(int stencil);
constexpr int kWaveSlots = 5;  // register slots per lane of the sweep kernels
// CTA-pipelined 27-point sweep (k_wave2.cu)
template <typename T>
cudaError_t build_cta_units(const std::vector<Dims>& dims, int warps, WaveUnits* out);
bool cta_warps_supported(int warps);
int cta_default_warps(int dtype_is_f64, const std::vector<Dims>& dims);
// b.x partials of the largest schedule of these problems
int cta_rz_partials_max(const std::vector<Dims>& dims);
// Qin and Qout hold Q/26; b is b/26 when Qout is written, b when the b.x
// partials are (c.rz_partials), and unused otherwise.
template <typename T>
cudaError_t launch_gs27_cta(const WaveUnits& u, const WaveCall& c, const T* Qin, T* Qout,
                            const T* b, T* x, cudaStream_t st);
void free_wave_units(WaveUnits* u);

// Pentadiagonal line solves (k_line.cu): FP64 values of the work array.
i64 line_penta_work_doubles(int nx, int ny, int nz);
cudaError_t launch_line_penta(int nx, int ny, int nz, int axis, const double* coef, double* rhs,
                              int k, double* work, cudaStream_t st);
// ILU(0) of the HPCG 27-point matrix (k_ilu.cu): factors F[n][27] over the
// 3x3x3 box offsets; one launch per hyperplane x + 2y + 4z.
int ilu_hyperplanes(const Dims& d);
// Finv[n]: the pivots' rounded reciprocals 1/F[p][13], written by the
// factorisation and used in place of divisions
cudaError_t launch_ilu_factor(const Dims& d, double* F, double* Finv, cudaStream_t st);
// Block-tridiagonal (5x5) line solves (k_line.cu).
i64 line_btri_work_doubles(int nx, int ny, int nz);

// range-check records of the instrumented translation units (see
// m2s_bounds.cuh): out[0] violations (-1: checks not compiled in), out[1]
// source line and out[2] index of the first; cleared by the read
cudaError_t bounds_read_block(long long* out);
cudaError_t bounds_read_ilu(long long* out);
// ILU(0) application as two CTA-wavefront launches (k_ilu_wave.cu): weight
// records Lw, Uw ([n][16] each, packed over problems) from F and Finv, and
// the sweep units of the problems (made at the first call).
cudaError_t ilu_wave_setup(const std::vector<Dims>& dims, i64 n, const double* F,
                           const double* Finv, double* Lw, double* Uw, WaveUnits* units,
                           cudaStream_t st);
// forward (rev 0: Wt = Lw, in = r, out = z) or backward (rev 1: Wt = Uw,
// in = out = z) substitution of all problems, one launch
// stall_unit >= 0: that unit (ticket order) neither computes nor publishes
// (host-side fault injection for tests; its consumers' waits expire)
cudaError_t launch_ilu_wave(const WaveUnits& u, int rev, long long spin_ns, DevStatus* status,
                            const double* Wt, const double* in, double* out, int stall_unit,
                            cudaStream_t st);
cudaError_t bounds_read_line(long long* out);
cudaError_t launch_line_btri(int nx, int ny, int nz, int axis, const double* blk, double* rhs,
                             double* work, cudaStream_t st);


}  // namespace m2s
