/*
 * m2s.h -- C ABI of the GB300 (sm_103a) library for the matrix-free
 * structured-grid solver hot path studied in Mat2Stencil (arXiv 2204.13304).
 *
 * Problem statement (paper Sec. 1 and Sec. 2.1): solve A u = b on a regular
 * Cartesian grid where A is a structured sparse operator that is never
 * assembled (matrix-free, Sec. 2.1.2); the routines are the SpMV, Gauss-Seidel
 * / SSOR sweeps with spatial dependence, geometric-multigrid restriction and
 * prolongation, and the MG-preconditioned CG that HPCG runs (Sec. 4.3,
 * Sec. 7.1).
 *
 * Conventions shared by every entry point
 *   Layout     vectors are dense [nz][ny][nx] arrays (x fastest); the block
 *              operator's vectors are [nz][ny][nx][5].  The flat index of
 *              point (x,y,z) is p = (z*ny + y)*nx + x.  "Lexicographic order"
 *              is increasing p.
 *   Memory     every vector pointer is a DEVICE pointer owned by the caller,
 *              8-byte aligned (FP64) or 4-byte aligned (FP32); vectors of one
 *              call must not overlap unless stated.  Coefficients passed to
 *              m2s_grid_create are copied; the grid owns all workspaces.
 *   Batches    a grid may hold n_problems problems; vectors are then the
 *              problems' arrays packed back to back in problem order.
 *   Streams    `stream` is a cudaStream_t (NULL = legacy default stream).
 *              Every call is stream-ordered and asynchronous unless stated.
 *   Levels     level 0 is the finest grid; level l has extents
 *              ceil(n_{l-1} / 2) (coarse point i <-> fine point 2i).
 *   dtype      M2S_F64 or M2S_F32: the element type of the vector pointers
 *              of the call.  FP32 calls need a grid created with
 *              precond_dtype = M2S_F32 for the kappa operator (the 27-point
 *              operator has no coefficients and accepts both).
 *   Errors     functions return an m2s_status; nothing traps or aborts.
 *              Invalid arguments are rejected before any launch.  A kernel
 *              error word (for example an expired bounded spin-wait) is read
 *              at the next synchronising call (m2s_pcg_solve,
 *              m2s_adjoint_solve, m2s_grid_sync) and returned there.
 */
#ifndef M2S_H
#define M2S_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct m2s_grid m2s_grid; /* opaque, library-owned */

typedef enum {
    M2S_OK = 0,
    M2S_ERR_INVALID_ARG = 1,
    M2S_ERR_CUDA = 2,
    M2S_ERR_OOM = 3,
    M2S_ERR_TIMEOUT = 4,       /* a bounded spin-wait expired in a sweep */
    M2S_ERR_NOT_CONVERGED = 5, /* max_iters reached above rtol */
    M2S_ERR_BREAKDOWN = 6      /* NaN/Inf or p.Ap <= 0 in CG */
} m2s_status;

typedef enum {
    M2S_OP_HPCG27 = 0,      /* 27-point: a_pp = 26, a_pq = -1 (HPCG) */
    M2S_OP_DIFF7_KAPPA = 1, /* 7-point variable-coefficient diffusion */
    M2S_OP_BLOCK7_5x5 = 2,  /* 7-point 5x5-block operator (NPB-LU shape) */
    M2S_OP_BLOCK7_JAC = 3   /* the same, blocks formed from the state u */
} m2s_op;

typedef enum { M2S_F64 = 0, M2S_F32 = 1 } m2s_dtype;

typedef enum { M2S_FORWARD = 0, M2S_BACKWARD = 1 } m2s_direction;

/* One problem of a grid.
 *   nx, ny, nz     extents, each >= 1.
 *   op             operator family.
 *   mg_levels      1..8 multigrid levels (1 = symmetric GS preconditioner).
 *   precond_dtype  M2S_F32 selects the FP32 V-cycle inside m2s_pcg_solve
 *                  (flexible CG; residual, dots and x stay FP64).
 *   kappa          op = DIFF7_KAPPA: device FP64 [nz][ny][nx] cell
 *                  coefficients (> 0), copied at creation.  The face
 *                  coefficient is the mean of its two cells (the averaging
 *                  matrix of paper Sec. 4.1); a boundary face uses the
 *                  cell's own value with a zero ghost value.
 *   D, L, U        op = BLOCK7_5x5: device FP64 per-point 5x5 row-major
 *                  blocks: D[n][5][5] diagonal blocks, L[n][3][5][5]
 *                  couplings to p-e_x, p-e_y, p-e_z, U[n][3][5][5] to
 *                  p+e_x, p+e_y, p+e_z (ignored where they leave the grid);
 *                  copied at creation.
 *   jac            op = BLOCK7_JAC: HOST FP64 array of 222 parameters,
 *                  copied at creation: sigma, nu, then for k = 0..3 (point
 *                  term, x, y, z) C_k (5x5 row-major), E_k (5x5), g_k (5).
 *                  The blocks are NPB-LU-style Jacobians (the SSOR of
 *                  paper Sec. 1 on the 5-vectors and 5x5 blocks of Sec.
 *                  4.2.3; NPB's own flux is not in the paper) of the synthetic
 *                  flux F_k(q) = C_k q + (g_k . q) E_k q evaluated at the
 *                  state, J_k(q) = C_k + (g_k . q) E_k + (E_k q) g_k^T:
 *                    D_p     = sigma I + J_0(u_p)
 *                    L_{p,d} = -nu I - J_{d+1}(u_{p-e_d}) / 2
 *                    U_{p,d} = -nu I + J_{d+1}(u_{p+e_d}) / 2
 *                  (couplings that leave the grid dropped).  They are
 *                  formed again from u at every use and never stored.  The
 *                  5x5 eliminations do not pivot: the caller keeps every
 *                  block row diagonally dominant along the iteration. */
typedef struct {
    int nx, ny, nz;
    m2s_op op;
    int mg_levels;
    m2s_dtype precond_dtype;
    const double* kappa;
    const double* D;
    const double* L;
    const double* U;
    const double* jac;
} m2s_grid_desc;

/* PCG options.  max_iters >= 1; rtol >= 0 (stop when |r|/|b| <= rtol);
 * fixed_iters = 1 runs exactly max_iters iterations (HPCG's 50-iteration
 * run) and never reports NOT_CONVERGED; check_every >= 1 is how often the
 * residual is copied to the host to test rtol (1 = every iteration). */
typedef struct {
    int max_iters;
    double rtol;
    int fixed_iters;
    int check_every;
} m2s_pcg_opts;

/* Filled after the stream synchronisation of a solve (host memory). */
typedef struct {
    int iters;              /* iterations performed */
    double rel_resid;       /* |r| / |b| after the last iteration (FP64) */
    double resid_hist_last; /* |r| after the last iteration */
} m2s_pcg_result;

/* Create a grid of n_problems problems (n_problems >= 1; every desc must
 * use the same op).  The grid is the problem statement of paper Sec. 2.1
 * (a linear system A u = b on a regular Cartesian grid, the operator never
 * assembled: Sec. 2.1.2) with the operator given as a row function over a
 * multi-dimensional domain (Sec. 4.2, Sec. 4.2.1; 5-vector unknowns and
 * 5x5 blocks as inner values, Sec. 4.2.3), and the multigrid hierarchy of
 * the HPCG solver of Sec. 7.1 (coarse domains derived from the fine one,
 * Sec. 4.2.2).  Allocates the multigrid hierarchy, coefficient copies,
 * the FP64 sweep workspaces and schedules, and the FP32 copies of the
 * variable-kappa operator when requested; copies coefficients with
 * stream-ordered copies on `stream` and synchronises it before returning.
 * The Krylov vectors are allocated by the first m2s_pcg_solve or
 * m2s_adjoint_solve, the 27-point operator's FP32 hierarchy by its first
 * FP32 call (or PCG with precond_dtype = F32); those calls can therefore
 * return M2S_ERR_OOM, after which the grid stays usable.  A grid that only
 * runs FP64 sweeps holds three level-sized FP64 arrays per level plus its
 * mailboxes (~1/10 of a level).  On failure *out is NULL and nothing is
 * leaked. */
m2s_status m2s_grid_create(const m2s_grid_desc* descs, int n_problems,
                           void* stream, m2s_grid** out);

/* Release the grid (synchronises the device first).  NULL is accepted. */
m2s_status m2s_grid_destroy(m2s_grid* grid);

/* Synchronise the grid's last stream and return (then clear) any kernel
 * error word, e.g. M2S_ERR_TIMEOUT from an expired spin-wait. */
m2s_status m2s_grid_sync(m2s_grid* grid, void* stream);

/* Number of points of level `level` of problem `problem` (0 if invalid). */
long long m2s_grid_points(const m2s_grid* grid, int problem, int level);

/* Sec. 4.3.1 SpMV on level `level`: y = A_level x (all problems of the
 * grid).  x and y must not overlap.  Op HPCG27 or DIFF7_KAPPA; for the
 * block operators level 0, FP64, [n][5] vectors: y = A x (BLOCK7_5x5) or
 * y = A(x) x with the blocks formed from x itself (BLOCK7_JAC). */
m2s_status m2s_spmv(m2s_grid* grid, int level, m2s_dtype dtype,
                    const void* x, void* y, void* stream);

/* Sec. 4.3.3 symmetric Gauss-Seidel on level `level`: n_sym_sweeps times
 * (one forward lexicographic sweep, then one backward sweep) of
 * x_p <- (b_p - sum_{q != p} a_pq x_q) / a_pp, in exact sequential order
 * (each point sees the new values of the points before it and the old
 * values of the points after it).  x is in/out; b and x must not overlap. */
m2s_status m2s_symgs(m2s_grid* grid, int level, m2s_dtype dtype,
                     const void* b, void* x, int n_sym_sweeps, void* stream);

/* One Gauss-Seidel sweep in one direction (forward = increasing p,
 * backward = decreasing p); the transpose of a forward sweep is a backward
 * sweep with the transposed couplings, which for these symmetric operators
 * are the same couplings. */
m2s_status m2s_gs_sweep(m2s_grid* grid, int level, m2s_dtype dtype,
                        const void* b, void* x, m2s_direction direction,
                        void* stream);

/* Multigrid transfer (paper Table 1 "HPCG Prolong" matrix: coarse point i
 * <-> fine point 2i).  Restriction of the residual:
 *   rc_i = r_{2i} - (A_level z)_{2i}, rc on level+1.
 * Prolongation (the transpose of injection): z_{2i} += zc_i. */
m2s_status m2s_mg_restrict(m2s_grid* grid, int level, m2s_dtype dtype,
                           const void* r, const void* z, void* rc, void* stream);
m2s_status m2s_mg_prolong(m2s_grid* grid, int level, m2s_dtype dtype,
                          const void* zc, void* z, void* stream);

/* One multigrid V-cycle z = M^-1 r (the multigrid preconditioner of the
 * HPCG solver, paper Sec. 7.1; its transfers are the "HPCG Prolong" row
 * function of Sec. 4.2 Table 1 and its transpose, fused into the
 * neighbouring sweeps as the strided loop fusion of Sec. 6.2.2 allows)
 * with the grid's mg_levels levels: z = 0;
 * coarsest level one symmetric GS; otherwise symmetric GS (pre-smoothing),
 * restrict the residual, recurse, prolongate, symmetric GS (post). dtype
 * F64 runs the FP64 hierarchy, F32 the FP32 one.  r and z must not
 * overlap. */
m2s_status m2s_mg_vcycle(m2s_grid* grid, m2s_dtype dtype, const void* r,
                         void* z, void* stream);

/* Preconditioned CG (the MG-preconditioned conjugate gradient that HPCG
 * runs, paper Sec. 7.1, 50 iterations per HPCG run; its vector updates are
 * the pointwise operations inlined into neighbouring loops in Sec. 6.2.1)
 * from x0 = 0 (r0 = b) with the V-cycle preconditioner
 * (FP64, or FP32 inside flexible CG when precond_dtype = F32).  b, x are
 * FP64.  Synchronises `stream`; fills *out (may be NULL).  Returns
 * M2S_ERR_NOT_CONVERGED if rtol was not met within max_iters (unless
 * fixed_iters), M2S_ERR_BREAKDOWN on p.Ap <= 0 or non-finite values. */
m2s_status m2s_pcg_solve(m2s_grid* grid, const double* b, double* x,
                         const m2s_pcg_opts* opts, m2s_pcg_result* out,
                         void* stream);

/* ILU(0) of the finest level's HPCG 27-point matrix (op HPCG27), the
 * incomplete-LU preconditioner of paper Sec. 1 on the 27-point stencil of
 * its ILU micro-benchmark (Sec. 7.2.1): factors L (unit lower) and U on the
 * pattern of A, every problem of the grid.  m2s_ilu0_setup computes them
 * (27 FP64 values per point, allocated by the first call, library-owned)
 * in lexicographic elimination order, ordered on `stream`.  May return
 * M2S_ERR_OOM. */
m2s_status m2s_ilu0_setup(m2s_grid* grid, void* stream);

/* Copy the factors of m2s_ilu0_setup to `out` (device, FP64,
 * [n][27] per point of the packed finest level: offset o = (dz+1)*9 +
 * (dy+1)*3 + (dx+1) of the 3x3x3 box; o < 13 L, o = 13 the pivot, o > 13
 * U; 0 off the domain), ordered on `stream`. */
m2s_status m2s_ilu0_factors(m2s_grid* grid, double* out, void* stream);

/* z = (L U)^{-1} r with the factors of m2s_ilu0_setup: forward substitution
 * with L, then backward substitution with U (packed FP64 finest-level
 * vectors of all problems).  r and z are either the same array or do not
 * overlap.  Each substitution is one persistent wavefront launch over all
 * problems (the dependence of the lexicographic Gauss-Seidel sweep),
 * ordered on `stream`; its spin-waits are bounded by the grid's spin limit
 * and an expired wait is reported as M2S_ERR_TIMEOUT by the next
 * synchronising call.  M2S_ERR_INVALID_ARG before m2s_ilu0_setup or for
 * another operator. */
m2s_status m2s_ilu0_apply(m2s_grid* grid, const double* r, double* z,
                          void* stream);

/* Direct solves of pentadiagonal systems along the grid lines of one axis:
 * the multi-diagonal direct solves of NPB-SP (paper Sec. 1; Sec. 7.2.2:
 * along each axis every line is swept forward and backward, the two
 * sweeps fused per line).  Grid nx, ny, nz, point p = (z*ny + y)*nx + x;
 * axis 0 = lines along x, 1 = along y, 2 = along z.  Point p at position
 * i of its line holds the equation
 *     a v[i-2] + b v[i-1] + c v[i] + d v[i+1] + e v[i+2] = r[i]
 * with coef[5p .. 5p+4] = (a, b, c, d, e) (device, FP64, [n][5]); terms
 * outside the line are ignored.  rhs (device, FP64, [n][k], 1 <= k <= 8)
 * holds k right-hand sides per point and is overwritten with the
 * solutions.  work: caller-owned device scratch of at least
 * m2s_line_penta_work_bytes(nx, ny, nz) bytes (3 FP64 values per point);
 * its contents on return are unspecified.  coef, rhs and work must be
 * 8-byte aligned and must not overlap.  No allocation, no host
 * synchronisation: the solve is ordered on `stream`.  Elimination without
 * pivoting: the caller supplies systems with nonzero pivots (e.g. strictly
 * diagonally dominant); a zero pivot makes that line's solutions
 * non-finite (not reported).  Errors: M2S_ERR_INVALID_ARG for bad sizes,
 * axis, k, NULL, misaligned or overlapping pointers or a short work
 * buffer; M2S_ERR_CUDA if the launch fails. */
long long m2s_line_penta_work_bytes(int nx, int ny, int nz);
m2s_status m2s_line_penta(int nx, int ny, int nz, int axis, const double* coef,
                          double* rhs, int k, void* work, long long work_bytes,
                          void* stream);

/* Direct solves of 5x5 block-tridiagonal systems along the grid lines of
 * one axis: the multi-diagonal direct solves of NPB-BT (paper Sec. 1, Sec.
 * 7.2.2).  Point p at position i of its line holds
 *     A v[i-1] + B v[i] + C v[i+1] = r[i]
 * with blk[75p .. 75p+74] = (A, B, C), each 5x5 row-major (entry (r, c)
 * at r*5 + c) (device, FP64, [n][3][5][5]); A of the first and C of the
 * last point of a line are ignored.  rhs (device, FP64, [n][5]) is
 * overwritten with v.  work: caller-owned device scratch of at least
 * m2s_line_btri_work_bytes(nx, ny, nz) bytes (25 FP64 values per point;
 * contents on return unspecified).  Block elimination without pivoting:
 * the caller supplies systems whose pivots are nonzero (e.g. strictly
 * block diagonally dominant); otherwise that line's solutions are
 * non-finite (not reported).  Axis, layout, alignment, no-overlap,
 * stream-ordering and error rules as m2s_line_penta; at most 2^32
 * points. */
long long m2s_line_btri_work_bytes(int nx, int ny, int nz);
m2s_status m2s_line_btri(int nx, int ny, int nz, int axis, const double* blk,
                         double* rhs, void* work, long long work_bytes,
                         void* stream);

/* Range-check record of the library variant built with -DM2S_DEBUG_BOUNDS
 * (the build's "bounds" variant): there, the block, ILU(0) and line-solve
 * kernels test every global index derived from a neighbour, a line, a
 * hyperplane or a scatter target against the extent it must stay in, skip a
 * violating access and count it (no trap, no fault).  Fills out[0..3] (host
 * memory): the number of violations since the last read, the source line
 * and index of the first, and its translation unit (0 block, 1 ILU, 2 line
 * solves); -1 where none.  Clears the record.  In the normal build out[0] =
 * -1 (checks not compiled in) and no CUDA call is made.  Call it after the
 * stream that ran the kernels has been synchronised. */
m2s_status m2s_debug_bounds_read(long long* out);

/* Block SSOR on the BLOCK7_5x5 operator (NPB-LU shape, paper Sec. 1 and
 * Sec. 4.3.3): n_iters times
 *   r = b - A u; lower sweep (D + omega L) v = r; upper sweep
 *   (D + omega U) w = D v; u += omega (2 - omega) w,
 * i.e. one forward and one backward block-SOR sweep per iteration.
 * On the BLOCK7_JAC operator every iteration first forms its blocks from
 * the u it starts from (A = A(u), the NPB-LU step with Jacobians formed
 * every step): one pass over the points forms each Jacobian once, a second
 * assembles the residual; no block is kept after the iteration.
 * 0 < omega < 2.  u is in/out ([n][5] FP64). */
m2s_status m2s_ssor_sweep(m2s_grid* grid, const double* b, double* u,
                          double omega, int n_iters, void* stream);

/* Adjoint of the kappa solve (op DIFF7_KAPPA).  The paper states no
 * adjoint: this is the implicit (solve-level) adjoint of the solve of A u = b
 * (Sec. 2.1) for the variable-coefficient diffusion operator whose face
 * coefficient averages its two cells (the averaging matrix of Sec. 4.1),
 * run with the transposed Gauss-Seidel sweeps of Sec. 4.3.3 (a transposed
 * forward sweep is a backward sweep with transposed couplings) inside the
 * same MG-PCG (Sec. 7.1).  Given the forward solution u
 * of A(kappa) u = b and dLdu, solves A^T lambda = dLdu with PCG (the
 * transposed V-cycle: transposed sweeps in mirrored order, which for this
 * symmetric operator is the same V-cycle) and writes
 *   dLdkappa_c = - sum_{faces f of c} dk_f/dk_c (lambda_p - lambda_q)
 *                (u_p - u_q) - (boundary faces of c) lambda_c u_c.
 * All vectors FP64.  Synchronises; fills *out (may be NULL). */
m2s_status m2s_adjoint_solve(m2s_grid* grid, const double* u,
                             const double* dLdu, double* lambda,
                             double* dLdkappa, const m2s_pcg_opts* opts,
                             m2s_pcg_result* out, void* stream);

/* dLdkappa from u and lambda alone (the stencil step of m2s_adjoint_solve). */
m2s_status m2s_kappa_grad(m2s_grid* grid, const double* u,
                          const double* lambda, double* dLdkappa,
                          void* stream);

/* Bound on every spin-wait of the dependent sweeps, in nanoseconds
 * (default 4e9).  A wait that exceeds it sets M2S_ERR_TIMEOUT, every sweep
 * in flight stops at its next wait, and the error is returned at the next
 * synchronising call. */
m2s_status m2s_set_spin_limit(m2s_grid* grid, long long limit_ns);

/* Symmetric Gauss-Seidel on the 27-point (HPCG) operator of an
 * nx x ny x nz grid that allocates no device memory: n_sym_sweeps times one
 * forward and one backward lexicographic sweep, exactly as m2s_symgs on a
 * grid of that operator.  (The paper has no counterpart: this entry point
 * exists for callers that cannot allocate -- applications that reserve all
 * device memory for their own pool, or latency-critical loops that cannot
 * afford cudaMalloc's implicit synchronisation.)
 *   b, x     device [nz][ny][nx] vectors of type dtype (x in/out); b and x
 *            must not share any byte (M2S_ERR_INVALID_ARG otherwise).
 *   limits   nx*ny*nz <= 262144 (64^3) points, at most 8192 wavefront
 *            units (so at most 32768 planes of z); larger requests return
 *            M2S_ERR_INVALID_ARG before any launch.
 *   scratch  one fixed-size array (about 4.4 MB) in the library's static
 *            device memory, shared by every call on every stream; the
 *            counters that must start at zero are cleared by each call.
 *            Calls that overlap on the GPU race on it: serialise them.
 *   set-up   the first call on a device looks up the array's device address
 *            (cudaGetSymbolAddress, that device current); make that first
 *            call before any stream capture.
 *   sync     every call copies its unit tables from host memory,
 *            synchronises `stream` before returning and reports an expired
 *            spin-wait as M2S_ERR_TIMEOUT.
 *   waits    every spin-wait is bounded by a fixed 4 s; m2s_set_spin_limit
 *            (a per-grid setting) does not apply to this entry point. */
m2s_status m2s_symgs_noalloc(int nx, int ny, int nz, m2s_dtype dtype,
                             const void* b, void* x, int n_sym_sweeps,
                             void* stream);

/* Shape of the 27-point sweep units (performance tuning; the paper's
 * task partitioning is fixed at compile time and has no counterpart): each
 * unit of the wavefront is one thread block of `warps` warps (4 or 8), one
 * grid plane per warp.  level = -1 sets every level.  The result of a sweep
 * does not depend on the shape; the b.x partials of the V-cycle's last
 * sweep are summed in a different order, so PCG iterates may differ in the
 * last bits.  Synchronises the device and reallocates the schedules: do not
 * call it while work of this grid is in flight or during stream capture.
 * Errors: M2S_ERR_INVALID_ARG (not a 27-point grid, level or warps out of
 * range), M2S_ERR_CUDA / M2S_ERR_OOM from the reallocation. */
m2s_status m2s_set_sweep_warps(m2s_grid* grid, int level, int warps);

/* Warps per unit (the unit height in planes) of the 27-point sweeps of one
 * level, FP64 in *warps_f64 and FP32 in *warps_f32 (host ints): the value
 * m2s_set_sweep_warps or m2s_autotune_sweeps set last, else the default
 * chosen with the schedule.  The default is 8 for FP32; for FP64 it is 4
 * while the wavefront of 4-warp units keeps at most 1.5 times the device's
 * SM count of units busy at once (the most units, over all problems of the
 * level, whose runs of nx + 65 steps, from step 60 U + 8 V of unit (U, V),
 * overlap), else 8: a lone warp per sub-partition steps faster, two finish
 * twice the points per SM.
 * Errors: M2S_ERR_INVALID_ARG (NULL grid or output, not a 27-point grid,
 * level out of range). */
m2s_status m2s_sweep_warps(m2s_grid* grid, int level, int* warps_f64, int* warps_f32);

/* Autotuner of the 27-point sweep units (form 2: tile shapes chosen by
 * measurement; the paper's partitioning has no counterpart).  For every
 * level and both dtypes it times `reps` forward sweeps with each unit shape
 * m2s_set_sweep_warps allows (4 and 8 warps) on the grid's own scratch
 * vectors and keeps the faster one.  chosen (host, optional, 2 * mg_levels
 * ints) receives the warps per unit of each level, FP64 then FP32.  It
 * synchronises the stream and reallocates the schedules: do not call it
 * while work of this grid is in flight or during stream capture.  The
 * result of a sweep does not depend on the shape.  Errors:
 * M2S_ERR_INVALID_ARG (NULL grid, not a 27-point grid, reps < 1),
 * M2S_ERR_CUDA, M2S_ERR_OOM, M2S_ERR_TIMEOUT. */
m2s_status m2s_autotune_sweeps(m2s_grid* grid, int reps, void* stream, int* chosen);

/* CUDA-graph replay of the PCG iteration (default on).  From the second
 * iteration on, m2s_pcg_solve records one iteration of each parity (the
 * search-direction buffers alternate) into a CUDA graph on the caller's
 * stream and replays it, so an iteration costs one graph launch instead of
 * one launch per kernel.  The graphs are kept for the solution pointer of
 * the solve that captured them and rebuilt when it changes; they are not
 * used while per-launch sweep timing is on.  Results are identical with and
 * without graphs (the same kernels run in the same order).  enable = 0
 * releases the graphs and launches every kernel.  Errors:
 * M2S_ERR_INVALID_ARG for a NULL grid. */
m2s_status m2s_set_graphs(m2s_grid* grid, int enable);

/* Per-launch timing of the Gauss-Seidel sweeps (instrumentation; the
 * paper has no counterpart).  enable = 1 clears the counters and, from the
 * next sweep on, brackets every sweep kernel the grid launches (any entry
 * point, any level, either dtype) with a pair of CUDA events recorded on the
 * stream the sweep is launched on; enable = 0 stops recording.  At most
 * 16384 launches per level are recorded, later ones are counted as dropped.
 * Events are created by the library (no device memory is allocated).
 * m2s_sweep_timing_read waits for the recorded events and returns, for
 * `level`, the number of recorded launches, their summed device time in
 * milliseconds and the number of dropped launches (any output may be NULL).
 * Errors: M2S_ERR_INVALID_ARG for a NULL grid or a level out of range,
 * M2S_ERR_CUDA if an event cannot be created or read. */
m2s_status m2s_sweep_timing(m2s_grid* grid, int enable);
m2s_status m2s_sweep_timing_read(m2s_grid* grid, int level, int* launches,
                                 double* total_ms, int* dropped);

/* Fault-injection hook for tests (host side; nothing faults on the GPU):
 * in the next Gauss-Seidel sweep on `level` (level = -1: in the forward
 * substitution of the next m2s_ilu0_apply of this 27-point grid), wavefront
 * unit `unit` (in ticket order) neither computes nor publishes its progress.  The units that wait
 * on it run into their bounded spin-wait, every sweep unit stops, and the
 * next synchronising call returns M2S_ERR_TIMEOUT; the sweep machinery is
 * reset and usable afterwards.  The sweep's output is then undefined. */
m2s_status m2s_debug_stall_unit(m2s_grid* grid, int level, int unit);

/* Static description of a status code. */
const char* m2s_status_string(m2s_status status);

#ifdef __cplusplus
}
#endif

#endif /* M2S_H */
