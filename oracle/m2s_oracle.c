/*
 * m2s_oracle.c -- serial CPU oracle for the matrix-free structured-grid
 * solver hot path of Mat2Stencil (arXiv 2204.13304).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  It shares no code, header,
 * table or helper with the CUDA library, and neither side includes the other.
 *
 * Every routine is the plain definition of the step, written as serial loops
 * over the grid in lexicographic order, in IEEE double precision (the FP32
 * preconditioner routines, suffix _f32, are the same loops in float because
 * that form fixes FP32 by definition).  Build with -ffp-contract=off so that
 * no a*b+c is fused behind our back (results are then identical on x86-64 and
 * aarch64).
 *
 * Conventions
 *   grid      nx, ny, nz points; point (x, y, z) has flat index
 *             p = (z*ny + y)*nx + x  (x fastest, z outermost).
 *   order     "lexicographic" = increasing p, i.e. z outermost, then y, then
 *             x -- the dictionary order of the domain loops (Sec. 4.3, the
 *             SymGS routine's loops; Sec. 6.1.1 "lexicographical execution
 *             order" within each thread).
 *   boundary  neighbours outside [0,nx)x[0,ny)x[0,nz) are dropped (zero
 *             Dirichlet), as in the HPCG operator.
 *   kinds     M2SO_HPCG27 = 0 : a_pp = 26, a_pq = -1 for every in-domain
 *                               neighbour of the 3x3x3 box (HPCG's operator).
 *             M2SO_KAPPA7 = 1 : variable-coefficient 7-point diffusion,
 *                               (A u)_p = sum_faces k_f (u_p - u_q), with the
 *                               face coefficient the average of the two cell
 *                               values (the averaging matrix A = [1/2 1/2] of
 *                               Sec. 4.1); at a boundary face k_f = k_p and
 *                               u_q = 0.
 * Citations name the paper's section / equation / definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long long i64;

#define M2SO_HPCG27 0
#define M2SO_KAPPA7 1

static i64 pidx(int nx, int ny, int x, int y, int z) {
    return ((i64)z * ny + y) * nx + x;
}
static int inside(int nx, int ny, int nz, int x, int y, int z) {
    return x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
}

/* ------------------------------------------------------------------------ */
/* Row functions (Sec. 4.2: a sparse matrix is a function from a row index  */
/* to its list of (column, value) non-zeros).  Non-zeros come out in        */
/* increasing column order; the diagonal is included.                      */
/* ------------------------------------------------------------------------ */

/* HPCG 27-point row: 26 on the diagonal, -1 for each in-domain neighbour. */
static int row_hpcg27(int nx, int ny, int nz, int x, int y, int z,
                      i64* col, double* val) {
    int c = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int qx = x + dx, qy = y + dy, qz = z + dz;
                if (!inside(nx, ny, nz, qx, qy, qz)) continue;
                col[c] = pidx(nx, ny, qx, qy, qz);
                val[c] = (dx == 0 && dy == 0 && dz == 0) ? 26.0 : -1.0;
                ++c;
            }
    return c;
}

/* Face coefficient between cell p and its neighbour q (interior face):
 * the arithmetic mean (averaging matrix A of Sec. 4.1). */
static double face_kappa(double kp, double kq) { return 0.5 * (kp + kq); }

/* Variable-kappa 7-point row.  For each of the 6 faces of cell p:
 *   interior face to q:  diagonal += k_f, entry (p,q) = -k_f, k_f = (k_p+k_q)/2
 *   boundary face:       diagonal += k_p (the ghost value u_q is 0).
 * The diagonal accumulates its six face terms in the fixed face order
 * -z, -y, -x, +x, +y, +z. */
static int row_kappa7(int nx, int ny, int nz, const double* kappa,
                      int x, int y, int z, i64* col, double* val) {
    static const int off[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0},
                                  {1, 0, 0},  {0, 1, 0},  {0, 0, 1}};
    i64 p = pidx(nx, ny, x, y, z);
    double kp = kappa[p];
    double diag = 0.0;
    double offv[6];
    i64 offc[6];
    int has[6];
    for (int f = 0; f < 6; ++f) {
        int qx = x + off[f][0], qy = y + off[f][1], qz = z + off[f][2];
        if (inside(nx, ny, nz, qx, qy, qz)) {
            i64 q = pidx(nx, ny, qx, qy, qz);
            double kf = face_kappa(kp, kappa[q]);
            diag += kf;
            offv[f] = -kf;
            offc[f] = q;
            has[f] = 1;
        } else {
            diag += kp;
            has[f] = 0;
        }
    }
    int c = 0;
    for (int f = 0; f < 3; ++f)
        if (has[f]) { col[c] = offc[f]; val[c] = offv[f]; ++c; }
    col[c] = p; val[c] = diag; ++c;
    for (int f = 3; f < 6; ++f)
        if (has[f]) { col[c] = offc[f]; val[c] = offv[f]; ++c; }
    return c;
}

static int row_of(int kind, int nx, int ny, int nz, const double* kappa,
                  int x, int y, int z, i64* col, double* val) {
    if (kind == M2SO_HPCG27) return row_hpcg27(nx, ny, nz, x, y, z, col, val);
    return row_kappa7(nx, ny, nz, kappa, x, y, z, col, val);
}

/* ------------------------------------------------------------------------ */
/* SpMV (Sec. 4.3.1): y_p = sum over the non-zeros of row p of a_pq * x_q,  */
/* in the row's column order.                                              */
/* ------------------------------------------------------------------------ */
void or_apply(int kind, int nx, int ny, int nz, const double* kappa,
              const double* x, double* y) {
    i64 col[27];
    double val[27];
    for (int z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy)
            for (int xx = 0; xx < nx; ++xx) {
                int c = row_of(kind, nx, ny, nz, kappa, xx, yy, z, col, val);
                double s = 0.0;
                for (int k = 0; k < c; ++k) s += val[k] * x[col[k]];
                y[pidx(nx, ny, xx, yy, z)] = s;
            }
}

/* ------------------------------------------------------------------------ */
/* Gauss-Seidel sweeps (Sec. 4.3.3, the SymGS routine; the loop reads and   */
/* writes the same vector, so a point sees the new values of the points     */
/* visited before it and the old values of the others).                    */
/*   x_p <- (b_p - sum_{q != p} a_pq x_q) / a_pp                           */
/* forward  : p increasing (lexicographic)                                 */
/* backward : p decreasing                                                 */
/* ------------------------------------------------------------------------ */
static void gs_point(int kind, int nx, int ny, int nz, const double* kappa,
                     const double* b, double* x, int xx, int yy, int z) {
    i64 col[27];
    double val[27];
    i64 p = pidx(nx, ny, xx, yy, z);
    int c = row_of(kind, nx, ny, nz, kappa, xx, yy, z, col, val);
    double s = b[p], diag = 0.0;
    for (int k = 0; k < c; ++k) {
        if (col[k] == p) { diag = val[k]; continue; }
        s -= val[k] * x[col[k]];
    }
    x[p] = s / diag;
}

void or_gs_forward(int kind, int nx, int ny, int nz, const double* kappa,
                   const double* b, double* x) {
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int xx = 0; xx < nx; ++xx)
                gs_point(kind, nx, ny, nz, kappa, b, x, xx, y, z);
}

void or_gs_backward(int kind, int nx, int ny, int nz, const double* kappa,
                    const double* b, double* x) {
    for (int z = nz - 1; z >= 0; --z)
        for (int y = ny - 1; y >= 0; --y)
            for (int xx = nx - 1; xx >= 0; --xx)
                gs_point(kind, nx, ny, nz, kappa, b, x, xx, y, z);
}

/* One symmetric Gauss-Seidel = one forward sweep then one backward sweep. */
void or_symgs(int kind, int nx, int ny, int nz, const double* kappa,
              const double* b, double* x, int n_sym_sweeps) {
    for (int s = 0; s < n_sym_sweeps; ++s) {
        or_gs_forward(kind, nx, ny, nz, kappa, b, x);
        or_gs_backward(kind, nx, ny, nz, kappa, b, x);
    }
}

/* Negative control for the ordering tests (NOT the method): the same update
 * applied colour by colour, 8 colours given by the parities of (x, y, z),
 * colours visited in the order 0..7 and each colour's points in increasing p.
 * Its results differ from the lexicographic sweep, which is what the tests
 * use to show that a reordered sweep would be caught. */
void or_gs_multicolor_forward(int kind, int nx, int ny, int nz,
                              const double* kappa, const double* b, double* x) {
    for (int color = 0; color < 8; ++color)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx) {
                    int cc = (xx & 1) | ((y & 1) << 1) | ((z & 1) << 2);
                    if (cc != color) continue;
                    gs_point(kind, nx, ny, nz, kappa, b, x, xx, y, z);
                }
}

/* ------------------------------------------------------------------------ */
/* Geometric multigrid pieces (Sec. 4.2 "HPCG Prolong" matrix with its      */
/* periodic sparsity pattern: coarse point i <-> fine point 2i, coarsening  */
/* by two per dimension; restriction is its transpose).                    */
/* ------------------------------------------------------------------------ */

/* coarse extent of a fine extent n: the fine points 0, 2, 4, ... */
int or_coarse_n(int n) { return (n + 1) / 2; }

/* rc_i = r_{2i} - (A z)_{2i}: residual of the fine level injected at the
 * even fine points. */
void or_restrict_residual(int kind, int nx, int ny, int nz, const double* kappa,
                          const double* r, const double* z, double* rc) {
    i64 n = (i64)nx * ny * nz;
    double* az = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    or_apply(kind, nx, ny, nz, kappa, z, az);
    int cx = or_coarse_n(nx), cy = or_coarse_n(ny), cz = or_coarse_n(nz);
    for (int k = 0; k < cz; ++k)
        for (int j = 0; j < cy; ++j)
            for (int i = 0; i < cx; ++i) {
                i64 f = pidx(nx, ny, 2 * i, 2 * j, 2 * k);
                rc[pidx(cx, cy, i, j, k)] = r[f] - az[f];
            }
    free(az);
}

/* z_{2i} += zc_i; the other fine points are unchanged (prolongation = the
 * transpose of injection). */
void or_prolong_add(int nx, int ny, int nz, const double* zc, double* z) {
    int cx = or_coarse_n(nx), cy = or_coarse_n(ny), cz = or_coarse_n(nz);
    for (int k = 0; k < cz; ++k)
        for (int j = 0; j < cy; ++j)
            for (int i = 0; i < cx; ++i)
                z[pidx(nx, ny, 2 * i, 2 * j, 2 * k)] += zc[pidx(cx, cy, i, j, k)];
}

/* Coarse kappa: mean of the fine cells {2i, 2i+1} x {2j, 2j+1} x {2k, 2k+1}
 * that lie inside the fine grid. */
void or_coarsen_kappa(int nx, int ny, int nz, const double* kf, double* kc) {
    int cx = or_coarse_n(nx), cy = or_coarse_n(ny), cz = or_coarse_n(nz);
    for (int k = 0; k < cz; ++k)
        for (int j = 0; j < cy; ++j)
            for (int i = 0; i < cx; ++i) {
                double s = 0.0;
                int cnt = 0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            int x = 2 * i + dx, y = 2 * j + dy, z = 2 * k + dz;
                            if (!inside(nx, ny, nz, x, y, z)) continue;
                            s += kf[pidx(nx, ny, x, y, z)];
                            ++cnt;
                        }
                kc[pidx(cx, cy, i, j, k)] = s / (double)cnt;
            }
}

/* V-cycle MG(l, r) -> z  (levels = total number of levels, >= 1):
 *   z = 0
 *   coarsest level: one symmetric Gauss-Seidel of A_l z = r
 *   otherwise:      symmetric GS (pre-smoothing); rc = R (r - A_l z);
 *                   zc = MG(l+1, rc); z += P zc; symmetric GS (post).
 * The coarse operator is the same stencil rediscretised on the coarse grid
 * (27-point: same coefficients; kappa: the coarsened kappa). */
void or_mg_vcycle(int kind, int nx, int ny, int nz, const double* kappa,
                  int levels, const double* r, double* z) {
    i64 n = (i64)nx * ny * nz;
    for (i64 i = 0; i < n; ++i) z[i] = 0.0;
    if (levels <= 1) {
        or_symgs(kind, nx, ny, nz, kappa, r, z, 1);
        return;
    }
    or_symgs(kind, nx, ny, nz, kappa, r, z, 1);
    int cx = or_coarse_n(nx), cy = or_coarse_n(ny), cz = or_coarse_n(nz);
    i64 nc = (i64)cx * cy * cz;
    double* rc = (double*)malloc(sizeof(double) * (size_t)nc);
    double* zc = (double*)malloc(sizeof(double) * (size_t)nc);
    double* kc = NULL;
    if (kind == M2SO_KAPPA7) {
        kc = (double*)malloc(sizeof(double) * (size_t)nc);
        or_coarsen_kappa(nx, ny, nz, kappa, kc);
    }
    or_restrict_residual(kind, nx, ny, nz, kappa, r, z, rc);
    or_mg_vcycle(kind, cx, cy, cz, kc, levels - 1, rc, zc);
    or_prolong_add(nx, ny, nz, zc, z);
    or_symgs(kind, nx, ny, nz, kappa, r, z, 1);
    free(rc);
    free(zc);
    free(kc);
}

/* ------------------------------------------------------------------------ */
/* The same V-cycle entirely in FP32 (the FP32-preconditioner form).  The   */
/* FP32 kappa of every level is the FP32 rounding of the FP64 kappa of that */
/* level; face averages and all sums are then taken in float.              */
/* ------------------------------------------------------------------------ */
static int row_of_f32(int kind, int nx, int ny, int nz, const float* kappa,
                      int x, int y, int z, i64* col, float* val) {
    if (kind == M2SO_HPCG27) {
        int c = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int qx = x + dx, qy = y + dy, qz = z + dz;
                    if (!inside(nx, ny, nz, qx, qy, qz)) continue;
                    col[c] = pidx(nx, ny, qx, qy, qz);
                    val[c] = (dx == 0 && dy == 0 && dz == 0) ? 26.0f : -1.0f;
                    ++c;
                }
        return c;
    }
    static const int off[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0},
                                  {1, 0, 0},  {0, 1, 0},  {0, 0, 1}};
    i64 p = pidx(nx, ny, x, y, z);
    float kp = kappa[p], diag = 0.0f, offv[6];
    i64 offc[6];
    int has[6];
    for (int f = 0; f < 6; ++f) {
        int qx = x + off[f][0], qy = y + off[f][1], qz = z + off[f][2];
        if (inside(nx, ny, nz, qx, qy, qz)) {
            i64 q = pidx(nx, ny, qx, qy, qz);
            float kf = 0.5f * (kp + kappa[q]);
            diag += kf;
            offv[f] = -kf;
            offc[f] = q;
            has[f] = 1;
        } else {
            diag += kp;
            has[f] = 0;
        }
    }
    int c = 0;
    for (int f = 0; f < 3; ++f)
        if (has[f]) { col[c] = offc[f]; val[c] = offv[f]; ++c; }
    col[c] = p; val[c] = diag; ++c;
    for (int f = 3; f < 6; ++f)
        if (has[f]) { col[c] = offc[f]; val[c] = offv[f]; ++c; }
    return c;
}

void or_apply_f32(int kind, int nx, int ny, int nz, const float* kappa,
                  const float* x, float* y) {
    i64 col[27];
    float val[27];
    for (int z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy)
            for (int xx = 0; xx < nx; ++xx) {
                int c = row_of_f32(kind, nx, ny, nz, kappa, xx, yy, z, col, val);
                float s = 0.0f;
                for (int k = 0; k < c; ++k) s += val[k] * x[col[k]];
                y[pidx(nx, ny, xx, yy, z)] = s;
            }
}

static void gs_point_f32(int kind, int nx, int ny, int nz, const float* kappa,
                         const float* b, float* x, int xx, int yy, int z) {
    i64 col[27];
    float val[27];
    i64 p = pidx(nx, ny, xx, yy, z);
    int c = row_of_f32(kind, nx, ny, nz, kappa, xx, yy, z, col, val);
    float s = b[p], diag = 0.0f;
    for (int k = 0; k < c; ++k) {
        if (col[k] == p) { diag = val[k]; continue; }
        s -= val[k] * x[col[k]];
    }
    x[p] = s / diag;
}

void or_symgs_f32(int kind, int nx, int ny, int nz, const float* kappa,
                  const float* b, float* x, int n_sym_sweeps) {
    for (int s = 0; s < n_sym_sweeps; ++s) {
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int xx = 0; xx < nx; ++xx)
                    gs_point_f32(kind, nx, ny, nz, kappa, b, x, xx, y, z);
        for (int z = nz - 1; z >= 0; --z)
            for (int y = ny - 1; y >= 0; --y)
                for (int xx = nx - 1; xx >= 0; --xx)
                    gs_point_f32(kind, nx, ny, nz, kappa, b, x, xx, y, z);
    }
}

/* kappa64 is the FP64 kappa of this level; the FP32 copy is derived here. */
static void mg_vcycle_f32_rec(int kind, int nx, int ny, int nz,
                              const double* kappa64, int levels,
                              const float* r, float* z) {
    i64 n = (i64)nx * ny * nz;
    float* k32 = NULL;
    if (kind == M2SO_KAPPA7) {
        k32 = (float*)malloc(sizeof(float) * (size_t)n);
        for (i64 i = 0; i < n; ++i) k32[i] = (float)kappa64[i];
    }
    for (i64 i = 0; i < n; ++i) z[i] = 0.0f;
    or_symgs_f32(kind, nx, ny, nz, k32, r, z, 1);
    if (levels > 1) {
        int cx = or_coarse_n(nx), cy = or_coarse_n(ny), cz = or_coarse_n(nz);
        i64 nc = (i64)cx * cy * cz;
        float* az = (float*)malloc(sizeof(float) * (size_t)n);
        float* rc = (float*)malloc(sizeof(float) * (size_t)nc);
        float* zc = (float*)malloc(sizeof(float) * (size_t)nc);
        double* kc = NULL;
        if (kind == M2SO_KAPPA7) {
            kc = (double*)malloc(sizeof(double) * (size_t)nc);
            or_coarsen_kappa(nx, ny, nz, kappa64, kc);
        }
        or_apply_f32(kind, nx, ny, nz, k32, z, az);
        for (int k = 0; k < cz; ++k)
            for (int j = 0; j < cy; ++j)
                for (int i = 0; i < cx; ++i) {
                    i64 f = pidx(nx, ny, 2 * i, 2 * j, 2 * k);
                    rc[pidx(cx, cy, i, j, k)] = r[f] - az[f];
                }
        mg_vcycle_f32_rec(kind, cx, cy, cz, kc, levels - 1, rc, zc);
        for (int k = 0; k < cz; ++k)
            for (int j = 0; j < cy; ++j)
                for (int i = 0; i < cx; ++i)
                    z[pidx(nx, ny, 2 * i, 2 * j, 2 * k)] += zc[pidx(cx, cy, i, j, k)];
        or_symgs_f32(kind, nx, ny, nz, k32, r, z, 1);
        free(az);
        free(rc);
        free(zc);
        free(kc);
    }
    free(k32);
}

void or_mg_vcycle_f32(int kind, int nx, int ny, int nz, const double* kappa64,
                      int levels, const float* r, float* z) {
    mg_vcycle_f32_rec(kind, nx, ny, nz, kappa64, levels, r, z);
}

/* ------------------------------------------------------------------------ */
/* Compensated dot product Dot2 (Ogita, Rump & Oishi, "Accurate sum and dot */
/* product", SIAM J. Sci. Comput. 26(6), 2005, Alg. 5.3): the result is as */
/* accurate as if computed in twice the working precision and then rounded, */
/* so it does not depend on the summation order to within ~1 ulp.  It is an */
/* evaluation of the plain definition sum_i a_i b_i, not a different one.   */
/* ------------------------------------------------------------------------ */
static void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double z = x - a;
    *s = x;
    *e = (a - (x - z)) + (b - z);
}
static void two_prod(double a, double b, double* p, double* e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}
double or_dot(i64 n, const double* a, const double* b) {
    if (n <= 0) return 0.0;
    double p, s, h, r, q;
    two_prod(a[0], b[0], &p, &s);
    for (i64 i = 1; i < n; ++i) {
        two_prod(a[i], b[i], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
    }
    return p + s;
}

/* ------------------------------------------------------------------------ */
/* Preconditioned conjugate gradients, x0 = 0, r0 = b:                      */
/*   z = M^-1 r; rho = r.z; p = z (k = 1) or p = z + (rho/rho_old) p;       */
/*   q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q; |r|.         */
/* levels = 0: no preconditioner (M = I); levels >= 1: one V-cycle with    */
/* that many levels (levels = 1 is one symmetric GS from z = 0).           */
/* precond_f32 = 1: the FP32 V-cycle, z = double(V32(float(r))), inside     */
/* the flexible (Polak-Ribiere) variant                                    */
/*   beta = (r_k.z_k - r_k.z_{k-1}) / rho_{k-1}.                           */
/* The residual, the dot products and the update of x stay in FP64.        */
/* fixed_iters = 1 runs exactly max_iters iterations; otherwise it stops    */
/* when |r|/|b| <= rtol.  resid_hist[k] = |r_k| (k = 0..iters).             */
/* Returns 0 on success, 1 if not converged, 2 on breakdown (p.q <= 0 or a  */
/* non-finite value).                                                      */
/* ------------------------------------------------------------------------ */
int or_pcg(int kind, int nx, int ny, int nz, const double* kappa, int levels,
           int precond_f32, const double* b, double* x, int max_iters,
           double rtol, int fixed_iters, double* resid_hist, int* iters_out) {
    i64 n = (i64)nx * ny * nz;
    size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(bytes);
    double* z = (double*)malloc(bytes);
    double* zold = (double*)malloc(bytes);
    double* p = (double*)malloc(bytes);
    double* q = (double*)malloc(bytes);
    float* r32 = NULL;
    float* z32 = NULL;
    if (precond_f32) {
        r32 = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
        z32 = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    }
    for (i64 i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; zold[i] = 0.0; }
    double nb = sqrt(or_dot(n, b, b));
    double nr = nb;
    if (resid_hist) resid_hist[0] = nr;
    double rho_old = 0.0;
    int k = 0, status = 1;
    if (nb == 0.0) { status = 0; goto done; }
    for (k = 1; k <= max_iters; ++k) {
        if (levels <= 0) {
            for (i64 i = 0; i < n; ++i) z[i] = r[i];
        } else if (precond_f32) {
            for (i64 i = 0; i < n; ++i) r32[i] = (float)r[i];
            or_mg_vcycle_f32(kind, nx, ny, nz, kappa, levels, r32, z32);
            for (i64 i = 0; i < n; ++i) z[i] = (double)z32[i];
        } else {
            or_mg_vcycle(kind, nx, ny, nz, kappa, levels, r, z);
        }
        double rho = or_dot(n, r, z);
        if (k == 1) {
            for (i64 i = 0; i < n; ++i) p[i] = z[i];
        } else {
            double beta;
            if (precond_f32) beta = (rho - or_dot(n, r, zold)) / rho_old;
            else beta = rho / rho_old;
            for (i64 i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        or_apply(kind, nx, ny, nz, kappa, p, q);
        double pq = or_dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(rho)) { status = 2; break; }
        double alpha = rho / pq;
        for (i64 i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (i64 i = 0; i < n; ++i) r[i] -= alpha * q[i];
        nr = sqrt(or_dot(n, r, r));
        if (resid_hist) resid_hist[k] = nr;
        if (precond_f32) for (i64 i = 0; i < n; ++i) zold[i] = z[i];
        rho_old = rho;
        if (!isfinite(nr)) { status = 2; break; }
        if (!fixed_iters && nr <= rtol * nb) { status = 0; break; }
    }
    if (k > max_iters) {
        k = max_iters;
        status = (fixed_iters || nr <= rtol * nb) ? 0 : 1;
    }
done:
    if (iters_out) *iters_out = k;
    free(r); free(z); free(zold); free(p); free(q); free(r32); free(z32);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the variable-kappa solve.  With A(kappa) u = b and            */
/* L = 0.5 |u - u*|^2, the adjoint state is lambda = A^-T (u - u*) and      */
/*   dL/dkappa_c = - lambda^T (dA/dkappa_c) u.                              */
/* An interior face f between p and q with k_f = (k_p + k_q)/2 adds          */
/* k_f (u_p - u_q) to row p and k_f (u_q - u_p) to row q, so it contributes */
/* (1/2)(lambda_p - lambda_q)(u_p - u_q) for each of its two cells; a       */
/* boundary face of cell c adds k_c u_c to row c, contributing lambda_c u_c.*/
/* g_c = -[ sum_{interior faces of c} (1/2)(lambda_c - lambda_q)(u_c - u_q) */
/*          + (number of boundary faces of c) * lambda_c u_c ]             */
/* ------------------------------------------------------------------------ */
void or_kappa_grad(int nx, int ny, int nz, const double* u, const double* lam,
                   double* g) {
    static const int off[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0},
                                  {1, 0, 0},  {0, 1, 0},  {0, 0, 1}};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                i64 c = pidx(nx, ny, x, y, z);
                double s = 0.0;
                for (int f = 0; f < 6; ++f) {
                    int qx = x + off[f][0], qy = y + off[f][1], qz = z + off[f][2];
                    if (inside(nx, ny, nz, qx, qy, qz)) {
                        i64 q = pidx(nx, ny, qx, qy, qz);
                        s += 0.5 * (lam[c] - lam[q]) * (u[c] - u[q]);
                    } else {
                        s += lam[c] * u[c];
                    }
                }
                g[c] = -s;
            }
}

/* ------------------------------------------------------------------------ */
/* Block (5x5) SSOR in the shape of NPB-LU (Sec. 4.2.3 inner values as      */
/* tensors: 5 unknowns per point; Sec. 1 / Sec. 4.3.3 name SSOR among the   */
/* routines).  Per point p, D[p] is a 5x5 block, L[p][d] and U[p][d]        */
/* (d = 0,1,2 for x,y,z) couple p to p - e_d and p + e_d.  Blocks are        */
/* row-major; couplings that leave the domain are dropped.                 */
/*   A u:   (A u)_p = D_p u_p + sum_d L_{p,d} u_{p-e_d} + U_{p,d} u_{p+e_d}  */
/*   SSOR step (Saad, Iterative Methods, Sec. 4.1.2; M = (D+wL) D^-1        */
/*   (D+wU) / (w(2-w)) ):                                                  */
/*     r = b - A u                                                         */
/*     lower, p increasing:  v_p = D_p^-1 (r_p - w sum_d L_{p,d} v_{p-e_d})  */
/*     upper, p decreasing:  w_p = v_p - w D_p^-1 sum_d U_{p,d} w_{p+e_d}    */
/*     u += w(2-w) w                                                       */
/* This is exactly one forward block-SOR sweep followed by one backward     */
/* block-SOR sweep on u (the tests check that identity).                   */
/* 5x5 solves: Gaussian elimination without pivoting, natural order.       */
/* ------------------------------------------------------------------------ */
static void solve5(const double* Dm, const double* rhs, double* out) {
    double a[5][5], t[5];
    for (int i = 0; i < 5; ++i) {
        for (int j = 0; j < 5; ++j) a[i][j] = Dm[i * 5 + j];
        t[i] = rhs[i];
    }
    for (int k = 0; k < 5; ++k)
        for (int i = k + 1; i < 5; ++i) {
            double m = a[i][k] / a[k][k];
            for (int j = k; j < 5; ++j) a[i][j] -= m * a[k][j];
            t[i] -= m * t[k];
        }
    for (int i = 4; i >= 0; --i) {
        double s = t[i];
        for (int j = i + 1; j < 5; ++j) s -= a[i][j] * out[j];
        out[i] = s / a[i][i];
    }
}

static void matvec5_acc(const double* M, const double* v, double* acc) {
    for (int i = 0; i < 5; ++i) {
        double s = 0.0;
        for (int j = 0; j < 5; ++j) s += M[i * 5 + j] * v[j];
        acc[i] += s;
    }
}

/* A u for the block operator, blocks taken in increasing column order
 * (z-1, y-1, x-1, p, x+1, y+1, z+1). */
void or_block_apply(int nx, int ny, int nz, const double* D, const double* L,
                    const double* U, const double* u, double* y) {
    for (int z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy)
            for (int x = 0; x < nx; ++x) {
                i64 p = pidx(nx, ny, x, yy, z);
                double acc[5] = {0, 0, 0, 0, 0};
                if (z > 0) matvec5_acc(L + (p * 3 + 2) * 25, u + pidx(nx, ny, x, yy, z - 1) * 5, acc);
                if (yy > 0) matvec5_acc(L + (p * 3 + 1) * 25, u + pidx(nx, ny, x, yy - 1, z) * 5, acc);
                if (x > 0) matvec5_acc(L + (p * 3 + 0) * 25, u + pidx(nx, ny, x - 1, yy, z) * 5, acc);
                matvec5_acc(D + p * 25, u + p * 5, acc);
                if (x < nx - 1) matvec5_acc(U + (p * 3 + 0) * 25, u + pidx(nx, ny, x + 1, yy, z) * 5, acc);
                if (yy < ny - 1) matvec5_acc(U + (p * 3 + 1) * 25, u + pidx(nx, ny, x, yy + 1, z) * 5, acc);
                if (z < nz - 1) matvec5_acc(U + (p * 3 + 2) * 25, u + pidx(nx, ny, x, yy, z + 1) * 5, acc);
                for (int i = 0; i < 5; ++i) y[p * 5 + i] = acc[i];
            }
}

void or_block_residual(int nx, int ny, int nz, const double* D, const double* L,
                       const double* U, const double* b, const double* u,
                       double* r) {
    i64 n5 = (i64)nx * ny * nz * 5;
    double* au = (double*)malloc(sizeof(double) * (size_t)(n5 > 0 ? n5 : 1));
    or_block_apply(nx, ny, nz, D, L, U, u, au);
    for (i64 i = 0; i < n5; ++i) r[i] = b[i] - au[i];
    free(au);
}

void or_block_lower(int nx, int ny, int nz, const double* D, const double* L,
                    double omega, const double* r, double* v) {
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                i64 p = pidx(nx, ny, x, y, z);
                double acc[5] = {0, 0, 0, 0, 0}, t[5];
                if (x > 0) matvec5_acc(L + (p * 3 + 0) * 25, v + pidx(nx, ny, x - 1, y, z) * 5, acc);
                if (y > 0) matvec5_acc(L + (p * 3 + 1) * 25, v + pidx(nx, ny, x, y - 1, z) * 5, acc);
                if (z > 0) matvec5_acc(L + (p * 3 + 2) * 25, v + pidx(nx, ny, x, y, z - 1) * 5, acc);
                for (int i = 0; i < 5; ++i) t[i] = r[p * 5 + i] - omega * acc[i];
                solve5(D + p * 25, t, v + p * 5);
            }
}

void or_block_upper(int nx, int ny, int nz, const double* D, const double* U,
                    double omega, const double* v, double* w) {
    for (int z = nz - 1; z >= 0; --z)
        for (int y = ny - 1; y >= 0; --y)
            for (int x = nx - 1; x >= 0; --x) {
                i64 p = pidx(nx, ny, x, y, z);
                double acc[5] = {0, 0, 0, 0, 0}, t[5];
                if (x < nx - 1) matvec5_acc(U + (p * 3 + 0) * 25, w + pidx(nx, ny, x + 1, y, z) * 5, acc);
                if (y < ny - 1) matvec5_acc(U + (p * 3 + 1) * 25, w + pidx(nx, ny, x, y + 1, z) * 5, acc);
                if (z < nz - 1) matvec5_acc(U + (p * 3 + 2) * 25, w + pidx(nx, ny, x, y, z + 1) * 5, acc);
                solve5(D + p * 25, acc, t);
                for (int i = 0; i < 5; ++i) w[p * 5 + i] = v[p * 5 + i] - omega * t[i];
            }
}

/* n_iters SSOR steps on u (in place). */
void or_ssor(int nx, int ny, int nz, const double* D, const double* L,
             const double* U, double omega, const double* b, double* u,
             int n_iters) {
    i64 n5 = (i64)nx * ny * nz * 5;
    size_t bytes = sizeof(double) * (size_t)(n5 > 0 ? n5 : 1);
    double* r = (double*)malloc(bytes);
    double* v = (double*)malloc(bytes);
    double* w = (double*)malloc(bytes);
    double scale = omega * (2.0 - omega);
    for (int it = 0; it < n_iters; ++it) {
        or_block_residual(nx, ny, nz, D, L, U, b, u, r);
        or_block_lower(nx, ny, nz, D, L, omega, r, v);
        or_block_upper(nx, ny, nz, D, U, omega, v, w);
        for (i64 i = 0; i < n5; ++i) u[i] += scale * w[i];
    }
    free(r); free(v); free(w);
}

/* ------------------------------------------------------------------------ */
/* Blocks formed from the state (the NPB-LU situation of Sec. 1 and Sec.    */
/* 4.2.3: the 5x5 blocks of the SSOR step are Jacobians evaluated at the    */
/* current u, formed again every step instead of stored).  NPB's own flux   */
/* formulas are not part of the paper, so the flux here is a synthetic      */
/* quadratic one with the same data dependence: each block is a nonlinear   */
/* function of ONE point's 5-vector.                                        */
/*                                                                          */
/* Parameters P, 2 + 4 * 55 doubles: sigma = P[0], nu = P[1]; for           */
/* k = 0..3 at P + 2 + 55 k: C_k (5x5 row-major), E_k (5x5), g_k (5).       */
/* k = 0 is the point term, k = 1, 2, 3 the x, y, z directions.             */
/*   flux      F_k(q) = C_k q + (g_k . q) E_k q                             */
/*   Jacobian  J_k(q) = C_k + (g_k . q) E_k + (E_k q) g_k^T                 */
/*   D_p       = sigma I + J_0(u_p)                                         */
/*   L_{p,d}   = -nu I - J_{d+1}(u_{p-e_d}) / 2   (p - e_d in the domain)   */
/*   U_{p,d}   = -nu I + J_{d+1}(u_{p+e_d}) / 2   (p + e_d in the domain)   */
/* i.e. a central difference of the flux plus a diffusion of weight nu;     */
/* couplings that leave the domain are 0.                                   */
/* ------------------------------------------------------------------------ */
static void jac_block(const double* Pk, const double* q, double* J) {
    const double* C = Pk;
    const double* E = Pk + 25;
    const double* g = Pk + 50;
    double gq = 0.0, Eq[5];
    for (int j = 0; j < 5; ++j) gq += g[j] * q[j];
    for (int i = 0; i < 5; ++i) {
        Eq[i] = 0.0;
        for (int j = 0; j < 5; ++j) Eq[i] += E[i * 5 + j] * q[j];
    }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) J[i * 5 + j] = C[i * 5 + j] + gq * E[i * 5 + j] + Eq[i] * g[j];
}

void or_block_jac(int nx, int ny, int nz, const double* P, const double* u,
                  double* D, double* L, double* U) {
    const double sigma = P[0], nu = P[1];
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                i64 p = pidx(nx, ny, x, y, z);
                double J[25];
                jac_block(P + 2, u + p * 5, J);
                for (int i = 0; i < 25; ++i) D[p * 25 + i] = J[i] + (i % 6 == 0 ? sigma : 0.0);
                for (int d = 0; d < 3; ++d) {
                    const int c[3] = {x, y, z};
                    const int ext[3] = {nx, ny, nz};
                    int lo[3] = {x, y, z}, hi[3] = {x, y, z};
                    lo[d] -= 1;
                    hi[d] += 1;
                    double* Lb = L + (p * 3 + d) * 25;
                    double* Ub = U + (p * 3 + d) * 25;
                    if (c[d] > 0) {
                        jac_block(P + 2 + 55 * (d + 1), u + pidx(nx, ny, lo[0], lo[1], lo[2]) * 5, J);
                        for (int i = 0; i < 25; ++i) Lb[i] = -0.5 * J[i] - (i % 6 == 0 ? nu : 0.0);
                    } else {
                        for (int i = 0; i < 25; ++i) Lb[i] = 0.0;
                    }
                    if (c[d] < ext[d] - 1) {
                        jac_block(P + 2 + 55 * (d + 1), u + pidx(nx, ny, hi[0], hi[1], hi[2]) * 5, J);
                        for (int i = 0; i < 25; ++i) Ub[i] = 0.5 * J[i] - (i % 6 == 0 ? nu : 0.0);
                    } else {
                        for (int i = 0; i < 25; ++i) Ub[i] = 0.0;
                    }
                }
            }
}

/* n_iters SSOR steps on u (in place), each with the blocks formed from the
 * u it starts from: u <- u + w(2-w) M(u)^-1 (b - A(u) u). */
void or_ssor_jac(int nx, int ny, int nz, const double* P, double omega,
                 const double* b, double* u, int n_iters) {
    i64 n = (i64)nx * ny * nz;
    size_t m = (size_t)(n > 0 ? n : 1);
    double* D = (double*)malloc(sizeof(double) * m * 25);
    double* L = (double*)malloc(sizeof(double) * m * 75);
    double* U = (double*)malloc(sizeof(double) * m * 75);
    for (int it = 0; it < n_iters; ++it) {
        or_block_jac(nx, ny, nz, P, u, D, L, U);
        or_ssor(nx, ny, nz, D, L, U, omega, b, u, 1);
    }
    free(D); free(L); free(U);
}

/* Version tag so the tests can check which oracle build is loaded. */
/* ------------------------------------------------------------------------ */
/* Direct solves of multi-diagonal systems along grid lines (the "direct    */
/* solving of multi-diagonal matrices" of NPB-SP, Sec. 1 and Sec. 7.2.2:    */
/* along each axis in turn, every line is swept forward and backward).      */
/* Point p at position i of its line carries the equation                   */
/*   a v_{i-2} + b v_{i-1} + c v_i + d v_{i+1} + e v_{i+2} = r_i,           */
/* coef[p][0..4] = (a, b, c, d, e); terms outside the line are dropped.     */
/* rhs[p][0..k-1] holds k right-hand sides and is overwritten with the      */
/* solutions.  The oracle is Gaussian elimination without pivoting on the   */
/* band of each line, in the textbook order: for every pivot row i,        */
/* subtract multiples of it from rows i+1 and i+2, then back-substitute.   */
/* ------------------------------------------------------------------------ */
void or_line_penta(int nx, int ny, int nz, int axis, const double* coef,
                   double* rhs, int k) {
    const int ext[3] = {nx, ny, nz};
    const i64 stride[3] = {1, nx, (i64)nx * ny};
    const int m = ext[axis];
    /* the two coordinates across the lines */
    const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
    double* A = (double*)malloc(sizeof(double) * 5 * (size_t)(m > 0 ? m : 1));
    double* R = (double*)malloc(sizeof(double) * (size_t)k * (size_t)(m > 0 ? m : 1));
    for (int c2 = 0; c2 < ext[o2]; ++c2)
        for (int c1 = 0; c1 < ext[o1]; ++c1) {
            const i64 base = (i64)c1 * stride[o1] + (i64)c2 * stride[o2];
            /* gather the band: A[i][j] multiplies v_{i+j-2} */
            for (int i = 0; i < m; ++i) {
                const i64 p = base + (i64)i * stride[axis];
                for (int j = 0; j < 5; ++j) {
                    const int col = i + j - 2;
                    A[5 * i + j] = (col >= 0 && col < m) ? coef[5 * p + j] : 0.0;
                }
                for (int t = 0; t < k; ++t) R[(size_t)k * i + t] = rhs[(i64)k * p + t];
            }
            /* elimination below each pivot */
            for (int i = 0; i < m; ++i) {
                for (int r = i + 1; r <= i + 2 && r < m; ++r) {
                    const int j = i - r + 2; /* column i in row r's band */
                    const double f = A[5 * r + j] / A[5 * i + 2];
                    for (int t = 0; t < 3 && j + t < 5; ++t)
                        A[5 * r + j + t] -= f * A[5 * i + 2 + t];
                    for (int t = 0; t < k; ++t) R[(size_t)k * r + t] -= f * R[(size_t)k * i + t];
                }
            }
            /* back substitution */
            for (int i = m - 1; i >= 0; --i)
                for (int t = 0; t < k; ++t) {
                    double s = R[(size_t)k * i + t];
                    if (i + 1 < m) s -= A[5 * i + 3] * R[(size_t)k * (i + 1) + t];
                    if (i + 2 < m) s -= A[5 * i + 4] * R[(size_t)k * (i + 2) + t];
                    R[(size_t)k * i + t] = s / A[5 * i + 2];
                }
            for (int i = 0; i < m; ++i) {
                const i64 p = base + (i64)i * stride[axis];
                for (int t = 0; t < k; ++t) rhs[(i64)k * p + t] = R[(size_t)k * i + t];
            }
        }
    free(A);
    free(R);
}

/* Block-tridiagonal systems along grid lines (NPB-BT's direct solves, the  */
/* 5x5-block counterpart of the above): point p at position i of its line  */
/* holds  A v_{i-1} + B v_i + C v_{i+1} = r_i  with 5x5 blocks             */
/* blk[p][0] = A, blk[p][1] = B, blk[p][2] = C (row-major, entry (r, c) at */
/* r*5 + c) and 5-vectors; A of the first and C of the last point of a     */
/* line are dropped.  rhs[p][0..4] is overwritten with v.  The oracle is    */
/* Gaussian elimination without pivoting on each line's dense 5m x 5m      */
/* matrix restricted to its band: every pivot column eliminates the rows   */
/* below it within the next block row, then back substitution.             */
void or_line_btri(int nx, int ny, int nz, int axis, const double* blk, double* rhs) {
    const int ext[3] = {nx, ny, nz};
    const i64 stride[3] = {1, nx, (i64)nx * ny};
    const int m = ext[axis];
    const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;
    const int N = 5 * m;
    /* band storage: row R holds columns R-9 .. R+9 (the widest a block row
       reaches), W[R][c - R + 9] */
    const int BW = 19;
    double* W = (double*)malloc(sizeof(double) * (size_t)BW * (size_t)(N > 0 ? N : 1));
    double* R = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int c2 = 0; c2 < ext[o2]; ++c2)
        for (int c1 = 0; c1 < ext[o1]; ++c1) {
            const i64 base = (i64)c1 * stride[o1] + (i64)c2 * stride[o2];
            memset(W, 0, sizeof(double) * (size_t)BW * (size_t)N);
            for (int i = 0; i < m; ++i) {
                const i64 p = base + (i64)i * stride[axis];
                for (int r = 0; r < 5; ++r) {
                    const int row = 5 * i + r;
                    for (int b = 0; b < 3; ++b) {
                        const int bi = i + b - 1; /* block column */
                        if (bi < 0 || bi >= m) continue;
                        for (int c = 0; c < 5; ++c)
                            W[(size_t)BW * row + (5 * bi + c) - row + 9] = blk[75 * p + 25 * b + 5 * r + c];
                    }
                    R[row] = rhs[5 * p + r];
                }
            }
            /* elimination: pivot column k clears rows k+1 .. min(k+9, N-1) */
            for (int k = 0; k < N; ++k) {
                const double piv = W[(size_t)BW * k + 9];
                for (int row = k + 1; row <= k + 9 && row < N; ++row) {
                    const double f = W[(size_t)BW * row + k - row + 9] / piv;
                    if (f == 0.0) continue;
                    for (int c = k; c <= k + 9 && c < N; ++c) {
                        const int jr = c - row + 9;
                        if (jr < 0 || jr >= BW) continue;
                        W[(size_t)BW * row + jr] -= f * W[(size_t)BW * k + c - k + 9];
                    }
                    R[row] -= f * R[k];
                }
            }
            for (int k = N - 1; k >= 0; --k) {
                double s = R[k];
                for (int c = k + 1; c <= k + 9 && c < N; ++c) s -= W[(size_t)BW * k + c - k + 9] * R[c];
                R[k] = s / W[(size_t)BW * k + 9];
            }
            for (int i = 0; i < m; ++i) {
                const i64 p = base + (i64)i * stride[axis];
                for (int r = 0; r < 5; ++r) rhs[5 * p + r] = R[5 * i + r];
            }
        }
    free(W);
    free(R);
}

/* ------------------------------------------------------------------------ */
/* ILU(0) of the HPCG 27-point matrix (the incomplete LU preconditioner of  */
/* Sec. 1 and the ILU micro-benchmark of Sec. 7.2.1, on the 27-point       */
/* stencil).  Factors on the matrix's own pattern: for every point p the   */
/* 27 values F[p][o], o = (dz+1)*9 + (dy+1)*3 + (dx+1) over the offsets of  */
/* the 3x3x3 box (o < 13: the strict lower part, L with a unit diagonal    */
/* implied; o = 13: the pivot u_pp; o > 13: the strict upper part of U);   */
/* entries of out-of-domain neighbours are 0.  Rows in lexicographic order,*/
/* each by the IKJ elimination restricted to the pattern (Saad, Iterative  */
/* Methods for Sparse Linear Systems, Sec. 10.3):                          */
/*   for k in pattern(p), k < p, increasing:  a_pk /= a_kk;                 */
/*     for j in pattern(p), j > k, j in pattern(k):  a_pj -= a_pk a_kj.     */
/* ------------------------------------------------------------------------ */
static int box_off(int dx, int dy, int dz) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

void or_ilu0_factor(int nx, int ny, int nz, double* F) {
    const i64 n = (i64)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const i64 p = pidx(nx, ny, x, y, z);
                double* Fp = F + 27 * p;
                /* the row of A on the pattern */
                for (int o = 0; o < 27; ++o) {
                    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                    Fp[o] = inside(nx, ny, nz, x + dx, y + dy, z + dz) ? (o == 13 ? 26.0 : -1.0) : 0.0;
                }
                /* eliminate the lower entries in increasing column order */
                for (int ok = 0; ok < 13; ++ok) {
                    const int kx = ok % 3 - 1, ky = (ok / 3) % 3 - 1, kz = ok / 9 - 1;
                    if (!inside(nx, ny, nz, x + kx, y + ky, z + kz)) continue;
                    const double* Fk = F + 27 * pidx(nx, ny, x + kx, y + ky, z + kz);
                    Fp[ok] /= Fk[13];
                    for (int oj = ok + 1; oj < 27; ++oj) {
                        const int jx = oj % 3 - 1, jy = (oj / 3) % 3 - 1, jz = oj / 9 - 1;
                        if (!inside(nx, ny, nz, x + jx, y + jy, z + jz)) continue;
                        /* column j relative to row k */
                        const int rx = jx - kx, ry = jy - ky, rz = jz - kz;
                        if (rx < -1 || rx > 1 || ry < -1 || ry > 1 || rz < -1 || rz > 1) continue;
                        Fp[oj] -= Fp[ok] * Fk[box_off(rx, ry, rz)];
                    }
                }
            }
    (void)n;
}

/* z = (LU)^{-1} r: forward substitution with the unit lower factor in     */
/* lexicographic order, then backward substitution with U in reverse.     */
void or_ilu0_apply(int nx, int ny, int nz, const double* F, const double* r, double* zout) {
    const i64 n = (i64)nx * ny * nz;
    double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy)
            for (int x = 0; x < nx; ++x) {
                const i64 p = pidx(nx, ny, x, yy, z);
                double s = r[p];
                for (int o = 0; o < 13; ++o) {
                    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                    if (inside(nx, ny, nz, x + dx, yy + dy, z + dz))
                        s -= F[27 * p + o] * y[pidx(nx, ny, x + dx, yy + dy, z + dz)];
                }
                y[p] = s;
            }
    for (int z = nz - 1; z >= 0; --z)
        for (int yy = ny - 1; yy >= 0; --yy)
            for (int x = nx - 1; x >= 0; --x) {
                const i64 p = pidx(nx, ny, x, yy, z);
                double s = y[p];
                for (int o = 14; o < 27; ++o) {
                    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
                    if (inside(nx, ny, nz, x + dx, yy + dy, z + dz))
                        s -= F[27 * p + o] * zout[pidx(nx, ny, x + dx, yy + dy, z + dz)];
                }
                zout[p] = s / F[27 * p + 13];
            }
    free(y);
}

int or_abi_version(void) { return 1; }
