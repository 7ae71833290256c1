"""Pins for the CPU oracle: each oracle routine is checked against something
other than itself -- closed forms, invariants, special cases that reduce to a
textbook routine, and brute-force dense linear algebra on tiny grids.

Paper references: Sec. 4.3.1 (SpMV), Sec. 4.3.3 (SymGS and other routines
with spatial dependence), Sec. 4.2 (HPCG prolongation matrix), Sec. 4.1
(averaging matrix), Sec. 7.1 (HPCG, NPB-LU workloads).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import m2s_inputs as gen
import oracle

H27 = oracle.HPCG27
K7 = oracle.KAPPA7

SHAPES_TINY = [(3, 4, 5), (5, 3, 4), (4, 5, 3), (1, 3, 2), (2, 1, 1)]


def dense_from_apply(kind, shape, kappa=None):
    """Dense A assembled column by column from the oracle SpMV."""
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    e = np.zeros(shape)
    for j in range(n):
        e.flat[j] = 1.0
        A[:, j] = oracle.apply(kind, e, kappa).ravel()
        e.flat[j] = 0.0
    return A


def rnd(shape, k=0):
    return gen.random_vector(shape, seed=gen.BASE_SEED + 17 * k)


def kappa_small(shape, k=0):
    return np.exp(rnd(shape, 100 + k))


# --------------------------------------------------------------------------
# c2: 27-point operator
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", SHAPES_TINY + [(6, 6, 6)])
def test_hpcg27_row_sums_closed_form(shape):
    """(A 1)_p = 26 - #in-domain neighbours = 27 - prod_d (#valid offsets)."""
    nz, ny, nx = shape
    y = oracle.apply(H27, np.ones(shape))
    for z, yy, x in itertools.product(range(nz), range(ny), range(nx)):
        cnt = 1
        for c, n in ((x, nx), (yy, ny), (z, nz)):
            cnt *= sum(1 for d in (-1, 0, 1) if 0 <= c + d < n)
        assert y[z, yy, x] == 27 - cnt


def test_hpcg27_interior_corner_edge_face_values():
    y = oracle.apply(H27, np.ones((6, 6, 6)))
    assert y[3, 3, 3] == 0.0          # interior
    assert y[0, 0, 0] == 19.0         # corner: 7 neighbours
    assert y[0, 0, 3] == 15.0         # edge: 11 neighbours
    assert y[0, 3, 3] == 9.0          # face: 17 neighbours


@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 3, 4)])
def test_hpcg27_dense_structure(shape):
    """Dense A: 26 on the diagonal, -1 exactly at Chebyshev distance 1."""
    A = dense_from_apply(H27, shape)
    nz, ny, nx = shape
    coords = [(z, y, x) for z in range(nz) for y in range(ny) for x in range(nx)]
    for i, a in enumerate(coords):
        for j, b in enumerate(coords):
            d = max(abs(a[0] - b[0]), abs(a[1] - b[1]), abs(a[2] - b[2]))
            want = 26.0 if d == 0 else (-1.0 if d == 1 else 0.0)
            assert A[i, j] == want


def test_hpcg27_symmetric():
    shape = (7, 6, 5)
    x, y = rnd(shape, 1), rnd(shape, 2)
    a = oracle.dot(x, oracle.apply(H27, y))
    b = oracle.dot(y, oracle.apply(H27, x))
    assert abs(a - b) <= 1e-14 * max(abs(a), 1.0)


# --------------------------------------------------------------------------
# c8: variable-kappa 7-point operator
# --------------------------------------------------------------------------
def laplacian7_kron(shape):
    """Standard 7-point Dirichlet Laplacian as a Kronecker sum of 1-D
    tridiag(-1, 2, -1) matrices (independent construction)."""
    nz, ny, nx = shape

    def t(n):
        return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)

    Iz, Iy, Ix = np.eye(nz), np.eye(ny), np.eye(nx)
    return (np.kron(np.kron(t(nz), Iy), Ix) + np.kron(np.kron(Iz, t(ny)), Ix)
            + np.kron(np.kron(Iz, Iy), t(nx)))


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 3, 1)])
def test_kappa7_unit_kappa_is_laplacian(shape):
    A = dense_from_apply(K7, shape, np.ones(shape))
    assert np.array_equal(A, laplacian7_kron(shape))


@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 4, 4)])
def test_kappa7_row_sums_are_boundary_terms(shape):
    """A 1 = sum over the boundary faces of cell p of kappa_p."""
    kap = kappa_small(shape)
    y = oracle.apply(K7, np.ones(shape), kap)
    nz, ny, nx = shape
    for z, yy, x in itertools.product(range(nz), range(ny), range(nx)):
        nb = sum(1 for c, n in ((x, nx), (yy, ny), (z, nz)) for d in (-1, 1)
                 if not 0 <= c + d < n)
        assert abs(y[z, yy, x] - nb * kap[z, yy, x]) <= 1e-13 * (1 + abs(y[z, yy, x]))


def test_kappa7_symmetric_positive_definite():
    shape = (3, 4, 5)
    kap = kappa_small(shape, 3)
    A = dense_from_apply(K7, shape, kap)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    # off-diagonal (p, q) = -(k_p + k_q)/2 for face neighbours
    nz, ny, nx = shape
    p = (1 * ny + 2) * nx + 3
    q = (1 * ny + 2) * nx + 4
    assert A[p, q] == -0.5 * (kap.flat[p] + kap.flat[q])


# --------------------------------------------------------------------------
# c1 / c3: Gauss-Seidel sweeps: ordering, brute force, fixed point
# --------------------------------------------------------------------------
def dense_gs_forward(A, b, x0):
    """x1 = (D + L)^-1 (b - U x0) with L/U split by flattened index."""
    DL = np.tril(A)
    U = np.triu(A, 1)
    return np.linalg.solve(DL, b - U @ x0)


def dense_gs_backward(A, b, x0):
    DU = np.triu(A)
    L = np.tril(A, -1)
    return np.linalg.solve(DU, b - L @ x0)


@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 3, 4), (4, 5, 3)])
@pytest.mark.parametrize("kind", [H27, K7])
def test_gs_sweeps_match_dense_triangular_solves(kind, shape):
    kap = kappa_small(shape, 5) if kind == K7 else None
    A = dense_from_apply(kind, shape, kap)
    b, x0 = rnd(shape, 6), rnd(shape, 7)
    f = oracle.gs_forward(kind, b, x0, kap)
    fd = dense_gs_forward(A, b.ravel(), x0.ravel())
    assert np.max(np.abs(f.ravel() - fd)) <= 1e-13 * np.max(np.abs(fd))
    g = oracle.gs_backward(kind, b, f, kap)
    gd = dense_gs_backward(A, b.ravel(), fd)
    assert np.max(np.abs(g.ravel() - gd)) <= 1e-13 * np.max(np.abs(gd))
    s = oracle.symgs(kind, b, x0, 1, kap)
    assert np.array_equal(s, g)


def test_gs_axis_order_matters():
    """A transposed axis order would give a different sweep: the dense check
    above therefore pins x fastest, z outermost."""
    shape = (3, 4, 5)
    A = dense_from_apply(H27, shape)
    b, x0 = rnd(shape, 8), rnd(shape, 9)
    # the same sweep, but with the points visited with y fastest
    perm = np.arange(np.prod(shape)).reshape(shape).transpose(0, 2, 1).ravel()
    Ap = A[np.ix_(perm, perm)]
    wrong = np.empty(A.shape[0])
    wrong[perm] = dense_gs_forward(Ap, b.ravel()[perm], x0.ravel()[perm])
    f = oracle.gs_forward(H27, b, x0)
    assert np.max(np.abs(f.ravel() - wrong)) > 1e-3


@pytest.mark.parametrize("shape", [(8, 8, 8), (5, 7, 3)])
def test_symgs_bitwise_fixed_point(shape):
    """b = A 1, x = 1: every update is an exact integer sum / 26 = 1."""
    b = oracle.apply(H27, np.ones(shape))
    x = oracle.symgs(H27, b, np.ones(shape), 3)
    assert np.array_equal(x, np.ones(shape))


def test_symgs_error_a_norm_monotone():
    shape = (6, 5, 7)
    A = dense_from_apply(H27, shape)
    xs = rnd(shape, 10).ravel()
    b = (A @ xs).reshape(shape)
    x = np.zeros(shape)
    prev = np.inf
    for _ in range(6):
        x = oracle.symgs(H27, b, x, 1)
        e = x.ravel() - xs
        en = e @ A @ e
        assert en <= prev * (1 + 1e-12)
        prev = en


def test_negative_control_multicolor_differs():
    """A reordered (8-colour) sweep differs from the lexicographic one far
    above the 1e-13 parity tolerance after 10 sweeps."""
    shape = (16, 16, 16)
    b = rnd(shape, 11)
    x1 = np.zeros(shape)
    x2 = np.zeros(shape)
    for _ in range(10):
        x1 = oracle.gs_forward(H27, b, x1)
        x2 = oracle.gs_multicolor_forward(H27, b, x2)
    rel = np.max(np.abs(x1 - x2)) / np.max(np.abs(x1))
    assert rel > 1e-3


# --------------------------------------------------------------------------
# c4: restriction, prolongation, V-cycle
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(6, 6, 6), (5, 7, 4), (1, 2, 3)])
def test_restriction_is_injection_and_prolongation_its_transpose(shape):
    r = rnd(shape, 12)
    rc = oracle.restrict_residual(H27, r, np.zeros(shape))
    assert np.array_equal(rc, r[::2, ::2, ::2])
    zc = rnd(rc.shape, 13)
    z = rnd(shape, 14)
    zp = oracle.prolong_add(zc, z)
    want = z.copy()
    want[::2, ::2, ::2] += zc
    assert np.array_equal(zp, want)
    # <R f, c> = <f, P c>
    f = rnd(shape, 15)
    Rf = oracle.restrict_residual(H27, f, np.zeros(shape))
    Pc = oracle.prolong_add(zc, np.zeros(shape))
    assert oracle.dot(Rf, zc) == oracle.dot(f, Pc)


def test_restriction_of_residual():
    shape = (6, 5, 7)
    r, z = rnd(shape, 16), rnd(shape, 17)
    rc = oracle.restrict_residual(H27, r, z)
    res = r - (dense_from_apply(H27, shape) @ z.ravel()).reshape(shape)
    assert np.max(np.abs(rc - res[::2, ::2, ::2])) <= 1e-13 * np.max(np.abs(res))


def test_coarsen_kappa_is_block_mean():
    k = kappa_small((6, 4, 8))
    kc = oracle.coarsen_kappa(k)
    want = k.reshape(3, 2, 2, 2, 4, 2).mean(axis=(1, 3, 5))
    assert np.max(np.abs(kc - want)) <= 1e-15 * np.max(want)
    # ragged: an odd extent keeps a single fine cell at the end
    k = kappa_small((3, 2, 2))
    kc = oracle.coarsen_kappa(k)
    assert kc.shape == (2, 1, 1)
    assert abs(kc[1, 0, 0] - k[2].mean()) <= 1e-15 * k.max()


def test_vcycle_one_level_is_symgs_from_zero():
    shape = (5, 6, 7)
    r = rnd(shape, 18)
    assert np.array_equal(oracle.mg_vcycle(H27, r, 1),
                          oracle.symgs(H27, r, np.zeros(shape), 1))


def _dense_symgs_operator(A):
    """z = S r for one symmetric GS from z = 0: S = (D+U)^-1 D (D+L)^-1."""
    DL, DU, D = np.tril(A), np.triu(A), np.diag(np.diag(A))
    return np.linalg.solve(DU, D @ np.linalg.solve(DL, np.eye(A.shape[0])))


@pytest.mark.parametrize("kind", [H27, K7])
def test_two_level_vcycle_dense(kind):
    """Two-level V-cycle assembled from dense matrices."""
    shape = (4, 6, 5)
    kap = kappa_small(shape, 19) if kind == K7 else None
    A = dense_from_apply(kind, shape, kap)
    cshape = tuple((n + 1) // 2 for n in shape)
    kc = oracle.coarsen_kappa(kap) if kind == K7 else None
    Ac = dense_from_apply(kind, cshape, kc)
    S, Sc = _dense_symgs_operator(A), _dense_symgs_operator(Ac)
    n = A.shape[0]
    idx = np.arange(n).reshape(shape)[::2, ::2, ::2].ravel()
    R = np.zeros((len(idx), n))
    R[np.arange(len(idx)), idx] = 1.0
    P = R.T
    I = np.eye(n)
    V = S + (I - S @ A) @ (S + P @ Sc @ R @ (I - A @ S))
    r = rnd(shape, 20)
    z = oracle.mg_vcycle(kind, r, 2, kap)
    zd = V @ r.ravel()
    assert np.max(np.abs(z.ravel() - zd)) <= 1e-12 * np.max(np.abs(zd))


@pytest.mark.parametrize("kind", [H27, K7])
def test_vcycle_symmetric(kind):
    shape = (16, 16, 16)
    kap = gen.kappa_field(16, seed=7) if kind == K7 else None
    x, y = rnd(shape, 21), rnd(shape, 22)
    a = oracle.dot(oracle.mg_vcycle(kind, x, 4, kap), y)
    b = oracle.dot(x, oracle.mg_vcycle(kind, y, 4, kap))
    assert abs(a - b) <= 1e-13 * abs(a)


def test_forward_sweep_transpose_is_backward_sweep():
    """<S_f b1, b2> = <b1, S_b b2> (from zero): the transposed forward sweep is
    the backward sweep with transposed couplings (A symmetric)."""
    shape = (9, 8, 7)
    kap = kappa_small(shape, 23)
    for kind, k in ((H27, None), (K7, kap)):
        b1, b2 = rnd(shape, 24), rnd(shape, 25)
        f = oracle.gs_forward(kind, b1, np.zeros(shape), k)
        g = oracle.gs_backward(kind, b2, np.zeros(shape), k)
        a, c = oracle.dot(f, b2), oracle.dot(b1, g)
        assert abs(a - c) <= 1e-14 * abs(a)


# --------------------------------------------------------------------------
# c5: Dot2 and PCG
# --------------------------------------------------------------------------
def test_dot2_near_exact():
    for k in range(3):
        a = rnd((1000,), 30 + k) * 10.0 ** rnd((1000,), 40 + k) * 3
        b = rnd((1000,), 50 + k)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        d = oracle.dot(a, b)
        assert abs(Fraction(d) - exact) <= abs(exact) * Fraction(2.3e-16)


def test_dot2_ill_conditioned():
    """Cancellation that a plain sum gets wrong but Dot2 gets right."""
    a = np.array([1e16, 1.0, -1e16, 1.0])
    b = np.ones(4)
    assert oracle.dot(a, b) == 2.0


@pytest.mark.parametrize("kind,levels", [(H27, 0), (H27, 1), (H27, 2), (K7, 0), (K7, 2)])
def test_pcg_converges_to_dense_solution(kind, levels):
    shape = (4, 4, 6)
    kap = kappa_small(shape, 26) if kind == K7 else None
    A = dense_from_apply(kind, shape, kap)
    b = rnd(shape, 27)
    x, it, hist, st = oracle.pcg(kind, b, levels, kap, max_iters=200, rtol=1e-12,
                                 fixed_iters=False)
    assert st == 0
    xd = np.linalg.solve(A, b.ravel())
    assert np.max(np.abs(x.ravel() - xd)) <= 1e-10 * np.max(np.abs(xd))
    # the recurrence residual equals the true residual
    rt = np.linalg.norm(b.ravel() - A @ x.ravel())
    assert abs(hist[-1] - rt) <= 1e-12 * np.linalg.norm(b)


def test_pcg_recovers_ones():
    shape = (16, 16, 16)
    b = oracle.apply(H27, np.ones(shape))
    x, it, hist, st = oracle.pcg(H27, b, 4, max_iters=50, fixed_iters=True)
    assert st == 0 and it == 50
    assert np.max(np.abs(x - 1.0)) < 1e-9
    # MG-PCG reduces the residual by many orders of magnitude
    assert hist[-1] / hist[0] < 1e-10


def test_pcg_mg_faster_than_sgs_faster_than_cg():
    shape = (16, 16, 16)
    b = oracle.apply(H27, np.ones(shape))
    its = []
    for levels in (0, 1, 4):
        _, it, _, st = oracle.pcg(H27, b, levels, max_iters=500, rtol=1e-10,
                                  fixed_iters=False)
        assert st == 0
        its.append(it)
    assert its[0] > its[1] > its[2]


@pytest.mark.parametrize("kind", [H27, K7])
def test_fp32_preconditioned_pcg_reaches_1e10(kind):
    n = 16
    kap = gen.kappa_field(n, seed=3) if kind == K7 else None
    b = oracle.apply(kind, np.ones((n, n, n)), kap)
    x64, it64, h64, st64 = oracle.pcg(kind, b, 3, kap, max_iters=200, rtol=1e-10,
                                      fixed_iters=False)
    x32, it32, h32, st32 = oracle.pcg(kind, b, 3, kap, max_iters=200, rtol=1e-10,
                                      fixed_iters=False, precond_f32=True)
    assert st64 == 0 and st32 == 0
    assert h32[-1] <= 1e-10 * h32[0]
    assert np.max(np.abs(x32 - x64)) <= 1e-7 * np.max(np.abs(x64))
    assert it32 <= it64 + 3


def test_fp32_vcycle_close_to_fp64_vcycle():
    n = 16
    kap = gen.kappa_field(n, seed=4)
    r = rnd((n, n, n), 28)
    for kind, k in ((H27, None), (K7, kap)):
        z64 = oracle.mg_vcycle(kind, r, 3, k)
        z32 = oracle.mg_vcycle_f32(kind, r.astype(np.float32), 3, k)
        assert np.max(np.abs(z32 - z64)) <= 1e-5 * np.max(np.abs(z64))
        y32 = oracle.apply_f32(kind, r.astype(np.float32),
                               None if k is None else k.astype(np.float32))
        y64 = oracle.apply(kind, r, k)
        assert np.max(np.abs(y32 - y64)) <= 1e-5 * np.max(np.abs(y64))


# --------------------------------------------------------------------------
# c10: adjoint gradient
# --------------------------------------------------------------------------
def test_kappa_gradient_matches_finite_differences():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    n = 8
    shape = (n, n, n)
    kap = gen.kappa_field(n, seed=5)
    b = np.ones(shape)
    ut = gen.target(shape, seed=6)

    def solve(k):
        A = sp.csc_matrix(dense_from_apply(K7, shape, k))
        return spla.spsolve(A, b.ravel()).reshape(shape)

    def loss(k):
        u = solve(k)
        return 0.5 * np.sum((u - ut) ** 2)

    u = solve(kap)
    A = sp.csc_matrix(dense_from_apply(K7, shape, kap))
    lam = spla.spsolve(A.T, (u - ut).ravel()).reshape(shape)
    g = oracle.kappa_grad(u, lam)
    cells = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, 3, 4), (3, 0, 5), (4, 5, 0),
             (3, 3, 3), (2, 5, 6), (7, 1, 2), (5, 7, 3), (1, 6, 7)]
    for c in cells:
        h = 1e-5 * kap[c]
        kp, km = kap.copy(), kap.copy()
        kp[c] += h
        km[c] -= h
        fd = (loss(kp) - loss(km)) / (2 * h)
        assert abs(fd - g[c]) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(g)))


# --------------------------------------------------------------------------
# c7: block SSOR
# --------------------------------------------------------------------------
def block_dense(D, L, U):
    """Dense 5N x 5N matrix of the block operator (built from the block
    definition by scattering blocks)."""
    nz, ny, nx = D.shape[:3]
    n = nx * ny * nz
    A = np.zeros((5 * n, 5 * n))

    def P(x, y, z):
        return (z * ny + y) * nx + x

    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        p = P(x, y, z)
        A[5 * p:5 * p + 5, 5 * p:5 * p + 5] = D[z, y, x]
        for d, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            if x - dx >= 0 and y - dy >= 0 and z - dz >= 0:
                q = P(x - dx, y - dy, z - dz)
                A[5 * p:5 * p + 5, 5 * q:5 * q + 5] = L[z, y, x, d]
            if x + dx < nx and y + dy < ny and z + dz < nz:
                q = P(x + dx, y + dy, z + dz)
                A[5 * p:5 * p + 5, 5 * q:5 * q + 5] = U[z, y, x, d]
    return A


def test_block_sweeps_match_dense():
    shape = (2, 4, 3)
    D, L, U, b = gen.block_ssor_inputs(0, shape=shape, seed=31)
    A = block_dense(D, L, U)
    u = rnd(shape + (5,), 32)
    y = oracle.block_apply(D, L, U, u)
    assert np.max(np.abs(y.ravel() - A @ u.ravel())) <= 1e-13 * np.max(np.abs(y))
    om = 1.2
    Dd = np.zeros_like(A)
    for p in range(A.shape[0] // 5):
        Dd[5 * p:5 * p + 5, 5 * p:5 * p + 5] = A[5 * p:5 * p + 5, 5 * p:5 * p + 5]
    Ld = np.tril(A - Dd)
    Ud = np.triu(A - Dd)
    r = rnd(shape + (5,), 33)
    v = oracle.block_lower(D, L, om, r)
    vd = np.linalg.solve(Dd + om * Ld, r.ravel())
    assert np.max(np.abs(v.ravel() - vd)) <= 1e-13 * np.max(np.abs(vd))
    w = oracle.block_upper(D, U, om, v)
    wd = np.linalg.solve(Dd + om * Ud, Dd @ vd)
    assert np.max(np.abs(w.ravel() - wd)) <= 1e-13 * np.max(np.abs(wd))


def test_ssor_delta_form_equals_forward_backward_sor():
    """u + w(2-w) (D+wU)^-1 D (D+wL)^-1 (b - A u) equals one classical
    in-place forward block-SOR sweep followed by one backward sweep."""
    shape = (3, 2, 4)
    D, L, U, b = gen.block_ssor_inputs(0, shape=shape, seed=34)
    A = block_dense(D, L, U)
    om = 1.2
    nb = A.shape[0] // 5
    u = rnd(shape + (5,), 35).ravel()

    def sor_sweep(u, order):
        u = u.copy()
        for p in order:
            s = slice(5 * p, 5 * p + 5)
            off = A[s] @ u - A[s, s] @ u[s]
            u[s] = (1 - om) * u[s] + om * np.linalg.solve(A[s, s], b.ravel()[s] - off)
        return u

    classic = sor_sweep(sor_sweep(u, range(nb)), reversed(range(nb)))
    delta = oracle.ssor(D, L, U, om, b, u.reshape(shape + (5,)), 1)
    assert np.max(np.abs(delta.ravel() - classic)) <= 1e-13 * np.max(np.abs(classic))


def test_ssor_scalar_special_case_is_symgs():
    """D = 6 I, L = U = -I, omega = 1: each of the 5 components is the 7-point
    Laplacian and one SSOR step from u is one symmetric GS from u."""
    shape = (3, 4, 5)
    D = np.broadcast_to(6.0 * np.eye(5), shape + (5, 5)).copy()
    L = np.broadcast_to(-np.eye(5), shape + (3, 5, 5)).copy()
    U = L.copy()
    b = rnd(shape + (5,), 36)
    u0 = rnd(shape + (5,), 37)
    u1 = oracle.ssor(D, L, U, 1.0, b, u0, 1)
    for c in range(5):
        s = oracle.symgs(K7, b[..., c], u0[..., c], 1, np.ones(shape))
        assert np.max(np.abs(u1[..., c] - s)) <= 1e-13 * np.max(np.abs(s))


def test_ssor_converges_to_dense_solution():
    shape = (3, 3, 2)
    D, L, U, b = gen.block_ssor_inputs(0, shape=shape, seed=38)
    A = block_dense(D, L, U)
    u = oracle.ssor(D, L, U, 1.2, b, np.zeros(shape + (5,)), 60)
    ud = np.linalg.solve(A, b.ravel())
    assert np.max(np.abs(u.ravel() - ud)) <= 1e-12 * np.max(np.abs(ud))



# --------------------------------------------------------------------------
# Blocks formed from the state (NPB-LU's Jacobians, synthetic quadratic flux)
# --------------------------------------------------------------------------
def jac_parts(P, k):
    base = 2 + 55 * k
    return (P[base:base + 25].reshape(5, 5), P[base + 25:base + 50].reshape(5, 5),
            P[base + 50:base + 55])


def flux(P, k, q):
    """F_k(q) = C_k q + (g_k . q) E_k q for q of shape (..., 5)."""
    C, E, g = jac_parts(P, k)
    return q @ C.T + (q @ g)[..., None] * (q @ E.T)


def fd_jacobian(P, k, q, h=1e-3):
    """Central-difference Jacobian of F_k at q: exact for a quadratic flux up
    to rounding."""
    J = np.empty((5, 5))
    for j in range(5):
        e = np.zeros(5)
        e[j] = h
        J[:, j] = (flux(P, k, q + e) - flux(P, k, q - e)) / (2 * h)
    return J


def test_block_jac_blocks_are_flux_jacobians():
    """D_p - sigma I = dF_0/du at u_p; -2 (L_{p,d} + nu I) = dF_{d+1}/du at
    u_{p-e_d}; 2 (U_{p,d} + nu I) = dF_{d+1}/du at u_{p+e_d}; couplings that
    leave the grid are 0."""
    shape = (3, 4, 5)
    P, _, u = gen.block_jac_inputs(shape, seed=61)
    D, L, U = oracle.block_jac(P, u)
    sigma, nu = P[0], P[1]
    nz, ny, nx = shape
    I5 = np.eye(5)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        assert np.max(np.abs(D[z, y, x] - sigma * I5 - fd_jacobian(P, 0, u[z, y, x]))) <= 1e-10
        for d, (dx, dy, dz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            lo = (z - dz, y - dy, x - dx)
            hi = (z + dz, y + dy, x + dx)
            if min(lo) >= 0:
                J = fd_jacobian(P, d + 1, u[lo])
                assert np.max(np.abs(-2 * (L[z, y, x, d] + nu * I5) - J)) <= 1e-10
            else:
                assert not L[z, y, x, d].any()
            if hi[0] < nz and hi[1] < ny and hi[2] < nx:
                J = fd_jacobian(P, d + 1, u[hi])
                assert np.max(np.abs(2 * (U[z, y, x, d] + nu * I5) - J)) <= 1e-10
            else:
                assert not U[z, y, x, d].any()


def test_block_jac_depends_on_one_point_per_block():
    """Changing u at one point q changes exactly D_q, L_{q+e_d,d} and
    U_{q-e_d,d}, and nothing else."""
    shape = (4, 3, 5)
    P, _, u = gen.block_jac_inputs(shape, seed=62)
    D0, L0, U0 = oracle.block_jac(P, u)
    q = (2, 1, 3)
    u2 = u.copy()
    u2[q] += 0.25
    D1, L1, U1 = oracle.block_jac(P, u2)
    changed = set()
    nz, ny, nx = shape
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if np.any(D1[z, y, x] != D0[z, y, x]):
            changed.add(("D", z, y, x))
        for d in range(3):
            if np.any(L1[z, y, x, d] != L0[z, y, x, d]):
                changed.add(("L", z, y, x, d))
            if np.any(U1[z, y, x, d] != U0[z, y, x, d]):
                changed.add(("U", z, y, x, d))
    z, y, x = q
    want = {("D", z, y, x),
            ("L", z, y, x + 1, 0), ("L", z, y + 1, x, 1), ("L", z + 1, y, x, 2),
            ("U", z, y, x - 1, 0), ("U", z, y - 1, x, 1), ("U", z - 1, y, x, 2)}
    assert changed == want


def jac_operator_closed_form(P, u):
    """A(u) u from the flux alone (independent of the block assembly).  With
    J_k(q) q = 2 F_k(q) - C_k q (Euler's identity for the quadratic part) and
    zero padding (F_k(0) = 0 drops the couplings that leave the grid):
      (A(u) u)_p = sigma u_p + 2 F_0(u_p) - C_0 u_p - nu sum_{6 nbrs} u_q
                   + sum_d [G_d(u_{p+e_d}) - G_d(u_{p-e_d})] / 2,
    G_d(q) = 2 F_{d+1}(q) - C_{d+1} q."""
    sigma, nu = P[0], P[1]
    up = np.pad(u, ((1, 1), (1, 1), (1, 1), (0, 0)))
    c = up[1:-1, 1:-1, 1:-1]
    C0 = jac_parts(P, 0)[0]
    out = sigma * c + 2 * flux(P, 0, c) - c @ C0.T
    for d, ax in enumerate((2, 1, 0)):  # x, y, z are array axes 2, 1, 0
        hi = np.roll(up, -1, axis=ax)[1:-1, 1:-1, 1:-1]
        lo = np.roll(up, 1, axis=ax)[1:-1, 1:-1, 1:-1]
        Cd = jac_parts(P, d + 1)[0]
        G = lambda q: 2 * flux(P, d + 1, q) - q @ Cd.T  # noqa: E731
        out = out - nu * (hi + lo) + 0.5 * (G(hi) - G(lo))
    return out


@pytest.mark.parametrize("shape", [(3, 4, 5), (1, 2, 6), (5, 1, 1)])
def test_block_jac_operator_matches_flux_closed_form(shape):
    P, _, u = gen.block_jac_inputs(shape, seed=63)
    D, L, U = oracle.block_jac(P, u)
    got = oracle.block_apply(D, L, U, u)
    want = jac_operator_closed_form(P, u)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_ssor_jac_linear_flux_is_block_ssor_with_constant_blocks():
    """E_k = 0, g_k = 0: the blocks no longer depend on u (D = sigma I + C_0,
    L = -nu I - C_{d+1}/2, U = -nu I + C_{d+1}/2 inside the grid), and the
    steps are plain block SSOR steps with those blocks."""
    shape = (3, 4, 2)
    P, b, u0 = gen.block_jac_inputs(shape, seed=64)
    for k in range(4):
        P[2 + 55 * k + 25:2 + 55 * k + 55] = 0.0
    nz, ny, nx = shape
    D = np.broadcast_to(P[0] * np.eye(5) + jac_parts(P, 0)[0], shape + (5, 5)).copy()
    L = np.zeros(shape + (3, 5, 5))
    U = np.zeros(shape + (3, 5, 5))
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        for d, c in enumerate((x, y, z)):
            Cd = jac_parts(P, d + 1)[0]
            n = (nx, ny, nz)[d]
            if c > 0:
                L[z, y, x, d] = -P[1] * np.eye(5) - 0.5 * Cd
            if c < n - 1:
                U[z, y, x, d] = -P[1] * np.eye(5) + 0.5 * Cd
    got = oracle.ssor_jac(P, 1.2, b, u0, 3)
    want = oracle.ssor(D, L, U, 1.2, b, u0, 3)
    assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))


def test_ssor_jac_step_uses_blocks_of_its_start_state():
    shape = (2, 3, 4)
    P, b, u0 = gen.block_jac_inputs(shape, seed=65)
    u1 = oracle.ssor_jac(P, 1.2, b, u0, 1)
    D, L, U = oracle.block_jac(P, u0)
    want = oracle.ssor(D, L, U, 1.2, b, u0, 1)
    assert np.array_equal(u1, want)
    u2 = oracle.ssor_jac(P, 1.2, b, u0, 2)
    D, L, U = oracle.block_jac(P, u1)
    assert np.array_equal(u2, oracle.ssor(D, L, U, 1.2, b, u1, 1))


def test_block_jac_rows_stay_diagonally_dominant():
    """The input recipe's claim: for |u| <= 1.5 every Jacobian entry is below
    0.25, so every scalar row of A(u) is strictly diagonally dominant (the 5x5
    eliminations need no pivoting).  Checked on the recipe's parameters at
    u = +-1.5 with random signs, where the bound is tightest."""
    shape = (4, 5, 3)
    P, _, _ = gen.block_jac_inputs(shape, seed=67)
    rng = np.random.default_rng(3)
    u = 1.5 * rng.choice([-1.0, 1.0], size=shape + (5,))
    D, L, U = oracle.block_jac(P, u)
    for k in range(4):
        C, E, g = jac_parts(P, k)
        for q in u.reshape(-1, 5)[:20]:
            J = C + (g @ q) * E + np.outer(E @ q, g)
            assert np.max(np.abs(J)) < 0.25
    diag = np.abs(D[..., range(5), range(5)])
    off = np.abs(D).sum(axis=-1) - diag + np.abs(L).sum(axis=(-3, -1)) + np.abs(U).sum(axis=(-3, -1))
    assert np.all(diag > off) and diag.min() >= 9.75 and off.max() < 8.0


def test_ssor_jac_converges_to_the_nonlinear_solution():
    """The fixed point of the steps solves A(u) u = b, checked with the
    closed form of A(u) u (not with the oracle's blocks)."""
    shape = (4, 3, 5)
    P, b, u0 = gen.block_jac_inputs(shape, seed=66)
    u = oracle.ssor_jac(P, 1.2, b, u0, 40)
    res = b - jac_operator_closed_form(P, u)
    assert np.max(np.abs(res)) <= 1e-12 * np.max(np.abs(b))
    assert np.max(np.abs(b - jac_operator_closed_form(P, u0))) > 1.0

# --------------------------------------------------------------------------
# c9 / c11: inputs
# --------------------------------------------------------------------------
def test_splitmix64_reference_value():
    """SplitMix64 from state 0: first output 0xE220A8397B1DCDAF (published
    reference sequence)."""
    v = gen._mix(np.uint64(0) + gen.GAMMA)
    assert int(v) == 0xE220A8397B1DCDAF


def test_inputs_deterministic_and_distributed():
    a = gen.uniform(5, 2, 1000)
    assert np.array_equal(a, gen.uniform(5, 2, 1000))
    assert not np.array_equal(a, gen.uniform(6, 2, 1000))
    assert 0.0 <= a.min() and a.max() < 1.0
    z = gen.normal(1, 1, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.02
    k = gen.kappa_field(48, seed=9)
    lk = np.log(k)
    assert abs(lk.mean()) < 0.3 and 0.5 < lk.var() < 1.5
    assert np.array_equal(k, gen.kappa_field(48, seed=9))
    s = gen.batch_sides(64)
    assert len(s) == 64 and set(s) <= set(gen.BATCH_SIDES) and len(set(s)) >= 4


@pytest.mark.parametrize("make", [
    lambda seed: gen.block_ssor_inputs(0, shape=(3, 4, 5), seed=seed),
    lambda seed: gen.block_jac_inputs((3, 4, 5), seed=seed),
    lambda seed: gen.line_penta_inputs((3, 4, 5), k=5, seed=seed),
    lambda seed: gen.line_btri_inputs((3, 4, 5), seed=seed),
])
def test_every_generator_is_deterministic_per_seed(make):
    """Same seed: bitwise the same arrays; another seed: different ones (the
    counter-based streams depend on the seed, the array id and the index
    only)."""
    a, b, c = make(11), make(11), make(12)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y)
        if np.size(x) > 2:  # the parameter vector's fixed sigma, nu aside
            assert not np.array_equal(x, z)


@pytest.mark.parametrize("n", [64, 128, 256])
def test_stored_pcg_histories_start_at_closed_form_norm_of_b(n):
    """The stored oracle residual histories (tests/golden) start at
    ||r0|| = ||b|| with b = A*ones, whose entries are 27 - prod(3 or 2 per
    axis): 0 inside, 9 on faces, 15 on edges, 19 at corners; and they end
    below 1e-10 ||b|| (the stopping rule), the step before not."""
    import os
    from math import comb
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "hpcg_pcg_history_%d.txt" % n)
    with open(path) as f:
        hist = np.array([float(v) for v in f if v.strip() and not v.startswith("#")])
    bb = sum(comb(3, k) * 2 ** k * (n - 2) ** (3 - k) * (27 - 3 ** (3 - k) * 2 ** k) ** 2
             for k in range(4))
    assert abs(hist[0] - np.sqrt(bb)) <= 1e-12 * np.sqrt(bb)
    assert hist[-1] <= 1e-10 * hist[0] < hist[-2]


def _load_samples(n, mode):
    import os
    hist, idx, val, iters = [], [], [], None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "hpcg_pcg_samples_%d_%s.txt" % (n, mode))
    with open(path) as f:
        for line in f:
            if line.startswith("# iterations"):
                iters = int(line.split()[2])
            elif line.startswith("#") or not line.strip():
                continue
            elif line.startswith("h "):
                hist.append(float(line.split()[2]))
            else:
                a, v = line.split()
                idx.append(int(a))
                val.append(float(v))
    return iters, np.array(hist), np.array(idx), np.array(val)


@pytest.mark.parametrize("n", [128, 256])
def test_stored_pcg_samples_are_consistent_oracle_runs(n):
    """The stored samples of the oracle's full-size MG-PCG solves
    (tests/golden/make_hpcg_pcg_samples.py) against facts outside the run
    that wrote them: the history starts at the closed-form ||b||; the
    50-iteration run and the run to 1e-10 are separate oracle runs whose
    first 51 residuals agree bitwise (the stopping rule does not change the
    iterates), and the run to 1e-10 reproduces the separately stored
    residual history; the sample positions are m2s_inputs.sample_points; the
    converged solution is the exact solution ones to within the solve's
    error (the system is A x = A*ones), while 50 iterations are not yet."""
    import os
    from math import comb
    it50, h50, i50, x50 = _load_samples(n, "fixed50")
    itr, hr, ir, xr = _load_samples(n, "rtol")
    bb = sum(comb(3, k) * 2 ** k * (n - 2) ** (3 - k) * (27 - 3 ** (3 - k) * 2 ** k) ** 2
             for k in range(4))
    assert abs(h50[0] - np.sqrt(bb)) <= 1e-12 * np.sqrt(bb)
    assert it50 == 50 and len(h50) == 51 and itr == len(hr) - 1
    assert np.array_equal(h50, hr[:51])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "hpcg_pcg_history_%d.txt" % n)
    with open(path) as f:
        stored = np.array([float(v) for v in f if v.strip() and not v.startswith("#")])
    assert np.array_equal(hr, stored)
    want = gen.sample_points((n, n, n), 16384)
    assert np.array_equal(i50, want) and np.array_equal(ir, want)
    assert np.max(np.abs(xr - 1.0)) <= 1e-8
    assert np.max(np.abs(x50 - 1.0)) > 1e-8


# ---------------------------------------------------------------------------
# NPB-SP-shaped line solves (Sec. 1, Sec. 7.2.2): pentadiagonal systems along
# the lines of one axis, terms outside a line dropped.
# ---------------------------------------------------------------------------
LINE_SHAPES = [(3, 4, 5), (5, 3, 4), (4, 5, 3), (1, 2, 7), (6, 1, 2)]


def _line_dense(coef, axis):
    """Per line (in the order of the other two coordinates) the dense m x m
    matrix assembled from the band, independently of the oracle."""
    c = np.moveaxis(coef, 2 - axis, 2)  # line axis last among the grid axes
    m = c.shape[2]
    mats = {}
    for i0 in range(c.shape[0]):
        for i1 in range(c.shape[1]):
            A = np.zeros((m, m))
            for i in range(m):
                for j, off in enumerate((-2, -1, 0, 1, 2)):
                    if 0 <= i + off < m:
                        A[i, i + off] = c[i0, i1, i, j]
            mats[(i0, i1)] = A
    return mats


@pytest.mark.parametrize("shape", LINE_SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_line_penta_matches_dense_solves(shape, axis):
    coef, rhs = gen.line_penta_inputs(shape, k=3, seed=gen.BASE_SEED + 31)
    v = oracle.line_penta(coef, rhs, axis)
    mats = _line_dense(coef, axis)
    r = np.moveaxis(rhs, 2 - axis, 2)
    vv = np.moveaxis(v, 2 - axis, 2)
    for (i0, i1), A in mats.items():
        ref = np.linalg.solve(A, r[i0, i1])
        assert np.max(np.abs(vv[i0, i1] - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
        # residual of the band applied to the oracle's solution
        assert np.max(np.abs(A @ vv[i0, i1] - r[i0, i1])) <= 1e-13


def test_line_penta_tridiagonal_matches_solve_banded():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    shape = (4, 3, 9)
    coef, rhs = gen.line_penta_inputs(shape, k=2, seed=gen.BASE_SEED + 32)
    coef[..., 0] = 0.0
    coef[..., 4] = 0.0
    v = oracle.line_penta(coef, rhs, 0)
    for z in range(shape[0]):
        for y in range(shape[1]):
            ab = np.zeros((3, shape[2]))
            ab[0, 1:] = coef[z, y, :-1, 3]   # super-diagonal: d of row i at column i+1
            ab[1, :] = coef[z, y, :, 2]
            ab[2, :-1] = coef[z, y, 1:, 1]   # sub-diagonal: b of row i at column i-1
            ref = scipy_linalg.solve_banded((1, 1), ab, rhs[z, y])
            assert np.max(np.abs(v[z, y] - ref)) <= 1e-13


def test_line_penta_diagonal_is_exact_division():
    shape = (3, 5, 4)
    coef, rhs = gen.line_penta_inputs(shape, k=4, seed=gen.BASE_SEED + 33)
    coef[..., [0, 1, 3, 4]] = 0.0
    for axis in range(3):
        v = oracle.line_penta(coef, rhs, axis)
        assert np.array_equal(v, rhs / coef[..., 2:3])


def test_line_penta_axis_permutation():
    """Solving along x equals solving along z of the grid with x and z
    exchanged (the same lines, the same arithmetic): pins the axis order."""
    shape = (3, 4, 6)
    coef, rhs = gen.line_penta_inputs(shape, k=2, seed=gen.BASE_SEED + 34)
    vx = oracle.line_penta(coef, rhs, 0)
    ct = np.ascontiguousarray(np.transpose(coef, (2, 1, 0, 3)))
    rt = np.ascontiguousarray(np.transpose(rhs, (2, 1, 0, 3)))
    vz = oracle.line_penta(ct, rt, 2)
    assert np.array_equal(vx, np.transpose(vz, (2, 1, 0, 3)))
    vy = oracle.line_penta(coef, rhs, 1)
    ct = np.ascontiguousarray(np.transpose(coef, (0, 2, 1, 3)))
    rt = np.ascontiguousarray(np.transpose(rhs, (0, 2, 1, 3)))
    assert np.array_equal(vy, np.transpose(oracle.line_penta(ct, rt, 0), (0, 2, 1, 3)))


# ---------------------------------------------------------------------------
# NPB-BT-shaped line solves: 5x5 block-tridiagonal systems along the lines
# of one axis.
# ---------------------------------------------------------------------------
def _btri_dense(blk, axis):
    b = np.moveaxis(blk, 2 - axis, 2)
    m = b.shape[2]
    mats = {}
    for i0 in range(b.shape[0]):
        for i1 in range(b.shape[1]):
            A = np.zeros((5 * m, 5 * m))
            for i in range(m):
                for k, off in enumerate((-1, 0, 1)):
                    j = i + off
                    if 0 <= j < m:
                        A[5 * i:5 * i + 5, 5 * j:5 * j + 5] = b[i0, i1, i, k]
            mats[(i0, i1)] = A
    return mats


@pytest.mark.parametrize("shape", LINE_SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_line_btri_matches_dense_solves(shape, axis):
    blk, rhs = gen.line_btri_inputs(shape, seed=gen.BASE_SEED + 35)
    v = oracle.line_btri(blk, rhs, axis)
    r = np.moveaxis(rhs, 2 - axis, 2)
    vv = np.moveaxis(v, 2 - axis, 2)
    for (i0, i1), A in _btri_dense(blk, axis).items():
        ref = np.linalg.solve(A, r[i0, i1].ravel())
        assert np.max(np.abs(vv[i0, i1].ravel() - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(A @ vv[i0, i1].ravel() - r[i0, i1].ravel())) <= 1e-13


def test_line_btri_diagonal_blocks_reduce_to_tridiagonal():
    """Blocks that are multiples of the identity decouple the 5 components
    into 5 scalar tridiagonal systems (scipy's banded solver)."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    shape = (3, 2, 8)
    rng = np.random.default_rng(5)
    s = rng.uniform(-0.25, 0.25, size=shape + (3,))
    s[..., 1] += 3.0
    blk = s[..., :, None, None] * np.eye(5)
    _, rhs = gen.line_btri_inputs(shape, seed=gen.BASE_SEED + 36)
    v = oracle.line_btri(blk, rhs, 0)
    for z in range(shape[0]):
        for y in range(shape[1]):
            ab = np.zeros((3, shape[2]))
            ab[0, 1:] = s[z, y, :-1, 2]
            ab[1, :] = s[z, y, :, 1]
            ab[2, :-1] = s[z, y, 1:, 0]
            for c in range(5):
                ref = scipy_linalg.solve_banded((1, 1), ab, rhs[z, y, :, c])
                assert np.max(np.abs(v[z, y, :, c] - ref)) <= 1e-13


def test_line_btri_axis_permutation():
    shape = (3, 4, 6)
    blk, rhs = gen.line_btri_inputs(shape, seed=gen.BASE_SEED + 37)
    vx = oracle.line_btri(blk, rhs, 0)
    bt = np.ascontiguousarray(np.transpose(blk, (2, 1, 0, 3, 4, 5)))
    rt = np.ascontiguousarray(np.transpose(rhs, (2, 1, 0, 3)))
    assert np.array_equal(vx, np.transpose(oracle.line_btri(bt, rt, 2), (2, 1, 0, 3)))


# ---------------------------------------------------------------------------
# ILU(0) of the HPCG 27-point matrix (Sec. 1; the ILU micro-benchmark of
# Sec. 7.2.1 uses the 27-point stencil).
# ---------------------------------------------------------------------------
ILU_SHAPES = [(3, 4, 5), (5, 3, 4), (4, 4, 4), (2, 6, 3)]


def _offsets27():
    return [((o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1) for o in range(27)]


def _dense_hpcg(shape):
    nz, ny, nx = shape
    n = nx * ny * nz
    A = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = (z * ny + y) * nx + x
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            qx, qy, qz = x + dx, y + dy, z + dz
                            if 0 <= qx < nx and 0 <= qy < ny and 0 <= qz < nz:
                                A[p, (qz * ny + qy) * nx + qx] = 26.0 if (dx, dy, dz) == (0, 0, 0) else -1.0
    return A


def _dense_factors(F):
    nz, ny, nx, _ = F.shape
    n = nx * ny * nz
    L, U = np.eye(n), np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = (z * ny + y) * nx + x
                for o, (dx, dy, dz) in enumerate(_offsets27()):
                    qx, qy, qz = x + dx, y + dy, z + dz
                    if 0 <= qx < nx and 0 <= qy < ny and 0 <= qz < nz:
                        q = (qz * ny + qy) * nx + qx
                        (L if o < 13 else U)[p, q] = F[z, y, x, o]
    return L, U


@pytest.mark.parametrize("shape", ILU_SHAPES)
def test_ilu0_matches_a_on_its_pattern(shape):
    """The defining property of ILU(0): (L U)_pq = a_pq wherever a_pq != 0."""
    A = _dense_hpcg(shape)
    L, U = _dense_factors(oracle.ilu0_factor(shape))
    LU = L @ U
    mask = A != 0
    assert np.max(np.abs(LU[mask] - A[mask])) <= 1e-12
    # and it is not the exact factorisation (fill-in outside the pattern)
    if min(shape) >= 2:
        assert np.max(np.abs(LU - A)) > 1e-3


@pytest.mark.parametrize("shape", ILU_SHAPES)
def test_ilu0_apply_solves_lu(shape):
    F = oracle.ilu0_factor(shape)
    L, U = _dense_factors(F)
    r = gen.random_vector(shape, seed=gen.BASE_SEED + 90)
    z = oracle.ilu0_apply(F, r)
    assert np.max(np.abs(L @ (U @ z.ravel()) - r.ravel())) <= 1e-12


def test_ilu0_of_a_symmetric_matrix_has_u_equal_d_lt():
    """A is symmetric, so ILU(0) gives U = D L^T (D the pivots)."""
    L, U = _dense_factors(oracle.ilu0_factor((3, 4, 5)))
    D = np.diag(np.diag(U))
    assert np.max(np.abs(U - D @ L.T)) <= 1e-12


def test_ilu0_of_a_line_is_the_exact_lu():
    """On a 1 x 1 x m grid the pattern is tridiagonal: no fill, so ILU(0) is
    the exact LU and its application the exact solve."""
    shape = (1, 1, 9)
    A = _dense_hpcg(shape)
    F = oracle.ilu0_factor(shape)
    L, U = _dense_factors(F)
    assert np.max(np.abs(L @ U - A)) <= 1e-13
    r = gen.random_vector(shape, seed=gen.BASE_SEED + 91)
    assert np.max(np.abs(oracle.ilu0_apply(F, r).ravel() - np.linalg.solve(A, r.ravel()))) <= 1e-13
