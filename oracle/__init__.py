"""Serial CPU oracle for the Mat2Stencil solver hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the library never imports it.
It shares no code with the CUDA path.  Every routine is the plain definition
of its step as serial loops in lexicographic order (z outermost, x fastest),
in IEEE FP64 (the ``*_f32`` routines are the FP32-preconditioner form).

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` (closed forms, invariants, brute force on tiny
grids); none is "parity unpinned".

Operator kinds (paper Sec. 4.2 row functions, Sec. 7.1 HPCG):
  HPCG27 = 0  27-point, a_pp = 26, a_pq = -1, zero Dirichlet
  KAPPA7 = 1  variable-coefficient 7-point diffusion, face kappa = mean
"""
import ctypes
import numpy as np

from . import build as _build

HPCG27 = 0
KAPPA7 = 1

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i = ctypes.c_int
_ll = ctypes.c_longlong
_d = ctypes.c_double


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "or_apply": [_i, _i, _i, _i, _dp, _dp, _dp],
            "or_gs_forward": [_i, _i, _i, _i, _dp, _dp, _dp],
            "or_gs_backward": [_i, _i, _i, _i, _dp, _dp, _dp],
            "or_symgs": [_i, _i, _i, _i, _dp, _dp, _dp, _i],
            "or_gs_multicolor_forward": [_i, _i, _i, _i, _dp, _dp, _dp],
            "or_restrict_residual": [_i, _i, _i, _i, _dp, _dp, _dp, _dp],
            "or_prolong_add": [_i, _i, _i, _dp, _dp],
            "or_coarsen_kappa": [_i, _i, _i, _dp, _dp],
            "or_mg_vcycle": [_i, _i, _i, _i, _dp, _i, _dp, _dp],
            "or_apply_f32": [_i, _i, _i, _i, _fp, _fp, _fp],
            "or_symgs_f32": [_i, _i, _i, _i, _fp, _fp, _fp, _i],
            "or_mg_vcycle_f32": [_i, _i, _i, _i, _dp, _i, _fp, _fp],
            "or_dot": [_ll, _dp, _dp],
            "or_pcg": [_i, _i, _i, _i, _dp, _i, _i, _dp, _dp, _i, _d, _i, _dp,
                       ctypes.POINTER(_i)],
            "or_kappa_grad": [_i, _i, _i, _dp, _dp, _dp],
            "or_block_apply": [_i, _i, _i, _dp, _dp, _dp, _dp, _dp],
            "or_block_residual": [_i, _i, _i, _dp, _dp, _dp, _dp, _dp, _dp],
            "or_block_lower": [_i, _i, _i, _dp, _dp, _d, _dp, _dp],
            "or_block_upper": [_i, _i, _i, _dp, _dp, _d, _dp, _dp],
            "or_ssor": [_i, _i, _i, _dp, _dp, _dp, _d, _dp, _dp, _i],
            "or_block_jac": [_i, _i, _i, _dp, _dp, _dp, _dp, _dp],
            "or_ssor_jac": [_i, _i, _i, _dp, _d, _dp, _dp, _i],
            "or_line_penta": [_i, _i, _i, _i, _dp, _dp, _i],
            "or_line_btri": [_i, _i, _i, _i, _dp, _dp],
            "or_ilu0_factor": [_i, _i, _i, _dp],
            "or_ilu0_apply": [_i, _i, _i, _dp, _dp, _dp],
            "or_coarse_n": [_i],
            "or_abi_version": [],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None
        L.or_dot.restype = _d
        L.or_pcg.restype = _i
        L.or_coarse_n.restype = _i
        L.or_abi_version.restype = _i
        _lib = L
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _p(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.float32:
        return a.ctypes.data_as(_fp)
    raise TypeError(a.dtype)


def _dims(shape):
    nz, ny, nx = shape
    return nx, ny, nz


def coarse_n(n):
    return lib().or_coarse_n(int(n))


def apply(kind, x, kappa=None):
    """y = A x (Sec. 4.3.1 SpMV); x has shape (nz, ny, nx)."""
    x = _f64(x)
    y = np.empty_like(x)
    k = None if kappa is None else _f64(kappa)
    lib().or_apply(kind, *_dims(x.shape), _p(k), _p(x), _p(y))
    return y


def gs_forward(kind, b, x, kappa=None):
    """One lexicographic forward Gauss-Seidel sweep; returns the new x."""
    b = _f64(b)
    x = _f64(x).copy()
    k = None if kappa is None else _f64(kappa)
    lib().or_gs_forward(kind, *_dims(b.shape), _p(k), _p(b), _p(x))
    return x


def gs_backward(kind, b, x, kappa=None):
    b = _f64(b)
    x = _f64(x).copy()
    k = None if kappa is None else _f64(kappa)
    lib().or_gs_backward(kind, *_dims(b.shape), _p(k), _p(b), _p(x))
    return x


def symgs(kind, b, x, sweeps=1, kappa=None):
    """`sweeps` symmetric GS (forward then backward each); returns new x."""
    b = _f64(b)
    x = _f64(x).copy()
    k = None if kappa is None else _f64(kappa)
    lib().or_symgs(kind, *_dims(b.shape), _p(k), _p(b), _p(x), int(sweeps))
    return x


def gs_multicolor_forward(kind, b, x, kappa=None):
    """Negative control only: 8-colour reordered GS sweep (not the method)."""
    b = _f64(b)
    x = _f64(x).copy()
    k = None if kappa is None else _f64(kappa)
    lib().or_gs_multicolor_forward(kind, *_dims(b.shape), _p(k), _p(b), _p(x))
    return x


def restrict_residual(kind, r, z, kappa=None):
    r = _f64(r)
    z = _f64(z)
    nz, ny, nx = r.shape
    rc = np.empty((coarse_n(nz), coarse_n(ny), coarse_n(nx)))
    k = None if kappa is None else _f64(kappa)
    lib().or_restrict_residual(kind, nx, ny, nz, _p(k), _p(r), _p(z), _p(rc))
    return rc


def prolong_add(zc, z):
    z = _f64(z).copy()
    zc = _f64(zc)
    nz, ny, nx = z.shape
    lib().or_prolong_add(nx, ny, nz, _p(zc), _p(z))
    return z


def coarsen_kappa(kappa):
    kappa = _f64(kappa)
    nz, ny, nx = kappa.shape
    kc = np.empty((coarse_n(nz), coarse_n(ny), coarse_n(nx)))
    lib().or_coarsen_kappa(nx, ny, nz, _p(kappa), _p(kc))
    return kc


def mg_vcycle(kind, r, levels, kappa=None):
    r = _f64(r)
    z = np.empty_like(r)
    k = None if kappa is None else _f64(kappa)
    lib().or_mg_vcycle(kind, *_dims(r.shape), _p(k), int(levels), _p(r), _p(z))
    return z


def apply_f32(kind, x, kappa32=None):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    k = None if kappa32 is None else np.ascontiguousarray(kappa32, dtype=np.float32)
    lib().or_apply_f32(kind, *_dims(x.shape), _p(k), _p(x), _p(y))
    return y


def symgs_f32(kind, b, x, sweeps=1, kappa32=None):
    b = np.ascontiguousarray(b, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32).copy()
    k = None if kappa32 is None else np.ascontiguousarray(kappa32, dtype=np.float32)
    lib().or_symgs_f32(kind, *_dims(b.shape), _p(k), _p(b), _p(x), int(sweeps))
    return x


def mg_vcycle_f32(kind, r32, levels, kappa=None):
    """FP32 V-cycle; kappa is the FP64 fine kappa (FP32 copies derived inside)."""
    r32 = np.ascontiguousarray(r32, dtype=np.float32)
    z = np.empty_like(r32)
    k = None if kappa is None else _f64(kappa)
    lib().or_mg_vcycle_f32(kind, *_dims(r32.shape), _p(k), int(levels), _p(r32), _p(z))
    return z


def dot(a, b):
    a = _f64(a).ravel()
    b = _f64(b).ravel()
    return lib().or_dot(a.size, _p(a), _p(b))


def pcg(kind, b, levels, kappa=None, max_iters=50, rtol=0.0, fixed_iters=True,
        precond_f32=False):
    """PCG from x0 = 0.  Returns (x, iters, resid_hist, status)."""
    b = _f64(b)
    x = np.empty_like(b)
    hist = np.zeros(max_iters + 1)
    it = _i(0)
    k = None if kappa is None else _f64(kappa)
    st = lib().or_pcg(kind, *_dims(b.shape), _p(k), int(levels), int(bool(precond_f32)),
                      _p(b), _p(x), int(max_iters), float(rtol), int(bool(fixed_iters)),
                      _p(hist), ctypes.byref(it))
    return x, it.value, hist[: it.value + 1].copy(), st


def kappa_grad(u, lam):
    u = _f64(u)
    lam = _f64(lam)
    g = np.empty_like(u)
    lib().or_kappa_grad(*_dims(u.shape), _p(u), _p(lam), _p(g))
    return g


def block_apply(D, L, U, u):
    u = _f64(u)
    y = np.empty_like(u)
    nz, ny, nx, _ = u.shape
    lib().or_block_apply(nx, ny, nz, _p(_f64(D)), _p(_f64(L)), _p(_f64(U)), _p(u), _p(y))
    return y


def block_residual(D, L, U, b, u):
    u = _f64(u)
    b = _f64(b)
    r = np.empty_like(u)
    nz, ny, nx, _ = u.shape
    lib().or_block_residual(nx, ny, nz, _p(_f64(D)), _p(_f64(L)), _p(_f64(U)), _p(b),
                            _p(u), _p(r))
    return r


def block_lower(D, L, omega, r):
    r = _f64(r)
    v = np.empty_like(r)
    nz, ny, nx, _ = r.shape
    lib().or_block_lower(nx, ny, nz, _p(_f64(D)), _p(_f64(L)), float(omega), _p(r), _p(v))
    return v


def block_upper(D, U, omega, v):
    v = _f64(v)
    w = np.empty_like(v)
    nz, ny, nx, _ = v.shape
    lib().or_block_upper(nx, ny, nz, _p(_f64(D)), _p(_f64(U)), float(omega), _p(v), _p(w))
    return w


def ssor(D, L, U, omega, b, u, n_iters):
    b = _f64(b)
    u = _f64(u).copy()
    nz, ny, nx, _ = u.shape
    lib().or_ssor(nx, ny, nz, _p(_f64(D)), _p(_f64(L)), _p(_f64(U)), float(omega),
                  _p(b), _p(u), int(n_iters))
    return u


JAC_PARAMS = 2 + 4 * 55


def block_jac(P, u):
    """(D, L, U) formed from the state u (nz, ny, nx, 5) with the parameters
    P (222 doubles: sigma, nu, then C_k, E_k, g_k for k = 0..3):
    D_p = sigma I + J_0(u_p), L_{p,d} = -nu I - J_{d+1}(u_{p-e_d}) / 2,
    U_{p,d} = -nu I + J_{d+1}(u_{p+e_d}) / 2, J_k the Jacobian of the flux
    F_k(q) = C_k q + (g_k . q) E_k q; couplings off the domain 0."""
    P = _f64(P)
    assert P.shape == (JAC_PARAMS,)
    u = _f64(u)
    nz, ny, nx, _ = u.shape
    D = np.empty((nz, ny, nx, 5, 5))
    L = np.empty((nz, ny, nx, 3, 5, 5))
    U = np.empty((nz, ny, nx, 3, 5, 5))
    lib().or_block_jac(nx, ny, nz, _p(P), _p(u), _p(D), _p(L), _p(U))
    return D, L, U


def ssor_jac(P, omega, b, u, n_iters):
    """n_iters SSOR steps, each with the blocks formed from the u it starts
    from (the NPB-LU situation: Jacobian blocks formed every step)."""
    P = _f64(P)
    assert P.shape == (JAC_PARAMS,)
    b = _f64(b)
    u = _f64(u).copy()
    nz, ny, nx, _ = u.shape
    lib().or_ssor_jac(nx, ny, nz, _p(P), float(omega), _p(b), _p(u), int(n_iters))
    return u

def line_penta(coef, rhs, axis):
    """Solutions of the pentadiagonal systems along the lines of `axis`
    (0 = x, 1 = y, 2 = z): coef (nz, ny, nx, 5) holds (a, b, c, d, e) of
    a v_{i-2} + b v_{i-1} + c v_i + d v_{i+1} + e v_{i+2} = r_i at each point
    (terms outside the line dropped), rhs (nz, ny, nx, k) the k right-hand
    sides (NPB-SP's direct solves, Sec. 1, Sec. 7.2.2)."""
    coef = _f64(coef)
    v = _f64(rhs).copy()
    nz, ny, nx, k = v.shape
    assert coef.shape == (nz, ny, nx, 5)
    lib().or_line_penta(nx, ny, nz, int(axis), _p(coef), _p(v), int(k))
    return v


def line_btri(blk, rhs, axis):
    """Solutions of the 5x5 block-tridiagonal systems along the lines of
    `axis`: blk (nz, ny, nx, 3, 5, 5) = (A, B, C) of
    A v_{i-1} + B v_i + C v_{i+1} = r_i at each point (A of a line's first
    point and C of its last dropped), rhs (nz, ny, nx, 5) (NPB-BT's direct
    solves)."""
    blk = _f64(blk)
    v = _f64(rhs).copy()
    nz, ny, nx, _ = v.shape
    assert blk.shape == (nz, ny, nx, 3, 5, 5) and v.shape[3] == 5
    lib().or_line_btri(nx, ny, nz, int(axis), _p(blk), _p(v))
    return v


def ilu0_factor(shape):
    """ILU(0) of the HPCG 27-point matrix on a grid of `shape` (nz, ny, nx):
    (nz, ny, nx, 27) values per point over the 3x3x3 box offsets
    o = (dz+1)*9 + (dy+1)*3 + (dx+1): o < 13 the unit-lower factor L, o = 13
    the pivot, o > 13 the strict upper part of U; 0 off the domain."""
    nz, ny, nx = shape
    F = np.zeros((nz, ny, nx, 27))
    lib().or_ilu0_factor(nx, ny, nz, _p(F))
    return F


def ilu0_apply(F, r):
    """(LU)^{-1} r with the factors of ilu0_factor."""
    F = _f64(F)
    r = _f64(r)
    z = np.empty_like(r)
    nz, ny, nx = r.shape
    lib().or_ilu0_apply(nx, ny, nz, _p(F), _p(r), _p(z))
    return z
