"""Python binding of the m2s C ABI (include/m2s.h).

Thin marshalling only: every function below forwards device pointers, sizes
and the current CUDA stream of PyTorch to the function of the same name in
``_build/libm2s.so`` (``_build_bounds/libm2s.so``, the range-checked variant,
when M2S_BUILD_VARIANT=bounds is set at import); all computation happens in
that library's CUDA kernels.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the
library has not been built (``paper_2204_13304_gb300.build.build()``) the
first call raises.

Vectors are contiguous CUDA tensors of shape (nz, ny, nx) (or (nz, ny, nx, 5)
for the block operator), FP64 or FP32; batches are packed back to back.
"""
import ctypes
import enum
import os

from . import build as _build_mod

_LIB = None


class Status(enum.IntEnum):
    OK = 0
    INVALID_ARG = 1
    CUDA = 2
    OOM = 3
    TIMEOUT = 4
    NOT_CONVERGED = 5
    BREAKDOWN = 6


class Op(enum.IntEnum):
    HPCG27 = 0
    DIFF7_KAPPA = 1
    BLOCK7_5x5 = 2
    BLOCK7_JAC = 3


JAC_PARAMS = 2 + 4 * 55  # sigma, nu, (C_k, E_k, g_k) for k = 0..3


class DType(enum.IntEnum):
    F64 = 0
    F32 = 1


FORWARD = 0
BACKWARD = 1


class M2SError(RuntimeError):
    def __init__(self, status, where):
        self.status = Status(status)
        super().__init__("%s: %s" % (where, status_string(status)))


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("op", ctypes.c_int), ("mg_levels", ctypes.c_int),
                ("precond_dtype", ctypes.c_int), ("kappa", ctypes.c_void_p),
                ("D", ctypes.c_void_p), ("L", ctypes.c_void_p), ("U", ctypes.c_void_p),
                ("jac", ctypes.c_void_p)]


class PcgOpts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("rtol", ctypes.c_double),
                ("fixed_iters", ctypes.c_int), ("check_every", ctypes.c_int)]


class PcgResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_resid", ctypes.c_double),
                ("resid_hist_last", ctypes.c_double)]


EXPORTS = (
    "m2s_grid_create", "m2s_grid_destroy", "m2s_grid_sync", "m2s_grid_points", "m2s_spmv",
    "m2s_symgs", "m2s_gs_sweep", "m2s_mg_restrict", "m2s_mg_prolong", "m2s_mg_vcycle",
    "m2s_pcg_solve", "m2s_ssor_sweep", "m2s_adjoint_solve", "m2s_kappa_grad",
    "m2s_set_spin_limit", "m2s_debug_stall_unit", "m2s_symgs_noalloc", "m2s_status_string",
    "m2s_sweep_timing", "m2s_sweep_timing_read", "m2s_set_sweep_warps", "m2s_sweep_warps",
    "m2s_set_graphs",
    "m2s_autotune_sweeps", "m2s_line_penta", "m2s_line_penta_work_bytes", "m2s_line_btri",
    "m2s_line_btri_work_bytes", "m2s_ilu0_setup", "m2s_ilu0_apply",
    "m2s_ilu0_factors", "m2s_debug_bounds_read",
)


def lib_path():
    return _build_mod.LIB


def load():
    """Load libm2s.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libm2s.so is not built (%s); run paper_2204_13304_gb300.build.build()"
                           % path)
    L = ctypes.CDLL(path)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "m2s_grid_create": ([ctypes.POINTER(GridDesc), i, vp, ctypes.POINTER(vp)], i),
        "m2s_grid_destroy": ([vp], i),
        "m2s_grid_sync": ([vp, vp], i),
        "m2s_grid_points": ([vp, i, i], ll),
        "m2s_spmv": ([vp, i, i, vp, vp, vp], i),
        "m2s_symgs": ([vp, i, i, vp, vp, i, vp], i),
        "m2s_gs_sweep": ([vp, i, i, vp, vp, i, vp], i),
        "m2s_mg_restrict": ([vp, i, i, vp, vp, vp, vp], i),
        "m2s_mg_prolong": ([vp, i, i, vp, vp, vp], i),
        "m2s_mg_vcycle": ([vp, i, vp, vp, vp], i),
        "m2s_pcg_solve": ([vp, vp, vp, ctypes.POINTER(PcgOpts), ctypes.POINTER(PcgResult), vp], i),
        "m2s_ssor_sweep": ([vp, vp, vp, d, i, vp], i),
        "m2s_adjoint_solve": ([vp, vp, vp, vp, vp, ctypes.POINTER(PcgOpts),
                               ctypes.POINTER(PcgResult), vp], i),
        "m2s_kappa_grad": ([vp, vp, vp, vp, vp], i),
        "m2s_set_spin_limit": ([vp, ll], i),
        "m2s_debug_stall_unit": ([vp, i, i], i),
        "m2s_symgs_noalloc": ([i, i, i, i, vp, vp, i, vp], i),
        "m2s_status_string": ([i], ctypes.c_char_p),
        "m2s_sweep_timing": ([vp, i], i),
        "m2s_set_sweep_warps": ([vp, i, i], i),
        "m2s_sweep_warps": ([vp, i, ctypes.POINTER(i), ctypes.POINTER(i)], i),
        "m2s_set_graphs": ([vp, i], i),
        "m2s_autotune_sweeps": ([vp, i, vp, ctypes.POINTER(i)], i),
        "m2s_sweep_timing_read": ([vp, i, ctypes.POINTER(i), ctypes.POINTER(d),
                                   ctypes.POINTER(i)], i),
        "m2s_line_penta_work_bytes": ([i, i, i], ll),
        "m2s_line_penta": ([i, i, i, i, vp, vp, i, vp, ll, vp], i),
        "m2s_line_btri_work_bytes": ([i, i, i], ll),
        "m2s_line_btri": ([i, i, i, i, vp, vp, vp, ll, vp], i),
        "m2s_ilu0_setup": ([vp, vp], i),
        "m2s_ilu0_apply": ([vp, vp, vp, vp], i),
        "m2s_ilu0_factors": ([vp, vp, vp], i),
        "m2s_debug_bounds_read": ([ctypes.POINTER(ll)], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _LIB = L
    return L


def status_string(status):
    return load().m2s_status_string(int(status)).decode()


def m2s_status_string(status):
    return status_string(status)


def _check(status, where):
    if status != 0:
        raise M2SError(status, where)
    return status


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t, what):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % what)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    return t.data_ptr()


def _same(what, ref, *others, exact_shape=False):
    """Raise ValueError unless every tensor of `others` has the element count
    (the shape, if exact_shape), dtype and device of `ref`: checked before any
    pointer reaches the library, which cannot see the extent of a device
    allocation."""
    import torch
    if not isinstance(ref, torch.Tensor):
        raise TypeError("%s: vectors must be torch.Tensors" % what)
    for name, t in others:
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s: %s must be a torch.Tensor" % (what, name))
        size_ok = t.shape == ref.shape if exact_shape else t.numel() == ref.numel()
        if not size_ok or t.dtype != ref.dtype or t.device != ref.device:
            raise ValueError("%s: %s must match %s in shape, dtype and device "
                             "(%s %s %s vs %s %s %s)"
                             % (what, name, "the first vector", tuple(t.shape), t.dtype,
                                t.device, tuple(ref.shape), ref.dtype, ref.device))


def _dtype(t):
    import torch
    if t.dtype == torch.float64:
        return DType.F64
    if t.dtype == torch.float32:
        return DType.F32
    raise TypeError("unsupported dtype %s" % t.dtype)


def m2s_grid_create(descs, stream=None):
    """descs: list of GridDesc (or dicts with its fields; tensors for kappa/D/L/U;
    for op BLOCK7_JAC, `jac` the 222 host parameters, any FP64 array-like)."""
    arr = (GridDesc * len(descs))()
    keep = []  # host parameter buffers, alive until the library has copied them
    for k, d in enumerate(descs):
        if isinstance(d, GridDesc):
            arr[k] = d
            continue
        g = GridDesc()
        g.nx, g.ny, g.nz = int(d["nx"]), int(d["ny"]), int(d["nz"])
        g.op = int(d.get("op", Op.HPCG27))
        g.mg_levels = int(d.get("mg_levels", 1))
        g.precond_dtype = int(d.get("precond_dtype", DType.F64))
        for f in ("kappa", "D", "L", "U"):
            v = d.get(f)
            setattr(g, f, _ptr(v, f) if v is not None else None)
        if d.get("jac") is not None:
            if len(d["jac"]) != JAC_PARAMS:
                raise ValueError("jac needs %d parameters" % JAC_PARAMS)
            P = (ctypes.c_double * JAC_PARAMS)(*[float(t) for t in d["jac"]])
            keep.append(P)
            g.jac = ctypes.cast(P, ctypes.c_void_p)
        arr[k] = g
    h = ctypes.c_void_p()
    _check(load().m2s_grid_create(arr, len(descs), _stream(stream), ctypes.byref(h)),
           "m2s_grid_create")
    return h


def m2s_grid_destroy(grid):
    return _check(load().m2s_grid_destroy(grid), "m2s_grid_destroy")


def m2s_grid_sync(grid, stream=None):
    return _check(load().m2s_grid_sync(grid, _stream(stream)), "m2s_grid_sync")


def m2s_grid_points(grid, problem=0, level=0):
    return load().m2s_grid_points(grid, problem, level)


def m2s_set_spin_limit(grid, limit_ns):
    return _check(load().m2s_set_spin_limit(grid, int(limit_ns)), "m2s_set_spin_limit")


def m2s_debug_stall_unit(grid, level, unit):
    return _check(load().m2s_debug_stall_unit(grid, int(level), int(unit)), "m2s_debug_stall_unit")


def m2s_sweep_warps(grid, level):
    """(FP64, FP32) warps per unit of the 27-point sweeps of `level`."""
    w64, w32 = ctypes.c_int(), ctypes.c_int()
    _check(load().m2s_sweep_warps(grid, int(level), ctypes.byref(w64), ctypes.byref(w32)),
           "m2s_sweep_warps")
    return w64.value, w32.value


def m2s_set_sweep_warps(grid, level, warps):
    """Warps (4 or 8) per 27-point sweep unit on `level` (-1: all levels)."""
    return _check(load().m2s_set_sweep_warps(grid, int(level), int(warps)), "m2s_set_sweep_warps")


def m2s_autotune_sweeps(grid, levels, reps=3, stream=None):
    """Time 4- and 8-warp sweep units on every level and keep the faster;
    returns [(warps FP64, warps FP32) per level]."""
    out = (ctypes.c_int * (2 * levels))()
    _check(load().m2s_autotune_sweeps(grid, int(reps), _stream(stream), out),
           "m2s_autotune_sweeps")
    return [(out[2 * l], out[2 * l + 1]) for l in range(levels)]


def m2s_set_graphs(grid, enable=True):
    """CUDA-graph replay of the PCG iteration on (default) or off."""
    return _check(load().m2s_set_graphs(grid, 1 if enable else 0), "m2s_set_graphs")


def m2s_sweep_timing(grid, enable=True):
    """Start (clearing the counters) or stop per-launch event timing of the
    grid's Gauss-Seidel sweep kernels."""
    return _check(load().m2s_sweep_timing(grid, 1 if enable else 0), "m2s_sweep_timing")


def m2s_sweep_timing_read(grid, level):
    """(recorded launches, summed device ms, dropped launches) of `level`."""
    n, ms, dr = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    _check(load().m2s_sweep_timing_read(grid, int(level), ctypes.byref(n), ctypes.byref(ms),
                                        ctypes.byref(dr)), "m2s_sweep_timing_read")
    return n.value, ms.value, dr.value


def m2s_symgs_noalloc(b, x, n_sym_sweeps=1, stream=None):
    """Symmetric Gauss-Seidel (27-point operator) that allocates no device
    memory, for callers that cannot allocate (its scratch is a fixed static
    array of the library: at most 64^3 points; calls must not overlap).
    b and x are (nz, ny, nx) CUDA tensors of one dtype on one device."""
    import torch
    if not isinstance(x, torch.Tensor) or x.dim() != 3:
        raise ValueError("m2s_symgs_noalloc: x must be a (nz, ny, nx) tensor")
    _same("m2s_symgs_noalloc", x, ("b", b), exact_shape=True)
    nz, ny, nx = x.shape
    return _check(load().m2s_symgs_noalloc(nx, ny, nz, _dtype(x), _ptr(b, "b"), _ptr(x, "x"),
                                           int(n_sym_sweeps), _stream(stream)),
                  "m2s_symgs_noalloc")


def m2s_spmv(grid, level, x, y, stream=None):
    _same("m2s_spmv", x, ("y", y))
    return _check(load().m2s_spmv(grid, level, _dtype(x), _ptr(x, "x"), _ptr(y, "y"),
                                  _stream(stream)), "m2s_spmv")


def m2s_symgs(grid, level, b, x, n_sym_sweeps=1, stream=None):
    _same("m2s_symgs", x, ("b", b))
    return _check(load().m2s_symgs(grid, level, _dtype(x), _ptr(b, "b"), _ptr(x, "x"),
                                   int(n_sym_sweeps), _stream(stream)), "m2s_symgs")


def m2s_gs_sweep(grid, level, b, x, direction=FORWARD, stream=None):
    _same("m2s_gs_sweep", x, ("b", b))
    return _check(load().m2s_gs_sweep(grid, level, _dtype(x), _ptr(b, "b"), _ptr(x, "x"),
                                      int(direction), _stream(stream)), "m2s_gs_sweep")


def m2s_mg_restrict(grid, level, r, z, rc, stream=None):
    _same("m2s_mg_restrict", r, ("z", z))
    if rc.dtype != r.dtype or rc.device != r.device:
        raise ValueError("m2s_mg_restrict: rc must match r in dtype and device")
    return _check(load().m2s_mg_restrict(grid, level, _dtype(r), _ptr(r, "r"), _ptr(z, "z"),
                                         _ptr(rc, "rc"), _stream(stream)), "m2s_mg_restrict")


def m2s_mg_prolong(grid, level, zc, z, stream=None):
    if zc.dtype != z.dtype or zc.device != z.device:
        raise ValueError("m2s_mg_prolong: zc must match z in dtype and device")
    return _check(load().m2s_mg_prolong(grid, level, _dtype(z), _ptr(zc, "zc"), _ptr(z, "z"),
                                        _stream(stream)), "m2s_mg_prolong")


def m2s_mg_vcycle(grid, r, z, stream=None):
    _same("m2s_mg_vcycle", r, ("z", z))
    return _check(load().m2s_mg_vcycle(grid, _dtype(r), _ptr(r, "r"), _ptr(z, "z"),
                                       _stream(stream)), "m2s_mg_vcycle")


def _opts(max_iters, rtol, fixed_iters, check_every):
    o = PcgOpts()
    o.max_iters, o.rtol = int(max_iters), float(rtol)
    o.fixed_iters, o.check_every = int(bool(fixed_iters)), int(check_every)
    return o


def m2s_pcg_solve(grid, b, x, max_iters=50, rtol=0.0, fixed_iters=True, check_every=1,
                  stream=None, raise_on_error=True):
    """Returns (status, PcgResult).  Raises on errors other than NOT_CONVERGED
    unless raise_on_error is False."""
    _same("m2s_pcg_solve", b, ("x", x))
    o = _opts(max_iters, rtol, fixed_iters, check_every)
    res = PcgResult()
    st = load().m2s_pcg_solve(grid, _ptr(b, "b"), _ptr(x, "x"), ctypes.byref(o),
                              ctypes.byref(res), _stream(stream))
    if raise_on_error and st not in (Status.OK, Status.NOT_CONVERGED):
        raise M2SError(st, "m2s_pcg_solve")
    return Status(st), res


def m2s_line_penta_work_bytes(nx, ny, nz):
    return int(load().m2s_line_penta_work_bytes(int(nx), int(ny), int(nz)))


def m2s_line_penta(coef, rhs, axis, work=None, stream=None):
    """Pentadiagonal solves along the lines of `axis` (0 = x, 1 = y, 2 = z):
    coef (nz, ny, nx, 5) FP64 CUDA tensor of (a, b, c, d, e) per point, rhs
    (nz, ny, nx, k) FP64 CUDA tensor, overwritten with the solutions.  work:
    a CUDA tensor of at least m2s_line_penta_work_bytes bytes, or None (a
    scratch tensor is made with torch)."""
    nz, ny, nx, k = rhs.shape
    if tuple(coef.shape) != (nz, ny, nx, 5):
        raise M2SError(Status.INVALID_ARG, "m2s_line_penta: coef shape")
    need = m2s_line_penta_work_bytes(nx, ny, nz)
    if work is None:
        import torch
        work = torch.empty(need // 8, dtype=torch.float64, device=rhs.device)
    nbytes = work.numel() * work.element_size()
    return _check(load().m2s_line_penta(nx, ny, nz, int(axis), _ptr(coef, "coef"),
                                        _ptr(rhs, "rhs"), int(k), _ptr(work, "work"), nbytes,
                                        _stream(stream)), "m2s_line_penta")


def m2s_ilu0_setup(grid, stream=None):
    return _check(load().m2s_ilu0_setup(grid, _stream(stream)), "m2s_ilu0_setup")


def m2s_ilu0_factors(grid, out, stream=None):
    return _check(load().m2s_ilu0_factors(grid, _ptr(out, "out"), _stream(stream)),
                  "m2s_ilu0_factors")


def m2s_debug_bounds_read():
    """(violations, first line, first index, translation unit) of the range
    checks of the bounds variant of the library, cleared by the read;
    violations = -1 when the loaded library was built without them."""
    out = (ctypes.c_longlong * 4)()
    _check(load().m2s_debug_bounds_read(out), "m2s_debug_bounds_read")
    return tuple(int(v) for v in out)


def m2s_ilu0_apply(grid, r, z, stream=None):
    _same("m2s_ilu0_apply", r, ("z", z))
    return _check(load().m2s_ilu0_apply(grid, _ptr(r, "r"), _ptr(z, "z"), _stream(stream)),
                  "m2s_ilu0_apply")


def m2s_line_btri_work_bytes(nx, ny, nz):
    return int(load().m2s_line_btri_work_bytes(int(nx), int(ny), int(nz)))


def m2s_line_btri(blk, rhs, axis, work=None, stream=None):
    """5x5 block-tridiagonal solves along the lines of `axis`: blk
    (nz, ny, nx, 3, 5, 5) FP64 CUDA tensor of (A, B, C) per point, rhs
    (nz, ny, nx, 5) FP64 CUDA tensor, overwritten with the solutions.  work:
    a CUDA tensor of at least m2s_line_btri_work_bytes bytes, or None."""
    nz, ny, nx, five = rhs.shape
    if five != 5 or tuple(blk.shape) != (nz, ny, nx, 3, 5, 5):
        raise M2SError(Status.INVALID_ARG, "m2s_line_btri: shapes")
    need = m2s_line_btri_work_bytes(nx, ny, nz)
    if work is None:
        import torch
        work = torch.empty(need // 8, dtype=torch.float64, device=rhs.device)
    nbytes = work.numel() * work.element_size()
    return _check(load().m2s_line_btri(nx, ny, nz, int(axis), _ptr(blk, "blk"), _ptr(rhs, "rhs"),
                                       _ptr(work, "work"), nbytes, _stream(stream)),
                  "m2s_line_btri")


def m2s_ssor_sweep(grid, b, u, omega=1.2, n_iters=1, stream=None):
    _same("m2s_ssor_sweep", u, ("b", b))
    return _check(load().m2s_ssor_sweep(grid, _ptr(b, "b"), _ptr(u, "u"), float(omega),
                                        int(n_iters), _stream(stream)), "m2s_ssor_sweep")


def m2s_kappa_grad(grid, u, lam, dLdkappa, stream=None):
    _same("m2s_kappa_grad", u, ("lambda", lam), ("dLdkappa", dLdkappa))
    return _check(load().m2s_kappa_grad(grid, _ptr(u, "u"), _ptr(lam, "lambda"),
                                        _ptr(dLdkappa, "dLdkappa"), _stream(stream)),
                  "m2s_kappa_grad")


def m2s_adjoint_solve(grid, u, dLdu, lam, dLdkappa, max_iters=200, rtol=1e-10,
                      fixed_iters=False, check_every=1, stream=None, raise_on_error=True):
    _same("m2s_adjoint_solve", u, ("dLdu", dLdu), ("lambda", lam), ("dLdkappa", dLdkappa))
    o = _opts(max_iters, rtol, fixed_iters, check_every)
    res = PcgResult()
    st = load().m2s_adjoint_solve(grid, _ptr(u, "u"), _ptr(dLdu, "dLdu"), _ptr(lam, "lambda"),
                                  _ptr(dLdkappa, "dLdkappa"), ctypes.byref(o),
                                  ctypes.byref(res), _stream(stream))
    if raise_on_error and st not in (Status.OK, Status.NOT_CONVERGED):
        raise M2SError(st, "m2s_adjoint_solve")
    return Status(st), res


class Grid:
    """Owning wrapper of an m2s grid handle (destroyed on close/__del__)."""

    def __init__(self, descs, stream=None):
        self._keep = descs  # keep coefficient tensors alive until created
        self.handle = m2s_grid_create(descs, stream)
        self._keep = None

    def close(self):
        if self.handle is not None and self.handle.value:
            m2s_grid_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_solve_function():
    import torch

    class KappaSolve(torch.autograd.Function):
        """u = A(kappa)^-1 b by FP64 MG-PCG; backward = the hand-written
        adjoint (A^T lambda = dL/du, then the dL/dkappa stencil)."""

        @staticmethod
        def forward(ctx, kappa, b, mg_levels, rtol, max_iters):
            nz, ny, nx = kappa.shape
            g = Grid([dict(nx=nx, ny=ny, nz=nz, op=Op.DIFF7_KAPPA, mg_levels=mg_levels,
                           kappa=kappa.contiguous())])
            u = torch.empty_like(b)
            st, res = m2s_pcg_solve(g.handle, b.contiguous(), u, max_iters=max_iters,
                                    rtol=rtol, fixed_iters=False)
            if st != Status.OK:
                raise M2SError(st, "forward solve")
            ctx.grid = g
            ctx.opts = (rtol, max_iters)
            ctx.save_for_backward(u)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            (u,) = ctx.saved_tensors
            g = ctx.grid
            lam = torch.empty_like(u)
            dk = torch.empty_like(u)
            rtol, max_iters = ctx.opts
            st, _ = m2s_adjoint_solve(g.handle, u, grad_u.contiguous(), lam, dk,
                                      max_iters=max_iters, rtol=rtol)
            if st != Status.OK:
                raise M2SError(st, "adjoint solve")
            g.close()
            return dk, None, None, None, None

    return KappaSolve


_SOLVE = None


def pcg_solve(kappa, b, mg_levels=4, rtol=1e-10, max_iters=500):
    """Differentiable u = A(kappa)^-1 b (variable-kappa 7-point operator)."""
    global _SOLVE
    if _SOLVE is None:
        _SOLVE = _make_solve_function()
    return _SOLVE.apply(kappa, b, mg_levels, rtol, max_iters)
