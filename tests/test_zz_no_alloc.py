"""The allocation-free symmetric Gauss-Seidel entry point.

m2s_symgs_noalloc serves callers that cannot allocate device memory (an
application that owns all device memory in its own pool, or a loop that
cannot pay for cudaMalloc's implicit synchronisation): its scratch is one
fixed array inside the library.  It is the only caller of the single-warp
wavefront kernel, so besides matching m2s_symgs on a grid it is compared
with the oracle directly.  This file is collected last so that a failure
here never hides the results of the other GPU tests; it passes both on its
own in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import m2s_inputs as gen
import oracle

TOL64 = 1e-13
H27 = oracle.HPCG27


def err(g, o, floor=1e-2):
    scale = np.max(np.abs(o))
    den = np.maximum(np.abs(o), floor * scale)
    return float(np.max(np.abs(g - o) / den))


@pytest.fixture(scope="module")
def m():
    from paper_2204_13304_gb300 import build
    build.build()
    import paper_2204_13304_gb300 as m
    m.load()
    return m


def _call(m, nx, ny, nz, dtype, b_ptr, x_ptr, sweeps):
    import torch
    lib = m.load()
    return lib.m2s_symgs_noalloc(nx, ny, nz, int(dtype), ctypes.c_void_p(b_ptr),
                                 ctypes.c_void_p(x_ptr), sweeps,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.gpu
def test_noalloc_matches_grid_symgs_two_calls(m):
    """Two calls in a row through the C ABI, each against m2s_symgs on a grid
    (the existing entry point), within the FP64 parity tolerance."""
    import torch
    for k, shape in enumerate([(40, 33, 37), (64, 64, 64)]):
        nz, ny, nx = shape
        b = torch.from_numpy(gen.random_vector(shape, seed=900 + k)).cuda()
        x0 = torch.from_numpy(gen.random_vector(shape, seed=950 + k)).cuda()
        x_ref = x0.clone()
        g = m.Grid([dict(nx=nx, ny=ny, nz=nz, op=m.Op.HPCG27, mg_levels=1)])
        m.m2s_symgs(g.handle, 0, b, x_ref, 3)
        x = x0.clone()
        st = _call(m, nx, ny, nz, m.DType.F64, b.data_ptr(), x.data_ptr(), 3)
        assert st == m.Status.OK
        torch.cuda.synchronize()
        assert err(x.cpu().numpy(), x_ref.cpu().numpy()) <= TOL64
        g.close()


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 64), (64, 1, 1), (1, 64, 1), (9, 1, 13),
                                   (7, 17, 1), (33, 17, 35), (64, 64, 64), (1, 8, 4096)])
def test_noalloc_matches_oracle_ten_sweeps(m, shape):
    """Ten symmetric sweeps through the C ABI against the oracle, per entry:
    ragged and degenerate shapes (a single point, lines along each axis,
    planes, a tall column).  Workload-shaped data (b = A*ones, x0 = 0) at
    the workload floor 1e-3, and random-sign data at 1e-2, both 1e-13."""
    import torch
    nz, ny, nx = shape
    cases = [(oracle.apply(H27, np.ones(shape)), np.zeros(shape), 1e-3),
             (gen.random_vector(shape, seed=1200), gen.random_vector(shape, seed=1201), 1e-2)]
    for bh, x0, floor in cases:
        b = torch.from_numpy(np.ascontiguousarray(bh)).cuda()
        x = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
        st = _call(m, nx, ny, nz, m.DType.F64, b.data_ptr(), x.data_ptr(), 10)
        assert st == m.Status.OK
        torch.cuda.synchronize()
        o = oracle.symgs(H27, bh, x0, 10)
        assert err(x.cpu().numpy(), o, floor=floor) <= TOL64


@pytest.mark.gpu
def test_noalloc_float32_and_limits(m):
    import torch
    shape = (17, 33, 32)
    nz, ny, nx = shape
    b = torch.from_numpy(gen.random_vector(shape, seed=970)).float().cuda()
    x0 = torch.from_numpy(gen.random_vector(shape, seed=971)).float().cuda()
    x_ref = x0.clone()
    g = m.Grid([dict(nx=nx, ny=ny, nz=nz, op=m.Op.HPCG27, mg_levels=1)])
    m.m2s_symgs(g.handle, 0, b, x_ref, 2)
    x = x0.clone()
    m.m2s_symgs_noalloc(b, x, 2)
    assert err(x.cpu().numpy(), x_ref.cpu().numpy(), floor=1e-1) <= 1e-5
    assert err(x.cpu().numpy(), oracle.symgs_f32(H27, b.cpu().numpy(), x0.cpu().numpy(), 2),
               floor=1e-1) <= 1e-5
    big = torch.zeros((65, 64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(m.M2SError) as ei:
        m.m2s_symgs_noalloc(big.clone(), big, 1)
    assert ei.value.status == m.Status.INVALID_ARG
    g.close()


@pytest.mark.gpu
def test_noalloc_rejects_before_launch(m):
    """Shapes under the point limit whose wavefront has more units than the
    scratch holds (a tall column: 65536 rows of units; a thin 1 x 8 x 32768
    slab: 10922 units), and b overlapping x in part, are rejected with
    INVALID_ARG by the host checks; x is left untouched."""
    import torch
    for nz, ny, nx in [(262144, 1, 1), (32768, 8, 1)]:
        b = torch.zeros(nz * ny * nx, dtype=torch.float64, device="cuda")
        x = torch.ones_like(b)
        st = _call(m, nx, ny, nz, m.DType.F64, b.data_ptr(), x.data_ptr(), 1)
        assert st == m.Status.INVALID_ARG
        torch.cuda.synchronize()
        assert bool((x == 1.0).all())
    buf = torch.ones(2 * 4096, dtype=torch.float64, device="cuda")
    st = _call(m, 16, 16, 16, m.DType.F64, buf.data_ptr(), buf.data_ptr() + 8 * 100, 1)
    assert st == m.Status.INVALID_ARG
    torch.cuda.synchronize()
    assert bool((buf == 1.0).all())


def test_binding_rejects_mismatched_vectors_before_any_call():
    """The binding checks b against x (shape, dtype, device) before any
    pointer reaches the library: runs on the CPU, no library needed."""
    import torch
    import paper_2204_13304_gb300 as m
    x = torch.zeros((4, 5, 6), dtype=torch.float64)
    with pytest.raises(ValueError):
        m.m2s_symgs_noalloc(torch.zeros((4, 5, 5), dtype=torch.float64), x, 1)
    with pytest.raises(ValueError):
        m.m2s_symgs_noalloc(torch.zeros((4, 5, 6), dtype=torch.float32), x, 1)
    with pytest.raises(ValueError):
        m.m2s_symgs_noalloc(torch.zeros(120, dtype=torch.float64), x, 1)
    with pytest.raises(ValueError):
        m.m2s_symgs_noalloc(x, torch.zeros(120, dtype=torch.float64), 1)
    with pytest.raises(ValueError):
        m.m2s_symgs(None, 0, torch.zeros(119, dtype=torch.float64), x, 1)
    with pytest.raises(ValueError):
        m.m2s_pcg_solve(None, torch.zeros(120, dtype=torch.float32), x)
