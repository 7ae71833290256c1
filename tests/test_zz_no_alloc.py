"""The allocation-free symmetric Gauss-Seidel entry point.

m2s_symgs_noalloc serves callers that cannot allocate device memory (an
application that owns all device memory in its own pool, or a loop that
cannot pay for cudaMalloc's implicit synchronisation): its scratch is one
fixed array inside the library.  This file is collected last so that a
failure here never hides the results of the other GPU tests; it passes both
on its own in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import m2s_inputs as gen

pytestmark = pytest.mark.gpu

TOL64 = 1e-13


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


def test_noalloc_matches_grid_symgs_two_calls(m):
    """Two calls in a row through the C ABI, each against m2s_symgs on a grid
    (the existing entry point), within the FP64 parity tolerance."""
    import torch
    lib = m.load()
    for k, shape in enumerate([(40, 33, 37), (64, 64, 64)]):
        nz, ny, nx = shape
        b = torch.from_numpy(gen.random_vector(shape, seed=900 + k)).cuda()
        x0 = torch.from_numpy(gen.random_vector(shape, seed=950 + k)).cuda()
        x_ref = x0.clone()
        g = m.Grid([dict(nx=nx, ny=ny, nz=nz, op=m.Op.HPCG27, mg_levels=1)])
        m.m2s_symgs(g.handle, 0, b, x_ref, 3)
        x = x0.clone()
        st = lib.m2s_symgs_noalloc(nx, ny, nz, int(m.DType.F64), ctypes.c_void_p(b.data_ptr()),
                                   ctypes.c_void_p(x.data_ptr()), 3,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == m.Status.OK
        torch.cuda.synchronize()
        assert err(x.cpu().numpy(), x_ref.cpu().numpy()) <= TOL64
        g.close()


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
    big = torch.zeros((65, 64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(m.M2SError) as ei:
        m.m2s_symgs_noalloc(big.clone(), big, 1)
    assert ei.value.status == m.Status.INVALID_ARG
    g.close()
