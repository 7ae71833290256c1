"""GPU parity of the block SSOR step whose 5x5 blocks are formed from the
state every step (op BLOCK7_JAC; the NPB-LU situation of Sec. 1 and Sec.
4.2.3, with a synthetic quadratic flux in place of NPB's): the fused
block-forming pass plus the two block wavefront sweeps, called through the C
ABI, against the serial oracle (`oracle.block_jac`, `oracle.ssor_jac`),
element by element.

Tolerance: FP64, normwise against the scale of the step,
    e = max_i |g_i - o_i| / max(|u0|_inf, |o|_inf) <= 1e-13.
A step from u0 ~ U(0, 1) lands near the solution (|u| ~ 0.1): its residual
b - A(u) u sums terms of size sigma |u0| ~ 10 and cancels them, so its
rounding error is a few ulps of that scale, not of the (much smaller)
entries it produces; a per-entry bound floored at 1e-2 |o|_inf would ask
for ~1e-15 absolute where the arithmetic itself rounds at ~1e-15..1e-14.
The GPU also inverts each diagonal block by Gauss-Jordan and multiplies by
the inverse where the oracle eliminates per solve.  A wrong block, sign or
neighbour changes u by ~1e-4..1e-1 of its scale.  The per-entry error is
reported in the assertion message.
"""
import numpy as np
import pytest

import m2s_inputs as gen
import oracle

pytestmark = pytest.mark.gpu

TOL64 = 1e-13
OMEGA = 1.2


@pytest.fixture(scope="module")
def m():
    from paper_2204_13304_gb300 import build
    build.build()
    import paper_2204_13304_gb300 as m
    m.load()
    return m


def err_step(g, o, u0):
    """(normwise error against max(|u0|_inf, |o|_inf), per-entry error with
    the 1e-2 |o|_inf floor) of a result g against the oracle's o."""
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    d = np.abs(g - o)
    scale = max(float(np.max(np.abs(o))), float(np.max(np.abs(u0))))
    per_entry = float(np.max(d / np.maximum(np.abs(o), 1e-2 * np.max(np.abs(o)))))
    return float(np.max(d)) / scale, per_entry


def check(g, o, u0):
    e, per_entry = err_step(g, o, u0)
    assert e <= TOL64, "normwise %.3g (per entry %.3g)" % (e, per_entry)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.cpu().numpy()


def jac_grid(m, shape, P):
    nz, ny, nx = shape
    return m.Grid([dict(nx=nx, ny=ny, nz=nz, op=m.Op.BLOCK7_JAC, mg_levels=1, jac=P)])


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 3, 1), (7, 1, 9), (2, 4, 3), (9, 10, 12),
                                   (17, 6, 33)])
def test_block_jac_apply_and_ssor(m, shape):
    import torch
    P, b, u0 = gen.block_jac_inputs(shape, seed=71)
    g = jac_grid(m, shape, P)
    y = torch.empty(shape + (5,), dtype=torch.float64, device="cuda")
    m.m2s_spmv(g.handle, 0, dev(u0), y)
    D, L, U = oracle.block_jac(P, u0)
    check(host(y), oracle.block_apply(D, L, U, u0), u0)
    u = dev(u0)
    m.m2s_ssor_sweep(g.handle, dev(b), u, OMEGA, 3)
    m.m2s_grid_sync(g.handle)
    check(host(u), oracle.ssor_jac(P, OMEGA, b, u0, 3), u0)


def test_block_jac_batched_problems_own_parameters(m):
    """Three problems of different shapes and parameters in one handle."""
    shapes = [(9, 12, 7), (6, 17, 5), (4, 4, 4)]
    inputs = [gen.block_jac_inputs(s, seed=80 + i) for i, s in enumerate(shapes)]
    descs = []
    for s, (P, _, _) in zip(shapes, inputs):
        nz, ny, nx = s
        descs.append(dict(nx=nx, ny=ny, nz=nz, op=m.Op.BLOCK7_JAC, mg_levels=1, jac=P))
    g = m.Grid(descs)
    u = dev(np.concatenate([inp[2].ravel() for inp in inputs]))
    bb = dev(np.concatenate([inp[1].ravel() for inp in inputs]))
    m.m2s_ssor_sweep(g.handle, bb, u, OMEGA, 4)
    m.m2s_grid_sync(g.handle)
    uh = host(u)
    off = 0
    for s, (P, b, u0) in zip(shapes, inputs):
        n = int(np.prod(s)) * 5
        check(uh[off:off + n].reshape(s + (5,)), oracle.ssor_jac(P, OMEGA, b, u0, 4), u0)
        off += n


def test_block_jac_steps_converge_to_nonlinear_solution(m):
    """Many steps on the GPU: A(u) u = b at the fixed point, with A(u) u taken
    from the oracle's blocks at the GPU's final u."""
    shape = (8, 9, 10)
    P, b, u0 = gen.block_jac_inputs(shape, seed=90)
    g = jac_grid(m, shape, P)
    u = dev(u0)
    m.m2s_ssor_sweep(g.handle, dev(b), u, OMEGA, 40)
    m.m2s_grid_sync(g.handle)
    uh = host(u)
    D, L, U = oracle.block_jac(P, uh)
    assert np.max(np.abs(b - oracle.block_apply(D, L, U, uh))) <= 1e-12


def test_block_jac_full_size_step(m):
    """One step at 162^3 x 5 (NPB-LU class C), the benchmark's configuration,
    compared with the serial oracle entry by entry (the oracle's blocks of
    that step take 6 GB of host memory and a few seconds)."""
    shape = (162, 162, 162)
    P, b, u0 = gen.block_jac_inputs(shape, seed=gen.BASE_SEED)
    g = jac_grid(m, shape, P)
    u = dev(u0)
    m.m2s_ssor_sweep(g.handle, dev(b), u, OMEGA, 1)
    m.m2s_grid_sync(g.handle)
    got = host(u)
    g.close()
    check(got, oracle.ssor_jac(P, OMEGA, b, u0, 1), u0)
