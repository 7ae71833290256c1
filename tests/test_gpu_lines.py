"""GPU parity of the NPB-SP-shaped line solves (pentadiagonal systems along
the lines of one axis; Sec. 1, Sec. 7.2.2) through the C ABI.

Against the oracle, element by element: the systems are strictly diagonally
dominant (|c| >= 3 > |a| + |b| + |d| + |e|), so elimination without
pivoting is stable and the GPU (reciprocal multiplications, fused
multiply-adds) and the oracle (divisions, separate products) differ by a
few ulps per operation that do not grow along a line: 1e-13 per entry
against max(|o_i|, 1e-2 |o|_inf).

At 162^3 (NPB class C, k = 5: the benchmark's launch configuration) the
oracle is not re-run; every sampled point must satisfy its equation
a v[i-2] + b v[i-1] + c v[i] + d v[i+1] + e v[i+2] = r[i] to 1e-13 of the
sum of the magnitudes of its terms.
"""
import numpy as np
import pytest

import m2s_inputs as gen
import oracle

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (2, 1, 3), (3, 4, 5), (5, 3, 4), (13, 17, 19), (40, 3, 2), (2, 70, 33)]


@pytest.fixture(scope="module")
def m():
    from paper_2204_13304_gb300 import build
    build.build()
    import paper_2204_13304_gb300 as m
    m.load()
    return m


def err(g, o, floor=1e-2):
    scale = np.max(np.abs(o))
    den = np.maximum(np.abs(o), floor * scale)
    return float(np.max(np.abs(g - o) / den))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 5, 8])
def test_line_penta_matches_oracle(m, shape, axis, k):
    import torch
    coef, rhs = gen.line_penta_inputs(shape, k=k, seed=gen.BASE_SEED + 41 + k)
    want = oracle.line_penta(coef, rhs, axis)
    c = torch.from_numpy(coef).cuda()
    r = torch.from_numpy(rhs).cuda()
    m.m2s_line_penta(c, r, axis)
    torch.cuda.synchronize()
    assert err(r.cpu().numpy(), want) <= 1e-13


def test_line_penta_three_axes_in_turn(m):
    """x, then y, then z solves on the same right-hand sides (the order of
    NPB-SP's x_solve, y_solve, z_solve), with one work buffer."""
    import torch
    shape = (9, 11, 13)
    coefs = [gen.line_penta_inputs(shape, k=5, seed=gen.BASE_SEED + 60 + a)[0] for a in range(3)]
    _, rhs = gen.line_penta_inputs(shape, k=5, seed=gen.BASE_SEED + 63)
    want = rhs
    for a in range(3):
        want = oracle.line_penta(coefs[a], want, a)
    r = torch.from_numpy(rhs).cuda()
    work = torch.empty(m.m2s_line_penta_work_bytes(13, 11, 9) // 8, dtype=torch.float64,
                       device="cuda")
    for a in range(3):
        m.m2s_line_penta(torch.from_numpy(coefs[a]).cuda(), r, a, work=work)
    torch.cuda.synchronize()
    assert err(r.cpu().numpy(), want) <= 1e-13


@pytest.fixture(scope="module")
def inputs_162():
    import torch
    coef, rhs = gen.line_penta_inputs((162, 162, 162), k=5, seed=gen.BASE_SEED + 70)
    return torch.from_numpy(coef).cuda(), torch.from_numpy(rhs).cuda()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_line_penta_162_sampled_equations(m, inputs_162, axis):
    import torch
    n, k = 162, 5
    c, r0 = inputs_162
    v = r0.clone()
    m.m2s_line_penta(c, v, axis)
    torch.cuda.synchronize()
    rng = np.random.default_rng(71 + axis)
    pts = rng.integers(0, n ** 3, size=100000)
    z, y, x = pts // (n * n), (pts // n) % n, pts % n
    pos = (x, y, z)[axis]
    stride = (1, n, n * n)[axis]
    vf = v.reshape(-1, k)
    cf = c.reshape(-1, 5)
    rf = r0.reshape(-1, k)
    P = torch.from_numpy(pts).cuda()
    res = -rf[P].clone()
    mag = rf[P].abs().clone()
    for j, off in enumerate((-2, -1, 0, 1, 2)):
        ok = torch.from_numpy((pos + off >= 0) & (pos + off < n)).cuda()
        q = torch.where(ok, P + off * stride, P)
        term = cf[P, j].unsqueeze(1) * vf[q] * ok.unsqueeze(1)
        res += term
        mag += term.abs()
    assert float((res.abs() / mag).max()) <= 1e-13


# ---------------------------------------------------------------------------
# NPB-BT-shaped 5x5 block-tridiagonal line solves.  The blocks are strictly
# diagonally dominant (|B_jj| >= 9 > 6.5 >= the off-diagonal row sums), so
# block elimination without pivoting is stable and the GPU (reciprocal
# multiplications, fused multiply-adds, block order) and the oracle (scalar
# banded elimination, divisions) agree to a few ulps: 1e-13 per entry
# against max(|o_i|, 1e-2 |o|_inf).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_line_btri_matches_oracle(m, shape, axis):
    import torch
    blk, rhs = gen.line_btri_inputs(shape, seed=gen.BASE_SEED + 80)
    want = oracle.line_btri(blk, rhs, axis)
    b = torch.from_numpy(blk).cuda()
    r = torch.from_numpy(rhs).cuda()
    m.m2s_line_btri(b, r, axis)
    torch.cuda.synchronize()
    assert err(r.cpu().numpy(), want) <= 1e-13


@pytest.fixture(scope="module")
def btri_162():
    import torch
    blk, rhs = gen.line_btri_inputs((162, 162, 162), seed=gen.BASE_SEED + 81)
    return torch.from_numpy(blk).cuda(), torch.from_numpy(rhs).cuda()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_line_btri_162_sampled_equations(m, btri_162, axis):
    """Every sampled point satisfies A v[i-1] + B v[i] + C v[i+1] = r[i]
    (5 rows) to 1e-13 of the sum of the magnitudes of its terms."""
    import torch
    n = 162
    b, r0 = btri_162
    v = r0.clone()
    m.m2s_line_btri(b, v, axis)
    torch.cuda.synchronize()
    rng = np.random.default_rng(82 + axis)
    pts = rng.integers(0, n ** 3, size=50000)
    z, y, x = pts // (n * n), (pts // n) % n, pts % n
    pos = (x, y, z)[axis]
    stride = (1, n, n * n)[axis]
    vf = v.reshape(-1, 5)
    bf = b.reshape(-1, 3, 5, 5)
    P = torch.from_numpy(pts).cuda()
    res = -r0.reshape(-1, 5)[P].clone()
    mag = res.abs().clone()
    for j, off in enumerate((-1, 0, 1)):
        ok = torch.from_numpy((pos + off >= 0) & (pos + off < n)).cuda()
        q = torch.where(ok, P + off * stride, P)
        terms = bf[P, j] * vf[q].unsqueeze(1) * ok.view(-1, 1, 1)
        res += terms.sum(-1)
        mag += terms.abs().sum(-1)
    assert float((res.abs() / mag).max()) <= 1e-13
