"""CPU pins of the sampled sweep check (tests/sweep_defect.py) used by the
full-size GPU tests: the oracle's exact lexicographic sweeps satisfy it to
rounding at every point, and sweeps that are not the lexicographic
Gauss-Seidel sweep of Sec. 4.3.3 (a multicolour ordering, a Jacobi update,
the other direction) fail it by orders of magnitude."""
import numpy as np
import pytest

import m2s_inputs as gen
import oracle
from sweep_defect import sample_points, sweep_defect_numpy

H27 = oracle.HPCG27
SHAPES = [(3, 4, 5), (5, 3, 4), (7, 9, 6), (12, 5, 17)]


def every_point(shape):
    return np.arange(int(np.prod(shape)), dtype=np.int64)


def inputs(shape, k):
    b = gen.random_vector(shape, seed=gen.BASE_SEED + 700 + k)
    x0 = gen.random_vector(shape, seed=gen.BASE_SEED + 750 + k)
    return b, x0


@pytest.mark.parametrize("shape", SHAPES)
def test_oracle_sweeps_satisfy_the_identity(shape):
    b, x0 = inputs(shape, 0)
    xf = oracle.gs_forward(H27, b, x0)
    xb = oracle.gs_backward(H27, b, x0)
    pts = every_point(shape)
    assert sweep_defect_numpy(b, x0, xf, pts) <= 1e-14
    assert sweep_defect_numpy(b, x0, xb, pts, backward=True) <= 1e-14


@pytest.mark.parametrize("shape", SHAPES)
def test_other_sweeps_fail_the_identity(shape):
    b, x0 = inputs(shape, 1)
    pts = every_point(shape)
    # multicolour ordering (the negative control of the oracle)
    xm = oracle.gs_multicolor_forward(H27, b, x0)
    assert sweep_defect_numpy(b, x0, xm, pts) > 1e-3
    # Jacobi: every neighbour old
    xj = x0 + (b - oracle.apply(H27, x0)) / 26.0
    assert sweep_defect_numpy(b, x0, xj, pts) > 1e-3
    # a forward sweep is not a backward one
    xf = oracle.gs_forward(H27, b, x0)
    assert sweep_defect_numpy(b, x0, xf, pts, backward=True) > 1e-3


def test_sampling_includes_corners_and_is_seeded():
    shape = (9, 8, 7)
    a = sample_points(shape, 50, 3)
    assert np.array_equal(a, sample_points(shape, 50, 3))
    n = 9 * 8 * 7
    assert 0 in a and n - 1 in a and (8 * 8 + 7) * 7 + 0 in a
    assert a.min() >= 0 and a.max() < n


def test_kappa_oracle_sweeps_satisfy_the_identity():
    from sweep_defect import kappa_defect_numpy
    K7 = oracle.KAPPA7
    for shape in [(3, 4, 5), (7, 9, 6)]:
        kap = np.exp(gen.random_vector(shape, seed=gen.BASE_SEED + 760))
        b, x0 = inputs(shape, 2)
        pts = every_point(shape)
        assert kappa_defect_numpy(kap, b, x0, oracle.gs_forward(K7, b, x0, kap), pts) <= 1e-14
        assert kappa_defect_numpy(kap, b, x0, oracle.gs_backward(K7, b, x0, kap), pts,
                                  backward=True) <= 1e-14
        # a Jacobi update, the wrong direction and the 27-point sweep fail it
        xj = x0 + (b - oracle.apply(K7, x0, kap)) / kap_diag(kap)
        assert kappa_defect_numpy(kap, b, x0, xj, pts) > 1e-3
        assert kappa_defect_numpy(kap, b, x0, oracle.gs_forward(K7, b, x0, kap), pts,
                                  backward=True) > 1e-3
        assert kappa_defect_numpy(kap, b, x0, oracle.gs_forward(H27, b, x0), pts) > 1e-3


def kap_diag(kap):
    """a_pp of the 7-point operator by its definition (sum of the six face
    coefficients, boundary faces at kappa_p), independently of the oracle."""
    nz, ny, nx = kap.shape
    d = np.zeros_like(kap)
    for axis in range(3):
        for s in (-1, 1):
            nb = np.roll(kap, -s, axis=axis)
            face = 0.5 * (kap + nb)
            idx = [slice(None)] * 3
            idx[axis] = -1 if s == 1 else 0
            face[tuple(idx)] = kap[tuple(idx)]
            d += face
    return d
