"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module draws random numbers and shapes fields; it holds none of the
solver's arithmetic (no operator, sweep or reduction).  Right-hand sides that
are defined through the operator (``b = A * ones``) are computed by each side
with its own operator.

Generator: a counter-based SplitMix64 stream (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014).  Element ``i`` of
stream ``(seed, stream_id)`` is ``mix(key + (i + 1) * GAMMA)`` with
``key = mix(seed * GAMMA ^ (stream_id << 32))`` and ``mix`` the SplitMix64
finaliser.  Uniforms are ``(v >> 11) * 2**-53`` in [0, 1); normals use
Box-Muller on the uniform pairs (2i, 2i+1).

Workload recipes (shapes of the paper's benchmarks, Sec. 7.1):
  * HPCG 27-point: b = A * ones, x0 = 0 (no random numbers).
  * variable-kappa diffusion: log kappa = iid N(0,1) per cell, smoothed by a
    separable Gaussian (sigma = 4 cells, taps -12..12, periodic wrap),
    rescaled to unit marginal variance; kappa = exp(log kappa).
  * NPB-LU-shaped block SSOR: D_p = U(-1,1)^{5x5} + 10 I, L/U couplings
    U(-0.1, 0.1)^{5x5}, rhs U(-1,1), omega = 1.2.
  * batched problems: cube sides drawn from {32, 48, 64, 96, 128}.
  * NPB-SP-shaped line solves: per point a pentadiagonal row (a, b, c, d, e)
    with a, e ~ U(-0.25, 0.25), b, d ~ U(-1, 1), c ~ U(3, 4) (strictly
    diagonally dominant, so elimination needs no pivoting) and k = 5
    right-hand sides ~ U(-1, 1).
  * NPB-BT-shaped line solves: per point 5x5 blocks B = U(-1,1) + 10 I and
    A, C ~ U(-0.25, 0.25) (row sums of the off-diagonal magnitudes <= 6.5 <
    9 <= |B_jj|: strictly diagonally dominant), rhs ~ U(-1, 1).
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 13304

STREAM_KAPPA = 1
STREAM_D = 2
STREAM_L = 3
STREAM_U = 4
STREAM_RHS = 5
STREAM_TARGET = 6
STREAM_VEC = 7
STREAM_SIDES = 8
STREAM_PENTA = 9
STREAM_PENTA_RHS = 10
STREAM_BTRI = 11
STREAM_BTRI_RHS = 12
STREAM_JAC = 13
STREAM_JAC_RHS = 14
STREAM_JAC_U0 = 15
STREAM_SAMPLES = 16

BATCH_SIDES = (32, 48, 64, 96, 128)


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed, stream):
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA
    return _mix(s ^ (np.uint64(stream) << np.uint64(32)))


def raw_u64(seed, stream, n, start=0):
    """n raw 64-bit outputs of stream (seed, stream), elements start..start+n-1."""
    key = _key(seed, stream)
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + i * GAMMA)


def uniform(seed, stream, n, start=0, chunk=1 << 24):
    """n uniforms in [0, 1) (53-bit), FP64."""
    out = np.empty(n, dtype=np.float64)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        v = raw_u64(seed, stream, b - a, start + a)
        out[a:b] = (v >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return out


def normal(seed, stream, n):
    """n standard normals by Box-Muller on the uniform pairs (2i, 2i+1)."""
    u = uniform(seed, stream, 2 * n)
    u1 = u[0::2]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_taps(sigma=4.0, half_width=12):
    k = np.arange(-half_width, half_width + 1, dtype=np.float64)
    g = np.exp(-0.5 * (k / sigma) ** 2)
    return g / g.sum()


def kappa_field(n, seed=BASE_SEED, sigma=4.0, half_width=12, shape=None):
    """kappa = exp(smoothed unit-variance Gaussian field); shape (nz, ny, nx)."""
    from scipy.ndimage import convolve1d

    shape = (n, n, n) if shape is None else tuple(shape)
    f = normal(seed, STREAM_KAPPA, int(np.prod(shape))).reshape(shape)
    g = gaussian_taps(sigma, half_width)
    for ax in range(3):
        f = convolve1d(f, g, axis=ax, mode="wrap")
    f /= np.sum(g * g) ** 1.5
    return np.exp(f)


def block_ssor_inputs(n, seed=BASE_SEED, shape=None):
    """(D, L, U, rhs) for the NPB-LU-shaped block problem on an n^3 grid.

    D: (nz, ny, nx, 5, 5); L, U: (nz, ny, nx, 3, 5, 5) with index 0/1/2 the
    x/y/z coupling; rhs: (nz, ny, nx, 5).
    """
    shape = (n, n, n) if shape is None else tuple(shape)
    npts = int(np.prod(shape))
    D = (2.0 * uniform(seed, STREAM_D, npts * 25) - 1.0).reshape(shape + (5, 5))
    D += 10.0 * np.eye(5)
    L = (0.2 * uniform(seed, STREAM_L, npts * 75) - 0.1).reshape(shape + (3, 5, 5))
    U = (0.2 * uniform(seed, STREAM_U, npts * 75) - 0.1).reshape(shape + (3, 5, 5))
    rhs = (2.0 * uniform(seed, STREAM_RHS, npts * 5) - 1.0).reshape(shape + (5,))
    return D, L, U, rhs



def block_jac_inputs(shape, seed=BASE_SEED, sigma=10.0, nu=0.5):
    """(P, rhs, u0) for the SSOR step whose 5x5 blocks are formed from the
    state: P holds sigma, nu and, for k = 0..3 (point term, x, y, z), the
    flux parameters C_k ~ U(-0.1, 0.1) (5x5), E_k ~ U(-0.05, 0.05) (5x5),
    g_k ~ U(-0.2, 0.2) (5); rhs ~ U(-1, 1) and u0 ~ U(0, 1), (nz, ny, nx, 5).
    With |u| <= 1.5 every entry of a Jacobian is below 0.25 in magnitude, so
    each block row of A(u) is diagonally dominant (9.75 against < 8)."""
    shape = tuple(shape)
    npts = int(np.prod(shape))
    w = uniform(seed, STREAM_JAC, 4 * 55)
    P = np.empty(2 + 4 * 55)
    P[0], P[1] = sigma, nu
    for k in range(4):
        a = w[55 * k:55 * (k + 1)]
        base = 2 + 55 * k
        P[base:base + 25] = 0.2 * a[:25] - 0.1
        P[base + 25:base + 50] = 0.1 * a[25:50] - 0.05
        P[base + 50:base + 55] = 0.4 * a[50:55] - 0.2
    rhs = (2.0 * uniform(seed, STREAM_JAC_RHS, npts * 5) - 1.0).reshape(shape + (5,))
    u0 = uniform(seed, STREAM_JAC_U0, npts * 5).reshape(shape + (5,))
    return P, rhs, u0

def target(shape, seed=BASE_SEED):
    """u_target ~ U(0, 1)."""
    return uniform(seed, STREAM_TARGET, int(np.prod(shape))).reshape(shape)


def random_vector(shape, seed=BASE_SEED, stream_offset=0, lo=-1.0, hi=1.0):
    """A U(lo, hi) test vector (stream STREAM_VEC + stream_offset)."""
    u = uniform(seed, STREAM_VEC + 64 * stream_offset, int(np.prod(shape)))
    return (lo + (hi - lo) * u).reshape(shape)


def batch_sides(count=64, seed=BASE_SEED):
    """Cube sides of the batched problems, drawn from BATCH_SIDES."""
    u = uniform(seed, STREAM_SIDES, count)
    return [BATCH_SIDES[int(v * len(BATCH_SIDES))] for v in u]


def line_penta_inputs(shape, k=5, seed=BASE_SEED):
    """(coef, rhs) of the NPB-SP-shaped line solves on a grid of `shape`
    (nz, ny, nx): coef (nz, ny, nx, 5) = (a, b, c, d, e) per point, rhs
    (nz, ny, nx, k)."""
    shape = tuple(shape)
    npts = int(np.prod(shape))
    u = uniform(seed, STREAM_PENTA, npts * 5).reshape(shape + (5,))
    scale = np.array([0.5, 2.0, 1.0, 2.0, 0.5])
    shift = np.array([-0.25, -1.0, 3.0, -1.0, -0.25])
    coef = u * scale + shift
    rhs = (2.0 * uniform(seed, STREAM_PENTA_RHS, npts * k) - 1.0).reshape(shape + (k,))
    return coef, rhs


def line_btri_inputs(shape, seed=BASE_SEED):
    """(blk, rhs) of the NPB-BT-shaped line solves: blk (nz, ny, nx, 3, 5, 5)
    = (A, B, C) per point, rhs (nz, ny, nx, 5)."""
    shape = tuple(shape)
    npts = int(np.prod(shape))
    u = uniform(seed, STREAM_BTRI, npts * 75).reshape(shape + (3, 5, 5))
    blk = 0.5 * u - 0.25
    blk[..., 1, :, :] = 2.0 * u[..., 1, :, :] - 1.0 + 10.0 * np.eye(5)
    rhs = (2.0 * uniform(seed, STREAM_BTRI_RHS, npts * 5) - 1.0).reshape(shape + (5,))
    return blk, rhs


def sample_points(shape, count, seed=BASE_SEED):
    """Sorted distinct flat indices p = (z * ny + y) * nx + x of a grid of
    `shape` (nz, ny, nx) at which a full-size result is sampled: every
    corner, points on every edge and every face, points one cell inside the
    boundary, and uniform interior points; `count` is the number of drawn
    points before duplicates are removed (the corners come on top)."""
    nz, ny, nx = (int(v) for v in shape)
    ext = np.array([nx, ny, nz], dtype=np.int64)
    pts = []
    for cz in (0, nz - 1):
        for cy in (0, ny - 1):
            for cx in (0, nx - 1):
                pts.append((cx, cy, cz))
    corners = np.array(pts, dtype=np.int64).reshape(-1, 3)
    u = uniform(seed, STREAM_SAMPLES, 3 * count).reshape(count, 3)
    xyz = np.minimum((u * ext).astype(np.int64), ext - 1)
    q = count // 8
    # classes: [0, q) edges, [q, 3q) faces, [3q, 4q) one cell inside a face,
    # the rest interior
    cls = np.arange(count)
    sel = uniform(seed, STREAM_SAMPLES + 64, 2 * count).reshape(count, 2)
    axis = np.minimum((sel[:, 0] * 3).astype(np.int64), 2)
    side = sel[:, 1] < 0.5
    hi = ext[axis] - 1
    edge = cls < q
    face = (cls >= q) & (cls < 3 * q)
    inner = (cls >= 3 * q) & (cls < 4 * q)
    rows = np.arange(count)
    # faces: pin one coordinate to 0 or n - 1
    f = face | edge
    xyz[rows[f], axis[f]] = np.where(side[f], 0, hi[f])
    # edges: pin a second coordinate as well
    a2 = (axis + 1) % 3
    hi2 = ext[a2] - 1
    xyz[rows[edge], a2[edge]] = np.where(sel[edge, 0] * 6 % 1.0 < 0.5, 0, hi2[edge])
    # one cell inside a face
    xyz[rows[inner], axis[inner]] = np.where(side[inner], np.minimum(1, hi[inner]),
                                             np.maximum(hi[inner] - 1, 0))
    allp = np.concatenate([corners, xyz])
    flat = (allp[:, 2] * ny + allp[:, 1]) * nx + allp[:, 0]
    return np.unique(flat)
