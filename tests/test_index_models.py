"""CPU models of the index arithmetic of three kernels whose threads map to
grid points in a non-trivial way.  Each model restates, in Python, the
mapping the kernel's source uses, and checks the property the kernel relies
on over ragged shapes:

* ILU(0) hyperplane launches (csrc/k_ilu.cu: hyperplane_launch,
  hyperplane_point): over the launches t = 0 .. T-1 every point is visited
  exactly once, on its own hyperplane t = x + 2y + 4z, and each of its
  lexicographically lower 27-point neighbours lies on an earlier hyperplane
  (so stream order between the launches carries every dependence).
* The forming pass of the blocks formed from the state (csrc/k_block.cu:
  block_jac_form_kernel): every L and U slot of every point has exactly one
  writer -- the neighbour whose state the block reads, or the point itself
  writing zero where the grid ends.
* Line solves (csrc/k_line.cu: line_of and the launch's line count): the
  lines of an axis visit every point exactly once, each line in order along
  the axis, and for the y and z axes neighbouring threads hold neighbouring x
  (the coalescing the kernel's comment claims).
"""
import itertools

import pytest

SHAPES = [(1, 1, 1), (1, 3, 1), (7, 1, 9), (3, 4, 5), (5, 3, 4), (9, 11, 13), (16, 6, 33),
          (2, 17, 2), (12, 12, 12)]


def c_div(a, b):
    """C integer division (truncation toward zero)."""
    q = abs(a) // abs(b)
    return q if (a >= 0) == (b >= 0) else -q


# ---------------------------------------------------------------- ILU(0)
IB = 256


def hyperplane_launch(nx, ny, nz, t):
    reach = (nx - 1) + 2 * (ny - 1)
    zlo = max(0, c_div(t - reach + 3, 4))
    zhi = min(nz - 1, c_div(t, 4))
    win = c_div(nx, 2) + 2
    bs = min(IB, c_div(win + 31, 32) * 32)
    return (c_div(win + bs - 1, bs), max(0, zhi - zlo + 1)), bs, zlo


def hyperplane_point(nx, ny, nz, t, z0, bx, by, tx, bs):
    z = z0 + by
    rem = t - 4 * z
    if rem < 0:
        return None
    ylo = c_div(rem - (nx - 1) + 1, 2) if rem - (nx - 1) > 0 else 0
    y = ylo + bx * bs + tx
    x = rem - 2 * y
    return (x, y, z) if (y < ny and 0 <= x < nx) else None


@pytest.mark.parametrize("shape", SHAPES)
def test_ilu_hyperplanes_visit_every_point_once_in_dependence_order(shape):
    nz, ny, nx = shape
    T = (nx - 1) + 2 * (ny - 1) + 4 * (nz - 1) + 1
    seen = {}
    for t in range(T):
        (gx, gy), bs, z0 = hyperplane_launch(nx, ny, nz, t)
        for bx, by, tx in itertools.product(range(gx), range(gy), range(bs)):
            pt = hyperplane_point(nx, ny, nz, t, z0, bx, by, tx, bs)
            if pt is None:
                continue
            x, y, z = pt
            assert 0 <= z < nz and x + 2 * y + 4 * z == t
            assert pt not in seen
            seen[pt] = t
    assert len(seen) == nx * ny * nz
    for (x, y, z), t in seen.items():
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            lower = dz < 0 or (dz == 0 and (dy < 0 or (dy == 0 and dx < 0)))
            q = (x + dx, y + dy, z + dz)
            if lower and q in seen:
                assert seen[q] < t


# ------------------------------------------------- blocks formed from the state
@pytest.mark.parametrize("shape", SHAPES)
def test_block_forming_pass_has_one_writer_per_slot(shape):
    nz, ny, nx = shape
    n = nx * ny * nz
    st = (1, nx, nx * ny)
    writers = {}
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        p = (z * ny + y) * nx + x
        lo = (x > 0, y > 0, z > 0)
        hi = (x < nx - 1, y < ny - 1, z < nz - 1)
        for d in range(3):
            if hi[d]:  # L of p + e_d reads u_p
                writers.setdefault(("L", p + st[d], d), []).append(p)
            if lo[d]:  # U of p - e_d reads u_p
                writers.setdefault(("U", p - st[d], d), []).append(p)
            if not lo[d]:
                writers.setdefault(("L", p, d), []).append(p)
            if not hi[d]:
                writers.setdefault(("U", p, d), []).append(p)
    assert len(writers) == 2 * 3 * n
    assert all(len(w) == 1 for w in writers.values())
    assert all(0 <= slot[1] < n for slot in writers)


# ------------------------------------------------------------------ line solves
LB = 32


def line_of(nx, ny, nz, axis, t):
    if axis == 0:
        if t >= ny * nz:
            return None
        return t * nx, 1, nx
    if axis == 1:
        if t >= nx * nz:
            return None
        z, x = divmod(t, nx)
        return z * nx * ny + x, nx, ny
    if t >= nx * ny:
        return None
    return t, nx * ny, nz


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_lines_cover_every_point_once(shape, axis):
    nz, ny, nx = shape
    n = nx * ny * nz
    lines = (ny * nz, nx * nz, nx * ny)[axis]
    grid = c_div(lines + LB - 1, LB)
    seen = set()
    firsts = []
    for t in range(grid * LB):
        r = line_of(nx, ny, nz, axis, t)
        if r is None:
            continue
        base, stride, m = r
        firsts.append(base)
        pts = [base + i * stride for i in range(m)]
        assert 0 <= pts[0] and pts[-1] < n  # the two ends bound the line
        for i, q in enumerate(pts):
            x, y, z = q % nx, (q // nx) % ny, q // (nx * ny)
            assert (x, y, z)[axis] == i  # in order along the axis
            assert q not in seen
            seen.add(q)
    assert len(seen) == n
    if axis > 0:  # neighbouring threads start at neighbouring x of one row
        for a, b in zip(firsts, firsts[1:]):
            if a // nx == b // nx:
                assert b == a + 1
