"""A CPU model of the mailbox index arithmetic of the 27-point CTA sweep
(csrc/k_wave2.cu): units of 30 rows u = y + z by W planes v = z (one plane
per warp in both dtypes), a lane of warp w at row u = u0 - 2 + lane, halo
lanes 0-1 reading and lanes 30-31 writing the compact row mailbox, warp 0
reading and the top warp writing the plane-sum mailbox, x running forward or
backward.  The model restates, in Python, the formulas the kernel uses:

  mailbox row   ((v * ceil(NU / 30) + u / 30) * 2 + (u mod 30 - 28)) * nx
  plane sums    ((v / W) * NU + u) * nx,   NU = ny + nz - 1,

and the unit list of the kernel's set-up (units holding a valid row, plus
the ghost units underneath them whose top warp must publish plane sums).

Over every unit, lane, plane and x of a grid it checks that every index
stays inside the mailbox the set-up allocates (nz * ceil(NU / 30) * 2 * nx
row values, ceil(nz / W) * NU * nx plane-sum values), that every slot has
one writer, and that every read lands on the slot written for the same row
and x.  This is the check that was run before the kernel's first launch,
kept as a test of the layout on ragged shapes.
"""
import pytest


def unit_origins(nx, ny, nz, lanes, planes):
    """(u0, v0) of the units of one grid: those holding a valid row, plus
    ghost units below them."""
    umax = (ny - 1) + (nz - 1)
    org = []
    for V in range((nz + planes - 1) // planes):
        for U in range(umax // lanes + 1):
            u0, v0 = U * lanes, V * planes
            if any(max(u0, v) <= min(u0 + lanes - 1, v + ny - 1)
                   for v in range(v0, min(v0 + planes, nz))):
                org.append((u0, v0))
    has = {(o[1] // planes, o[0] // lanes) for o in org}
    for u0, v0 in list(org):
        U, V = u0 // lanes, v0 // planes
        if V >= 1 and (V - 1, U) not in has:
            has.add((V - 1, U))
            org.append((U * lanes, (V - 1) * planes))
    return org


def check_layout(nx, ny, nz, W, rev):
    NU = ny + nz - 1
    NUc = (NU - 1) // 30 + 1
    nbox = nz * NUc * 2 * nx
    ng = ((nz - 1) // W + 1) * NU * nx
    wbox, wg, rbox, rg = {}, {}, [], []
    R, sd = (nx - 1, -1) if rev else (0, 1)
    for (u0, v0) in unit_origins(nx, ny, nz, 30, W):
        for w in range(W):
            v = v0 + w
            for lane in range(32):
                u = u0 - 2 + lane
                halo = lane < 2
                mb_out = not halo and lane >= 30
                y = u - v
                rv = v < nz and 0 <= y < ny
                g_in = w == 0 and v >= 1
                yu = u - (v + 1)
                g_out = w == W - 1 and not halo and v + 1 < nz and 0 <= yu < ny
                mrow = ((v * NUc + u // 30) * 2 + (u % 30 - 28)) * nx \
                    if (u >= 0 and (halo or mb_out)) else 0
                grow_in = ((v // W) * NU + u) * nx if g_in else 0
                grow_out = (((v + 1) // W) * NU + u) * nx if g_out else 0
                for x in range(-3, nx + 3):
                    inx = 0 <= x < nx
                    xm = R + sd * x
                    if rv and inx and halo:
                        i = mrow + xm
                        assert 0 <= i < nbox
                        rbox.append((i, (u, v, x)))
                    if rv and inx and mb_out:
                        i = mrow + xm
                        assert 0 <= i < nbox and i not in wbox
                        wbox[i] = (u, v, x)
                    if rv and inx and not halo and g_in:
                        i = grow_in + xm
                        assert 0 <= i < ng
                        rg.append((i, (u, v, x)))
                    if g_out and 0 <= x - 1 < nx:
                        i = grow_out + R + sd * (x - 1)
                        assert 0 <= i < ng and i not in wg
                        wg[i] = (u, v + 1, x - 1)
    for i, key in rbox:
        assert wbox.get(i) == key, ("row read without its write", key)
    for i, key in rg:
        assert wg.get(i) == key, ("plane-sum read without its write", key)
    return len(rbox), len(rg)


SHAPES = [(5, 3, 4), (17, 33, 32), (33, 17, 35), (16, 64, 16), (40, 11, 3), (70, 5, 2),
          (3, 1, 1), (1, 1, 9), (4, 61, 2), (7, 30, 31), (2, 100, 17), (9, 31, 1), (6, 2, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("W", [4, 8])
@pytest.mark.parametrize("rev", [False, True])
def test_mailbox_layout(shape, W, rev):
    nz, ny, nx = shape
    check_layout(nx, ny, nz, W, rev)


def test_mailbox_reads_happen():
    """The model exercises both mailboxes on a grid of several units."""
    nrow, ng = check_layout(20, 40, 20, 4, False)
    assert nrow > 0 and ng > 0
