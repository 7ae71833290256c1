"""A CPU model of the mailbox index arithmetic of the ILU(0) wavefront
(csrc/k_ilu_wave.cu), which runs on the 27-point sweep's units (30 rows
u = y + z by W planes v = z, a lane of warp w at row u = u0 - 2 + lane) and
mailboxes, with one difference: warp 0 reads the three rows u - 2, u - 1, u
of the plane below (their values at x + 1) from a mailbox of full rows that
the top warp of every unit writes, instead of one plane sum.  The model
restates the kernel's formulas:

  row mailbox   ((v * ceil(NU / 30) + u / 30) * 2 + (u mod 30 - 28)) * nx
  plane rows    ((v / W) * NU + u) * nx,   NU = ny + nz - 1,

writers: lanes 30-31 (row mailbox) and the computing lanes of the top warp
(plane rows, for the plane above); readers: the halo lanes 0-1 (row
mailbox) and the computing lanes of warp 0, which read rows u - 2 + j wherever
x + 1 lies in the row (also at x = -1, whose window feeds x = 0).  Units
without a computing row are skipped by the kernel and write nothing.

Over every unit, lane, plane and x of a grid it checks that every index
stays inside the allocation of the sweep's set-up (nz * ceil(NU / 30) * 2 * nx
row values, ceil(nz / W) * NU * nx plane values), that every slot has one
writer, and that every read lands on the slot written for the same row,
plane and x.  This is the check run before the kernel's first launch.
"""
import pytest

from test_sweep_mailbox_model import unit_origins


def check_ilu_layout(nx, ny, nz, W, rev):
    NU = ny + nz - 1
    NUc = (NU - 1) // 30 + 1
    nbox = nz * NUc * 2 * nx
    npl = ((nz - 1) // W + 1) * NU * nx
    wbox, wpl, rbox, rpl = {}, {}, [], []
    R, sd = (nx - 1, -1) if rev else (0, 1)
    for (u0, v0) in unit_origins(nx, ny, nz, 30, W):
        computing = any(v0 + w < nz and 0 <= u0 - 2 + lane - (v0 + w) < ny
                        for w in range(W) for lane in range(2, 32))
        if not computing:
            continue
        for w in range(W):
            v = v0 + w
            for lane in range(32):
                u = u0 - 2 + lane
                halo = lane < 2
                mb_out = not halo and lane >= 30
                rv = v < nz and 0 <= u - v < ny
                mrow = ((v * NUc + u // 30) * 2 + (u % 30 - 28)) * nx \
                    if (u >= 0 and (halo or mb_out)) else 0
                t_out = w == W - 1 and not halo and rv and v + 1 < nz
                tout = (((v + 1) // W) * NU + u) * nx if t_out else 0
                pj = []
                for j in range(3):
                    uj = u - 2 + j
                    ok = w == 0 and not halo and rv and v >= 1 and 0 <= uj - (v - 1) < ny
                    pj.append((ok, ((v // W) * NU + uj) * nx if ok else 0, uj))
                for x in range(-3, nx + 3):
                    inx = 0 <= x < nx
                    if rv and inx and halo:
                        i = mrow + R + sd * x
                        assert 0 <= i < nbox
                        rbox.append((i, (u, v, x)))
                    if rv and inx and mb_out:
                        i = mrow + R + sd * x
                        assert 0 <= i < nbox and i not in wbox
                        wbox[i] = (u, v, x)
                    if t_out and inx:
                        i = tout + R + sd * x
                        assert 0 <= i < npl and i not in wpl
                        wpl[i] = (u, v, x)
                    for ok, base, uj in pj:
                        if ok and 0 <= x + 1 < nx:
                            i = base + R + sd * (x + 1)
                            assert 0 <= i < npl
                            rpl.append((i, (uj, v - 1, x + 1)))
    for i, key in rbox:
        assert wbox.get(i) == key, ("row read without its write", key)
    for i, key in rpl:
        assert wpl.get(i) == key, ("plane-row read without its write", key)
    return len(rbox), len(rpl)


SHAPES = [(5, 3, 4), (17, 33, 32), (33, 17, 35), (16, 64, 16), (40, 11, 3), (70, 5, 2),
          (3, 1, 1), (1, 1, 9), (4, 61, 2), (7, 30, 31), (2, 100, 17), (9, 31, 1), (6, 2, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("W", [4, 8])
@pytest.mark.parametrize("rev", [False, True])
def test_ilu_mailbox_layout(shape, W, rev):
    nz, ny, nx = shape
    check_ilu_layout(nx, ny, nz, W, rev)


def test_ilu_mailbox_reads_happen():
    """The model exercises both mailboxes on a grid of several units."""
    nrow, npl = check_ilu_layout(20, 40, 20, 4, False)
    assert nrow > 0 and npl > 0
