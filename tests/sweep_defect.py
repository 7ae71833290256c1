"""Sampled check of one exact lexicographic Gauss-Seidel sweep of the 27-point
HPCG operator (Sec. 4.3.3 SymGS; operator of Sec. 7.1: a_pp = 26, a_pq = -1
for the in-domain points of the 3x3x3 box).

After a forward sweep every point p satisfies

    26 x'_p = b_p + sum over in-domain neighbours q of
              x'_q  if q comes before p in lexicographic order (updated),
              x_q   otherwise (still the old value),

and a backward sweep is the same with the order reversed.  The identity
involves only the 27-point neighbourhood of p, so it can be checked on
sampled points of a grid of any size, where the serial oracle cannot run.
A sweep that reads an old value where the order requires the new one (or
the reverse), drops a neighbour or uses another diagonal leaves a residual
of the size of the values themselves; rounding leaves ~1e-15 of the sum of
the magnitudes.  Test infrastructure: numpy only, shared by the CPU pins of
this checker and the full-size GPU tests.
"""
import numpy as np

# the 26 neighbour offsets (dz, dy, dx); lexicographic order is z outermost,
# x fastest, so q precedes p iff the first nonzero offset is negative
OFFSETS = np.array([(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                    if (dz, dy, dx) != (0, 0, 0)], dtype=np.int64)
BEFORE = np.array([o[0] < 0 or (o[0] == 0 and (o[1] < 0 or (o[1] == 0 and o[2] < 0)))
                   for o in OFFSETS])


def sample_points(shape, k, seed):
    """k seeded points of the grid plus its 8 corners (sorted, unique)."""
    nz, ny, nx = shape
    n = nz * ny * nx
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, n, size=k, dtype=np.int64)
    corners = [(z * ny + y) * nx + x for z in (0, nz - 1) for y in (0, ny - 1) for x in (0, nx - 1)]
    return np.unique(np.concatenate([pts, np.array(corners, dtype=np.int64)]))


def neighbours(shape, p):
    """Flat indices q (len(p) x 26) of the neighbours of p and their in-domain
    mask; out-of-domain entries hold p itself (masked out)."""
    nz, ny, nx = shape
    p = np.asarray(p, dtype=np.int64)
    z, y, x = p // (ny * nx), (p // nx) % ny, p % nx
    qz = z[:, None] + OFFSETS[None, :, 0]
    qy = y[:, None] + OFFSETS[None, :, 1]
    qx = x[:, None] + OFFSETS[None, :, 2]
    valid = (qz >= 0) & (qz < nz) & (qy >= 0) & (qy < ny) & (qx >= 0) & (qx < nx)
    q = np.where(valid, (qz * ny + qy) * nx + qx, p[:, None])
    return q, valid


def defect(b_p, xnew_p, xnew_q, xold_q, valid, backward=False, diag=26.0):
    """Largest residual of the sweep identity over the sampled points,
    relative to the sum of the magnitudes of its terms."""
    b_p = np.asarray(b_p, dtype=np.float64)
    xnew_p = np.asarray(xnew_p, dtype=np.float64)
    first = ~BEFORE if backward else BEFORE
    vals = np.where(first[None, :], np.asarray(xnew_q, dtype=np.float64),
                    np.asarray(xold_q, dtype=np.float64))
    vals = np.where(valid, vals, 0.0)
    res = diag * xnew_p - b_p - vals.sum(axis=1)
    mag = diag * np.abs(xnew_p) + np.abs(b_p) + np.abs(vals).sum(axis=1)
    return float(np.max(np.abs(res) / np.maximum(mag, np.finfo(np.float64).tiny)))


def sweep_defect_numpy(b, x_old, x_new, samples, backward=False):
    """The check on host arrays of shape (nz, ny, nx)."""
    q, valid = neighbours(b.shape, samples)
    fb, fo, fn = b.reshape(-1), x_old.reshape(-1), x_new.reshape(-1)
    return defect(fb[samples], fn[samples], fn[q], fo[q], valid, backward)


def sweep_defect_torch(b, x_old, x_new, samples, backward=False):
    """The check on device tensors: the sampled neighbourhoods are gathered
    on the device and the identity is evaluated on the host in FP64."""
    import torch
    q, valid = neighbours(tuple(b.shape), samples)
    dev = b.device
    ps = torch.from_numpy(samples).to(dev)
    qs = torch.from_numpy(q.reshape(-1)).to(dev)
    fb, fo, fn = b.reshape(-1), x_old.reshape(-1), x_new.reshape(-1)
    got = [t.double().cpu().numpy() for t in (fb[ps], fn[ps], fn[qs], fo[qs])]
    return defect(got[0], got[1], got[2].reshape(q.shape), got[3].reshape(q.shape), valid, backward)


# ---------------------------------------------------------------------------
# The variable-kappa 7-point operator (face coefficient k_f = (kappa_p +
# kappa_q) / 2, a boundary face at kappa_p with a zero ghost value; Sec. 4.1
# averaging): after a forward sweep every point satisfies
#   a_pp x'_p = b_p + sum_{lower faces} k_f x'_q + sum_{upper faces} k_f x_q,
# a_pp the sum of its six face coefficients; a backward sweep mirrors it.
# ---------------------------------------------------------------------------
FACES = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]  # (dx, dy, dz)


def face_neighbours(shape, p):
    nz, ny, nx = shape
    p = np.asarray(p, dtype=np.int64)
    z, y, x = p // (ny * nx), (p // nx) % ny, p % nx
    qs, oks = [], []
    for dx, dy, dz in FACES:
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & \
             (z + dz >= 0) & (z + dz < nz)
        qs.append(np.where(ok, p + (dz * ny + dy) * nx + dx, p))
        oks.append(ok)
    return np.stack(qs, 1), np.stack(oks, 1)


def kappa_defect(b_p, kap_p, kap_q, xnew_p, xnew_q, xold_q, valid, backward=False):
    """Largest residual of the 7-point sweep identity relative to the sum of
    the magnitudes of its terms (arrays gathered at the sampled points)."""
    lower = np.array([d[0] + d[1] + d[2] < 0 for d in FACES])
    new = lower != backward
    kface = np.where(valid, 0.5 * (kap_p[:, None] + kap_q), kap_p[:, None])
    app = kface.sum(axis=1)
    terms = np.where(valid, kface * np.where(new[None, :], xnew_q, xold_q), 0.0)
    lhs = app * xnew_p
    res = lhs - b_p - terms.sum(axis=1)
    mag = np.abs(lhs) + np.abs(b_p) + np.abs(terms).sum(axis=1)
    return float(np.max(np.abs(res) / np.maximum(mag, np.finfo(np.float64).tiny)))


def kappa_defect_numpy(kappa, b, x_old, x_new, samples, backward=False):
    q, valid = face_neighbours(b.shape, samples)
    k, bf, xo, xn = kappa.reshape(-1), b.reshape(-1), x_old.reshape(-1), x_new.reshape(-1)
    return kappa_defect(bf[samples], k[samples], k[q], xn[samples], xn[q], xo[q], valid, backward)


def kappa_defect_torch(kappa, b, x_old, x_new, samples, backward=False):
    import torch
    q, valid = face_neighbours(tuple(b.shape), samples)
    dev = b.device
    ps = torch.from_numpy(samples).to(dev)
    qs = torch.from_numpy(q.reshape(-1)).to(dev)
    k, bf, xo, xn = kappa.reshape(-1), b.reshape(-1), x_old.reshape(-1), x_new.reshape(-1)
    g = [t.double().cpu().numpy() for t in (bf[ps], k[ps], k[qs], xn[ps], xn[qs], xo[qs])]
    return kappa_defect(g[0], g[1], g[2].reshape(q.shape), g[3], g[4].reshape(q.shape),
                        g[5].reshape(q.shape), valid, backward)
