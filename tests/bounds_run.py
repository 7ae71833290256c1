"""Runs the block, ILU(0) and line-solve entry points through the bounds
variant of the library (range checks compiled in, csrc/m2s_bounds.cuh) on
small ragged grids and prints one JSON line: the range-check record and the
largest error against the oracle.  Started by tests/test_gpu_bounds.py in a
process of its own with M2S_BUILD_VARIANT=bounds (the variant is chosen when
the package is imported)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    assert os.environ.get("M2S_BUILD_VARIANT") == "bounds"
    import numpy as np
    import torch

    import m2s_inputs as gen
    import oracle
    import paper_2204_13304_gb300 as m
    from paper_2204_13304_gb300 import build

    build.build()
    m.load()
    assert m.lib_path().endswith(os.path.join("_build_bounds", "libm2s.so"))
    torch.cuda.set_device(0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    errs = {}

    def rel(g, o):
        o = np.asarray(o)
        return float(np.max(np.abs(np.asarray(g) - o)) / max(np.max(np.abs(o)), 1e-300))

    # stored-block SSOR, two problems of different shapes
    shapes = [(3, 7, 5), (6, 2, 9)]
    ins = [gen.block_ssor_inputs(0, shape=s, seed=7 + i) for i, s in enumerate(shapes)]
    g = m.Grid([dict(nx=s[2], ny=s[1], nz=s[0], op=m.Op.BLOCK7_5x5, mg_levels=1,
                     D=dev(D), L=dev(L), U=dev(U)) for s, (D, L, U, b) in zip(shapes, ins)])
    u = torch.zeros(sum(int(np.prod(s)) * 5 for s in shapes), dtype=torch.float64, device="cuda")
    bb = dev(np.concatenate([b.ravel() for (_, _, _, b) in ins]))
    m.m2s_ssor_sweep(g.handle, bb, u, 1.2, 2)
    y = torch.empty_like(u)
    m.m2s_spmv(g.handle, 0, u, y)
    m.m2s_grid_sync(g.handle)
    g.close()
    uh, off, e = u.cpu().numpy(), 0, 0.0
    for s, (D, L, U, b) in zip(shapes, ins):
        n = int(np.prod(s)) * 5
        e = max(e, rel(uh[off:off + n].reshape(s + (5,)),
                       oracle.ssor(D, L, U, 1.2, b, np.zeros(s + (5,)), 2)))
        off += n
    errs["block_ssor"] = e

    # blocks formed from the state, two problems
    shapes = [(4, 5, 3), (1, 6, 2)]
    ins = [gen.block_jac_inputs(s, seed=11 + i) for i, s in enumerate(shapes)]
    g = m.Grid([dict(nx=s[2], ny=s[1], nz=s[0], op=m.Op.BLOCK7_JAC, mg_levels=1, jac=P)
                for s, (P, _, _) in zip(shapes, ins)])
    u = dev(np.concatenate([u0.ravel() for (_, _, u0) in ins]))
    bb = dev(np.concatenate([b.ravel() for (_, b, _) in ins]))
    y = torch.empty_like(u)
    m.m2s_spmv(g.handle, 0, u, y)
    m.m2s_ssor_sweep(g.handle, bb, u, 1.2, 2)
    m.m2s_grid_sync(g.handle)
    g.close()
    uh, off, e = u.cpu().numpy(), 0, 0.0
    for s, (P, b, u0) in zip(shapes, ins):
        n = int(np.prod(s)) * 5
        e = max(e, rel(uh[off:off + n].reshape(s + (5,)), oracle.ssor_jac(P, 1.2, b, u0, 2)))
        off += n
    errs["block_jac"] = e

    # ILU(0): two problems, factorisation and one application
    shapes = [(5, 4, 6), (3, 7, 2)]
    g = m.Grid([dict(nx=s[2], ny=s[1], nz=s[0], op=m.Op.HPCG27, mg_levels=1) for s in shapes])
    m.m2s_ilu0_setup(g.handle)
    rs = [gen.random_vector(s, seed=21 + i) for i, s in enumerate(shapes)]
    r = dev(np.concatenate([v.ravel() for v in rs]))
    z = torch.empty_like(r)
    m.m2s_ilu0_apply(g.handle, r, z)
    torch.cuda.synchronize()
    g.close()
    zh, off, e = z.cpu().numpy(), 0, 0.0
    for s, v in zip(shapes, rs):
        n = int(np.prod(s))
        e = max(e, rel(zh[off:off + n].reshape(s), oracle.ilu0_apply(oracle.ilu0_factor(s), v)))
        off += n
    errs["ilu0"] = e

    # line solves along every axis
    s = (5, 6, 7)
    coef, rhs = gen.line_penta_inputs(s, k=3)
    blk, rhs5 = gen.line_btri_inputs(s)
    e1 = e2 = 0.0
    for axis in (0, 1, 2):
        t = dev(rhs)
        m.m2s_line_penta(dev(coef), t, axis)
        e1 = max(e1, rel(t.cpu().numpy(), oracle.line_penta(coef, rhs, axis)))
        t = dev(rhs5)
        m.m2s_line_btri(dev(blk), t, axis)
        e2 = max(e2, rel(t.cpu().numpy(), oracle.line_btri(blk, rhs5, axis)))
    errs["line_penta"], errs["line_btri"] = e1, e2
    torch.cuda.synchronize()
    rec = m.m2s_debug_bounds_read()
    print(json.dumps({"bounds": rec, "errors": errs}))


if __name__ == "__main__":
    main()
