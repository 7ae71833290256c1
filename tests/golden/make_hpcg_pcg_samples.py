"""Writes sampled entries of the oracle's FP64 MG-PCG solution of the
27-point HPCG problem (b = A*ones, x0 = 0, 4-level V-cycle with symmetric
Gauss-Seidel smoothing; the HPCG workload of Sec. 7.1).

Calls only oracle/ (and m2s_inputs for the seeded sample positions).

  python tests/golden/make_hpcg_pcg_samples.py N fixed50
      exactly 50 PCG iterations (HPCG's run length, Sec. 7.1), writes
      hpcg_pcg_samples_N_fixed50.txt with the 51-entry residual history
  python tests/golden/make_hpcg_pcg_samples.py N rtol
      to relative residual 1e-10, writes hpcg_pcg_samples_N_rtol.txt

Each file holds a header (lines starting with '#', with the iteration count
and the final residual 2-norm), the residual history as lines
"h <k> <value>", then one line "<flat index> <x value>" per sample point
(m2s_inputs.sample_points(shape, COUNT)).  At N = 256 the serial oracle
needs about 10 minutes for 50 iterations and 30 for the 1e-10 solve.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import m2s_inputs as gen  # noqa: E402
import oracle  # noqa: E402

COUNT = 16384


def main():
    n = int(sys.argv[1])
    mode = sys.argv[2]
    assert mode in ("fixed50", "rtol")
    shape = (n, n, n)
    b = oracle.apply(oracle.HPCG27, np.ones(shape))
    t0 = time.time()
    if mode == "fixed50":
        x, iters, hist, st = oracle.pcg(oracle.HPCG27, b, 4, max_iters=50, fixed_iters=True)
        assert iters == 50
    else:
        x, iters, hist, st = oracle.pcg(oracle.HPCG27, b, 4, max_iters=500, rtol=1e-10,
                                        fixed_iters=False)
    assert st == 0, st
    dt = time.time() - t0
    idx = gen.sample_points(shape, COUNT)
    xs = x.ravel()[idx]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                       "hpcg_pcg_samples_%d_%s.txt" % (n, mode))
    with open(out, "w") as f:
        f.write("# oracle FP64 MG-PCG, HPCG 27-point %d^3, b = A*ones, x0 = 0, 4 levels, %s\n"
                % (n, "50 fixed iterations" if mode == "fixed50" else "rtol 1e-10"))
        f.write("# iterations %d\n" % iters)
        f.write("# final_resid %.17e\n" % hist[-1])
        f.write("# max_abs_x_minus_1 %.6e\n" % float(np.max(np.abs(x - 1.0))))
        f.write("# samples m2s_inputs.sample_points((%d, %d, %d), %d): %d points\n"
                % (n, n, n, COUNT, len(idx)))
        f.write("# oracle time %.1f s\n" % dt)
        for k, h in enumerate(hist):
            f.write("h %d %.17e\n" % (k, h))
        for p, v in zip(idx, xs):
            f.write("%d %.17e\n" % (p, v))
    print(out, iters, "%.1f s" % dt)


if __name__ == "__main__":
    main()
