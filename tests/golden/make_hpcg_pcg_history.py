"""Writes the oracle's residual history of the FP64 MG-PCG solve of the
27-point HPCG operator (b = A*ones, x0 = 0, 4-level V-cycle, symmetric
Gauss-Seidel smoothing, relative residual 1e-10; Sec. 7.1 HPCG workload).

Calls only oracle/.  Usage:  python tests/golden/make_hpcg_pcg_history.py N
writes tests/golden/hpcg_pcg_history_N.txt (one residual 2-norm per line,
iteration 0 first).  At N = 256 the serial oracle needs tens of minutes.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402


def main():
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    shape = (n, n, n)
    b = oracle.apply(oracle.HPCG27, np.ones(shape))
    x, iters, hist, st = oracle.pcg(oracle.HPCG27, b, 4, max_iters=500, rtol=1e-10,
                                    fixed_iters=False)
    assert st == 0, st
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hpcg_pcg_history_%d.txt" % n)
    with open(out, "w") as f:
        f.write("# oracle FP64 MG-PCG, HPCG 27-point %d^3, b = A*ones, x0 = 0, 4 levels, "
                "rtol 1e-10: %d iterations; max |x - 1| = %.3e\n"
                % (n, iters, float(np.max(np.abs(x - 1.0)))))
        for h in hist:
            f.write("%.17e\n" % h)
    print(out, iters)


if __name__ == "__main__":
    main()
