"""The bounds variant of the library (every global index derived from a
neighbour, a line, a hyperplane or a scatter target range-checked in the
block, ILU(0) and line-solve kernels; a violation is counted and skipped,
never trapped) runs those entry points on small ragged grids without a single
violation, with results equal to the oracle's.  It stands in for a memory
checker, which is closed on this machine."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_variant_records_no_violation():
    env = dict(os.environ, M2S_BUILD_VARIANT="bounds")
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    violations, line, index, unit = out["bounds"]
    assert violations == 0, "range check failed %d times; first: unit %d line %d index %d" % (
        violations, unit, line, index)
    for name, e in out["errors"].items():
        assert e <= 1e-12, (name, e)
