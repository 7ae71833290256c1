"""CPU-side checks of the boundary: the library builds for sm_103a, loads,
exports every function include/m2s.h declares, and rejects invalid
arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_13304_gb300 import build as b
    b.build()
    import paper_2204_13304_gb300 as m
    return m.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "m2s.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(m2s_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("m2s_grid_create", "m2s_grid_destroy", "m2s_spmv", "m2s_symgs",
                 "m2s_ssor_sweep", "m2s_mg_vcycle", "m2s_pcg_solve", "m2s_adjoint_solve"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_2204_13304_gb300 as m
    assert set(m.EXPORTS) == set(declared_functions())
    for name in m.EXPORTS:
        assert callable(getattr(m, name))


def test_status_strings(lib):
    for s in range(7):
        assert lib.m2s_status_string(s)
    assert b"timeout" in lib.m2s_status_string(4) or b"spin" in lib.m2s_status_string(4)


def test_invalid_arguments_rejected_without_gpu(lib):
    import paper_2204_13304_gb300 as m
    h = ctypes.c_void_p()
    assert lib.m2s_grid_create(None, 1, None, ctypes.byref(h)) == m.Status.INVALID_ARG
    d = (m.GridDesc * 1)()
    d[0].nx, d[0].ny, d[0].nz, d[0].op, d[0].mg_levels = 0, 4, 4, 0, 1
    assert lib.m2s_grid_create(d, 1, None, ctypes.byref(h)) == m.Status.INVALID_ARG
    assert not h.value
    d[0].nx, d[0].mg_levels = 4, 0
    assert lib.m2s_grid_create(d, 1, None, ctypes.byref(h)) == m.Status.INVALID_ARG
    d[0].mg_levels, d[0].op = 2, 1  # kappa operator without kappa
    assert lib.m2s_grid_create(d, 1, None, ctypes.byref(h)) == m.Status.INVALID_ARG
    assert lib.m2s_grid_create(d, 0, None, ctypes.byref(h)) == m.Status.INVALID_ARG
    d[0].mg_levels, d[0].op = 1, m.Op.BLOCK7_JAC  # blocks from the state without parameters
    assert lib.m2s_grid_create(d, 1, None, ctypes.byref(h)) == m.Status.INVALID_ARG
    d[0].op = 4  # no such operator
    assert lib.m2s_grid_create(d, 1, None, ctypes.byref(h)) == m.Status.INVALID_ARG
    assert not h.value
    assert lib.m2s_spmv(None, 0, 0, None, None, None) == m.Status.INVALID_ARG
    assert lib.m2s_symgs(None, 0, 0, None, None, 1, None) == m.Status.INVALID_ARG
    assert lib.m2s_pcg_solve(None, None, None, None, None, None) == m.Status.INVALID_ARG
    assert lib.m2s_ssor_sweep(None, None, None, 1.2, 1, None) == m.Status.INVALID_ARG
    assert lib.m2s_grid_destroy(None) == m.Status.OK


def test_grid_desc_layout_matches_header():
    """The ctypes descriptor has the header's fields in the header's order."""
    import re
    import paper_2204_13304_gb300 as m
    hdr = open(os.path.join(ROOT, "include", "m2s.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} m2s_grid_desc;", hdr).group(1)
    names = re.findall(r"(\w+)(?:\s*,\s*(\w+))?(?:\s*,\s*(\w+))?;", body)
    fields = [n for group in names for n in group if n]
    assert fields == [f[0] for f in m.GridDesc._fields_]


def test_bounds_record_of_the_normal_build_without_gpu(lib):
    """The normal build has no range checks compiled in: the record says so
    (-1) without a CUDA call."""
    import paper_2204_13304_gb300 as m
    assert m.m2s_debug_bounds_read()[0] == -1
    assert lib.m2s_debug_bounds_read(None) == m.Status.INVALID_ARG


def test_bounds_variant_builds_without_gpu():
    """The range-checked variant compiles for sm_103a into its own folder and
    exports the same symbols (it runs only in the GPU tests)."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r); "
            "from paper_2204_13304_gb300 import build as b; p = b.build(); "
            "import ctypes; L = ctypes.CDLL(p); L.m2s_debug_bounds_read; print(p)" % ROOT)
    env = dict(os.environ, M2S_BUILD_VARIANT="bounds")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.strip().endswith(os.path.join("_build_bounds", "libm2s.so"))


def test_library_is_sm103a_only():
    """The build targets exactly compute_103a/sm_103a."""
    from paper_2204_13304_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "--use_fast_math" not in b.FLAGS


def test_line_penta_rejects_invalid_arguments_without_gpu(lib):
    """Every rejected call returns before any CUDA call, so fake (never
    dereferenced) device addresses suffice."""
    import paper_2204_13304_gb300 as m
    nx, ny, nz, k = 4, 5, 6, 5
    n = nx * ny * nz
    need = lib.m2s_line_penta_work_bytes(nx, ny, nz)
    assert need == 3 * n * 8
    assert lib.m2s_line_penta_work_bytes(0, 5, 6) == 0
    coef, rhs, work = 1 << 20, 1 << 24, 1 << 28  # disjoint, 8-byte aligned
    bad = [
        (0, ny, nz, 0, coef, rhs, k, work, need),        # empty grid
        (nx, ny, nz, 3, coef, rhs, k, work, need),       # axis
        (nx, ny, nz, 0, coef, rhs, 0, work, need),       # k too small
        (nx, ny, nz, 0, coef, rhs, 9, work, need),       # k too large
        (nx, ny, nz, 0, None, rhs, k, work, need),       # NULL
        (nx, ny, nz, 0, coef + 4, rhs, k, work, need),   # misaligned
        (nx, ny, nz, 0, coef, rhs, k, work, need - 8),   # short work buffer
        (nx, ny, nz, 0, coef, coef + 8, k, work, need),  # rhs overlaps coef
        (nx, ny, nz, 0, coef, rhs, k, rhs + 8 * n, need),  # work overlaps rhs
    ]
    for a in bad:
        assert lib.m2s_line_penta(*a[:8], ctypes.c_longlong(a[8]), None) == m.Status.INVALID_ARG, a


def test_line_btri_rejects_invalid_arguments_without_gpu(lib):
    import paper_2204_13304_gb300 as m
    nx, ny, nz = 4, 5, 6
    n = nx * ny * nz
    need = lib.m2s_line_btri_work_bytes(nx, ny, nz)
    assert need == 25 * n * 8
    blk, rhs, work = 1 << 20, 1 << 24, 1 << 28
    bad = [
        (nx, 0, nz, 1, blk, rhs, work, need),
        (nx, ny, nz, -1, blk, rhs, work, need),
        (nx, ny, nz, 1, blk, None, work, need),
        (nx, ny, nz, 1, blk, rhs + 2, work, need),
        (nx, ny, nz, 1, blk, rhs, work, need - 1),
        (nx, ny, nz, 1, blk, blk + 8, work, need),
    ]
    for a in bad:
        assert lib.m2s_line_btri(*a[:7], ctypes.c_longlong(a[7]), None) == m.Status.INVALID_ARG, a


def test_ilu0_rejects_invalid_arguments_without_gpu(lib):
    import paper_2204_13304_gb300 as m
    assert lib.m2s_ilu0_setup(None, None) == m.Status.INVALID_ARG
    assert lib.m2s_ilu0_apply(None, None, None, None) == m.Status.INVALID_ARG
    assert lib.m2s_ilu0_factors(None, None, None) == m.Status.INVALID_ARG
