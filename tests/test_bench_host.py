"""Host logic of bench.py on the CPU: the figures it reads from the committed
ncu summaries (only while the kernel's sources hash to the summary's
source_sha256), the stored oracle results it reports against (iteration
count, solution samples) and the per-entry error it computes from them."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_profile_value_follows_the_source_hash(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_case.md").write_text(
        "# k\n\n- source_sha256: %s\n- dram_bytes_per_launch: 1234\n" % digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    val, why = bench.profile_value("k_case", "dram_bytes_per_launch", ("k.cu",))
    assert val == 1234.0 and "k_case.md" in why
    # the kernel changed since the capture: no figure
    src.write_text("__global__ void k() { }\n")
    val, why = bench.profile_value("k_case", "dram_bytes_per_launch", ("k.cu",))
    assert val is None and "changed" in why
    # no summary at all
    val, _ = bench.profile_value("missing", "dram_bytes_per_launch", ("k.cu",))
    assert val is None


def test_committed_sweep_profile_figures_are_plausible():
    """While the committed 27-point sweep summary matches the sources, its
    figures that bench.py reports are those of a 256^3 sweep."""
    val, why = bench.profile_value("gs27_cta_kernel_f64_256", "dram_bytes_per_launch")
    if val is None:
        pytest.skip(why)  # the sweep's sources changed since the committed capture
    # 256^3 rows moving the design's 32 B each, plus mailbox words
    assert 32 * 256 ** 3 <= val <= 48 * 256 ** 3
    fp64, _ = bench.profile_value("gs27_cta_kernel_f64_256", "fp64_warp_instructions_per_launch")
    # 7 (backward) to 8 (forward) FP64 operations per row, 32 rows per warp
    # instruction at most: never fewer warp instructions than that
    assert fp64 is not None and fp64 >= 7 * 256 ** 3 / 32


def test_stored_oracle_results_for_the_bench_size():
    iters, src = bench.oracle_iterations(256)
    assert iters == 153 and "hpcg_pcg_history_256" in src
    assert bench.oracle_iterations(100)[0] is None
    s = bench.oracle_samples(256)
    assert s is not None and len(s[0]) == len(s[1]) == 15756
    assert all(0 <= p < 256 ** 3 for p in s[0])
    # the oracle's solution of A x = A ones is within 1e-8 of ones
    assert max(abs(v - 1.0) for v in s[1]) < 1e-8
    assert bench.oracle_samples(100) is None


def test_err_vs_oracle_samples_is_the_per_entry_error():
    torch = pytest.importorskip("torch")
    idx = [0, 5, 9]
    val = [2.0, -4.0, 1e-6]
    x = torch.zeros(10, dtype=torch.float64)
    x[0], x[5], x[9] = 2.0, -4.0, 1e-6
    assert bench.err_vs_oracle_samples(torch, x, (idx, val)) == 0.0
    # an error of 1e-3 at the small entry is scaled by the floor 1e-3 max|o| = 4e-3
    x[9] = 1e-6 + 1e-3
    e = bench.err_vs_oracle_samples(torch, x, (idx, val))
    assert e == pytest.approx(1e-3 / 4e-3, rel=1e-12)
    # a relative error of 1e-12 at a large entry
    x[9] = 1e-6
    x[5] = -4.0 * (1 + 1e-12)
    assert bench.err_vs_oracle_samples(torch, x, (idx, val)) == pytest.approx(1e-12, rel=1e-3)
    assert bench.err_vs_oracle_samples(torch, x, None) is None
