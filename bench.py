"""Benchmark: FP64 MG-PCG to a relative residual of 1e-10 on the 256^3 HPCG
27-point problem (b = A*ones, x0 = 0, 4-level V-cycle with symmetric
Gauss-Seidel smoothing), the paper's HPCG workload shape (Sec. 7.1).

One step = one complete solve (every row of the hot path: SpMV, forward and
backward lexicographic sweeps, restriction, prolongation, V-cycle, PCG).
The JSON line also carries the FP32-preconditioned solve of the same problem,
per-kernel timings of the dominant kernels (CUDA events on the launching
stream), the roofline of the dominant kernel, an end-to-end time through the
public API with host buffers, and the serial oracle on the host CPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--size 256] [--impl ours|reference]

Multi-GPU: the solve does not shard (exact lexicographic Gauss-Seidel is
sequential across z-slabs), so N GPUs run N independent replicas; value is
the whole job's time per solve (max-over-ranks time / solves of all ranks).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MG-PCG time to 1e-10 at 256^3 (FP64 vs FP32-precond); SymGS/SpMV HBM GB/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 issue rate of a GB300: 152 SMs x 4 sub-partitions, one FP64 warp
# instruction per ~64 clocks each (2 FP64 lanes/clk/SM) at the 2070 MHz
# maximum SM clock -> 152 * 2 * 2.07e9 = 629 G FP64 operations/s
# (= 1.26 TFLOP/s counting an FMA as 2).
FP64_OPS_PEAK = 152 * 2 * 2.07e9


class Clocks:
    """Samples nvidia-smi during the timed region."""

    def __init__(self):
        self.samples = []
        self.proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", dev, "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        s = self.samples
        if not s:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        import statistics
        sm = [float(x[0]) for x in s if x[0].replace(".", "").isdigit()]
        mx = [float(x[1]) for x in s if x[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for x in s for i in range(4) if x[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(s)}


def dist_init(args, backend="nccl"):
    """One process per GPU (torchrun environment).  The solve does not shard:
    each rank runs a replica; ranks meet only at the barriers around the timed
    region and in the max over ranks of the time."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, t_rank):
    """Whole-job time per solve: the slowest rank's time per solve divided by
    the solves of all ranks (each rank solves one replica per step)."""
    return max_over_ranks(ws, t_rank) / ws


def oracle_pcg_seconds_per_iteration(n, iters):
    """The serial oracle's FP64 MG-PCG on the n^3 HPCG problem (b = A*ones,
    x0 = 0, 4 levels), run for exactly `iters` iterations (the oracle as it
    stands: V-cycle, SpMV, Dot2 dots and updates); returns seconds per
    iteration."""
    import numpy as np
    import oracle
    b = oracle.apply(oracle.HPCG27, np.ones((n, n, n)))
    t0 = time.perf_counter()
    oracle.pcg(oracle.HPCG27, b, 4, max_iters=iters, fixed_iters=True)
    return (time.perf_counter() - t0) / iters


def cpu_baseline(n, iters=3):
    """The serial oracle on a bounded sample of the workload: the first
    `iters` iterations of the same n^3 MG-PCG solve, timed on one host core
    and scaled to a solve by the oracle's iteration count."""
    per_iter = oracle_pcg_seconds_per_iteration(n, iters)
    return per_iter, iters


def oracle_config_times(gpu):
    """The serial oracle on the other workload configurations, one host core,
    each on a bounded sample stated beside it.  `gpu` holds the GPU run's
    iteration counts used to scale per-iteration samples to solves."""
    import numpy as np
    import m2s_inputs as gen
    import oracle
    out = {}
    tic = time.perf_counter

    # 32^3 HPCG: the whole configuration (SpMV, one symmetric GS, 50
    # SGS-PCG iterations)
    n = 32
    b = oracle.apply(oracle.HPCG27, np.ones((n, n, n)))
    t0 = tic()
    oracle.apply(oracle.HPCG27, b)
    t1 = tic()
    oracle.symgs(oracle.HPCG27, b, np.zeros_like(b), 1)
    t2 = tic()
    oracle.pcg(oracle.HPCG27, b, 1, max_iters=50, fixed_iters=True)
    t3 = tic()
    out["hpcg_32"] = {"spmv_us": (t1 - t0) * 1e6, "symgs_us": (t2 - t1) * 1e6,
                      "sgs_pcg_50_ms": (t3 - t2) * 1e3, "sample": "the whole configuration"}

    # 162^3 x 5 block SSOR: one iteration on a 64^3 x 5 grid of the same
    # recipe, scaled by the point count to 162^3 and by 50 iterations
    ns = 64
    D, L, U, rhs = gen.block_ssor_inputs(ns)
    t0 = tic()
    oracle.ssor(D, L, U, 1.2, rhs, np.zeros_like(rhs), 1)
    per_pt = (tic() - t0) / ns ** 3
    del D, L, U
    out["block_ssor_162x5"] = {"s_50_iters": per_pt * 162 ** 3 * 50,
                               "ms_per_iter": per_pt * 162 ** 3 * 1e3,
                               "sample": "one SSOR iteration on 64^3 x 5, scaled by points "
                                         "(x %.1f) and iterations (x 50)" % ((162 / 64) ** 3)}

    # 256^3 variable-kappa MG-PCG to 1e-10, FP64 and FP32 preconditioner:
    # two iterations of each at full size, scaled by the GPU's iteration
    # counts (the same method to the same tolerance)
    n = 256
    kap = gen.kappa_field(n)
    b = oracle.apply(oracle.KAPPA7, np.ones((n, n, n)), kap)
    r = {}
    for name, f32 in (("fp64", False), ("fp32_precond", True)):
        it = gpu.get("kappa_iters_" + name)
        t0 = tic()
        oracle.pcg(oracle.KAPPA7, b, 4, kap, max_iters=2, fixed_iters=True, precond_f32=f32)
        per = (tic() - t0) / 2
        r[name] = {"s": per * it if it else None, "s_per_iter": per,
                   "sample": "2 iterations at 256^3 x %s iterations (the GPU solve's count)"
                             % it}
    out["kappa_256"] = r
    del kap, b

    # 64 batched variable-kappa problems, forward solve and adjoint: two
    # forward iterations and one gradient on a 64^3 problem (3 levels), per
    # point, scaled by the batch's points and the GPU's iteration counts
    n = 64
    kap = gen.kappa_field(n)
    b = np.ones((n, n, n))
    t0 = tic()
    u, _, _, _ = oracle.pcg(oracle.KAPPA7, b, 3, kap, max_iters=2, fixed_iters=True)
    per_pt_it = (tic() - t0) / 2 / n ** 3
    t0 = tic()
    oracle.kappa_grad(u, u)
    per_pt_grad = (tic() - t0) / n ** 3
    pts = gpu.get("batch_points")
    itf, ita = gpu.get("batch_iters_forward"), gpu.get("batch_iters_adjoint")
    if pts and itf and ita:
        out["batched_adjoint_64"] = {
            "forward_s": per_pt_it * pts * itf, "adjoint_s": per_pt_it * pts * ita +
            per_pt_grad * pts,
            "sample": "2 PCG iterations and one dL/dkappa on a 64^3 problem, per point, x %d "
                      "points x the GPU's largest iteration counts (%d forward, %d adjoint)"
                      % (pts, itf, ita)}
    return out


def oracle_iterations(n):
    """Iterations the oracle's FP64 MG-PCG needs to reach 1e-10 on the n^3
    problem, from the history tests/golden/make_hpcg_pcg_history.py wrote."""
    path = os.path.join(ROOT, "tests", "golden", "hpcg_pcg_history_%d.txt" % n)
    try:
        with open(path) as f:
            vals = [ln for ln in f if ln.strip() and not ln.startswith("#")]
        return len(vals) - 1, "oracle iteration count from tests/golden/" + os.path.basename(path)
    except OSError:
        return None, "no stored oracle history for this size"


def oracle_samples(n):
    """Sample indices and values of the oracle's FP64 MG-PCG solution to 1e-10
    on the n^3 problem (tests/golden/make_hpcg_pcg_samples.py wrote them from
    the oracle alone), or None when no file is stored for this size."""
    path = os.path.join(ROOT, "tests", "golden", "hpcg_pcg_samples_%d_rtol.txt" % n)
    idx, val = [], []
    try:
        with open(path) as f:
            for ln in f:
                if ln.startswith("#") or ln.startswith("h ") or not ln.strip():
                    continue
                p_, v_ = ln.split()
                idx.append(int(p_))
                val.append(float(v_))
    except OSError:
        return None
    return idx, val


def err_vs_oracle_samples(torch, x, samples):
    """max_i |x_i - o_i| / max(|o_i|, 1e-3 max |o|) over the stored samples."""
    if samples is None:
        return None
    idx = torch.tensor(samples[0], dtype=torch.int64, device=x.device)
    g = x.reshape(-1).index_select(0, idx).double().cpu()
    o = torch.tensor(samples[1], dtype=torch.float64)
    den = torch.clamp(o.abs(), min=1e-3 * float(o.abs().max()))
    return float(((g - o).abs() / den).max())


def profile_value(kernel_tag, key, sources=None):
    """A machine-read figure (`- key: value` line) of the committed ncu summary
    profiles/<kernel_tag>.md, or None when the summary is missing or the
    kernel's sources changed since the capture (their sha256 must equal the
    summary's source_sha256)."""
    import hashlib
    sources = SWEEP_SOURCES if sources is None else sources
    path = os.path.join(ROOT, "profiles", "%s.md" % kernel_tag)
    try:
        with open(path) as f:
            txt = f.read()
    except OSError:
        return None, "no ncu summary"
    kv = {}
    for ln in txt.splitlines():
        if ln.startswith("- ") and ":" in ln:
            k, v = ln[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if kv.get("source_sha256") != h.hexdigest():
        return None, "kernel changed since the ncu capture"
    try:
        return float(kv[key]), "ncu capture " + os.path.basename(path)
    except (KeyError, ValueError):
        return None, "no %s in the ncu summary" % key


def sweep_traffic(kernel_tag):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel's sources changed since the capture."""
    return profile_value(kernel_tag, "dram_bytes_per_launch", SWEEP_SOURCES)


# sources of the dominant kernel (its DRAM traffic is invalid once they change)
# (the kernel's code; the shared declarations header is left out so that
# new entry points elsewhere do not void the capture)
SWEEP_SOURCES = ("paper_2204_13304_gb300/csrc/k_wave2.cu",
                 "paper_2204_13304_gb300/csrc/m2s_cta.cuh",
                 "paper_2204_13304_gb300/csrc/m2s_wave_sync.cuh")
SPMV_SOURCES = ("paper_2204_13304_gb300/csrc/k_st27_tma.cu",)

# FP64 operations the 27-point sweep executes per row: the separable box sums
# (row 3-sum, lane-below 2-sum, plane sum) and the update FMA: 8 in a forward
# sweep (which also writes the next sweep's sums), 7 in a backward one.
SWEEP_FP64_OPS_PER_ROW = 7.5


def profile_case(args):
    """--profile-case: a few launches of one kernel on an n^3 grid, for an ncu
    capture (nothing is printed but a marker)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2204_13304_gb300 as m
    n = args.n
    shape = (n, n, n)
    if args.profile_case == "block_ssor":
        import m2s_inputs as gen
        D, L, U, rhs = gen.block_ssor_inputs(n)
        dd, ld, ud = [torch.from_numpy(a_).cuda() for a_ in (D, L, U)]
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.BLOCK7_5x5, mg_levels=1, D=dd, L=ld, U=ud)])
        b = torch.from_numpy(rhs).cuda()
        u = torch.zeros_like(b)
        m.m2s_ssor_sweep(g.handle, b, u, 1.2, 3)
        torch.cuda.synchronize()
        g.close()
        print("profile case block_ssor n=%d done" % n)
        return 0
    if args.profile_case == "block_jac":
        import m2s_inputs as gen
        P, rhs, u0 = gen.block_jac_inputs(shape)
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.BLOCK7_JAC, mg_levels=1, jac=P)])
        b = torch.from_numpy(rhs).cuda()
        u = torch.from_numpy(u0).cuda()
        m.m2s_ssor_sweep(g.handle, b, u, 1.2, 2)
        torch.cuda.synchronize()
        g.close()
        print("profile case block_jac n=%d done" % n)
        return 0
    if args.profile_case == "ilu0":
        # one ILU(0) factorisation (one launch per hyperplane) then one
        # application (two launches per hyperplane), every launch recorded
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.HPCG27, mg_levels=1)])
        m.m2s_ilu0_setup(g.handle)
        r = torch.ones(shape, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        m.m2s_ilu0_apply(g.handle, r, z)
        torch.cuda.synchronize()
        g.close()
        print("profile case ilu0 n=%d done (%d hyperplanes)" % (n, 7 * (n - 1) + 1))
        return 0
    if args.profile_case == "line_btri":
        import m2s_inputs as gen
        blk, rhs = gen.line_btri_inputs(shape)
        b = torch.from_numpy(blk).cuda()
        r = torch.from_numpy(rhs).cuda()
        for a in (0, 1, 2):
            m.m2s_line_btri(b, r, a)
        torch.cuda.synchronize()
        print("profile case line_btri n=%d done" % n)
        return 0
    if args.profile_case == "line_penta":
        import m2s_inputs as gen
        coef, rhs = gen.line_penta_inputs(shape, k=5)
        c = torch.from_numpy(coef).cuda()
        r = torch.from_numpy(rhs).cuda()
        for a in (0, 1, 2):
            m.m2s_line_penta(c, r, a)
        torch.cuda.synchronize()
        print("profile case line_penta n=%d done" % n)
        return 0
    f32 = args.profile_case.endswith("32")
    dt = torch.float32 if f32 else torch.float64
    if args.profile_case.startswith("unit"):
        # one unit column fed by no other unit: W planes (the default unit
        # height, 4 in FP64 and 8 in FP32) of 31 - W rows, so that the 30
        # rows u = y + z of each plane form one unit, and nx = 8192 points
        # per row: the sweep takes nx + 65 + 2 W steps of that unit, which
        # gives the period of one unit-step with no wait on other units
        W = 8 if f32 else 4
        nx, ny, nz = 8192, 31 - W, W
        g = m.Grid([dict(nx=nx, ny=ny, nz=nz, op=m.Op.HPCG27, mg_levels=1,
                         precond_dtype=m.DType.F32 if f32 else m.DType.F64)])
        ones = torch.ones((nz, ny, nx), dtype=dt, device="cuda")
        b = torch.empty_like(ones)
        m.m2s_spmv(g.handle, 0, ones, b)
        x = torch.zeros_like(ones)
        for _ in range(3):
            m.m2s_gs_sweep(g.handle, 0, b, x, m.FORWARD)
        torch.cuda.synchronize()
        m.m2s_sweep_timing(g.handle, True)
        reps = 10
        for _ in range(reps):
            m.m2s_gs_sweep(g.handle, 0, b, x, m.FORWARD)
        torch.cuda.synchronize()
        nl, ms, _ = m.m2s_sweep_timing_read(g.handle, 0)
        m.m2s_sweep_timing(g.handle, False)
        g.close()
        steps = nx + 65 + 2 * W
        print("profile case %s: %d-warp unit, %.1f ns per unit-step (%d sweeps, %.3f ms each)" % (
            args.profile_case, W, ms / max(1, nl) * 1e6 / steps, nl, ms / max(1, nl)))
        return 0
    if args.profile_case.startswith("kappa"):
        import m2s_inputs as gen
        kap = torch.from_numpy(gen.kappa_field(n)).cuda()
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.DIFF7_KAPPA, mg_levels=1, kappa=kap)])
    else:
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.HPCG27, mg_levels=1,
                         precond_dtype=m.DType.F32 if f32 else m.DType.F64)])
    ones = torch.ones(shape, dtype=dt, device="cuda")
    b = torch.empty_like(ones)
    m.m2s_spmv(g.handle, 0, ones, b)
    x = torch.zeros_like(ones)
    for _ in range(3):
        if "sweep" in args.profile_case:
            m.m2s_symgs(g.handle, 0, b, x, 1)
        else:
            m.m2s_spmv(g.handle, 0, b, x)
    torch.cuda.synchronize()
    g.close()
    print("profile case %s n=%d done" % (args.profile_case, n))
    return 0


def time_cuda(torch, fn, reps=1, warm=1):
    """Mean device time of fn() in seconds (CUDA events on the current stream)."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    c.record()
    torch.cuda.synchronize()
    return a.elapsed_time(c) / 1e3 / reps


def other_configs(m, torch, hbm):
    """The other workload configurations of the hot path, measured in the same
    run (synthetic seeded inputs, m2s_inputs): 32^3 SGS-PCG, NPB-LU-shaped
    162^3 x 5 block SSOR, 256^3 variable-kappa MG-PCG in FP64 and with the
    FP32 preconditioner, 64 batched variable-kappa problems with the
    adjoint, and the 1536^3 FP64 symmetric Gauss-Seidel sweep."""
    import numpy as np
    import m2s_inputs as gen
    out = {}

    def guarded(name, fn):
        try:
            out[name] = fn()
        except Exception as e:  # report, keep the bench line
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        torch.cuda.synchronize()

    def cfg1():
        n = 32
        shape = (n, n, n)
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.HPCG27, mg_levels=1)])
        ones = torch.ones(shape, dtype=torch.float64, device="cuda")
        b = torch.empty_like(ones)
        m.m2s_spmv(g.handle, 0, ones, b)
        x = torch.zeros_like(ones)
        t_spmv = time_cuda(torch, lambda: m.m2s_spmv(g.handle, 0, ones, b), 20, 3)
        t_sgs = time_cuda(torch, lambda: m.m2s_symgs(g.handle, 0, b, x, 1), 20, 3)
        xx = torch.empty_like(ones)
        res = [None]

        def pcg():
            res[0] = m.m2s_pcg_solve(g.handle, b, xx, max_iters=50, fixed_iters=True)[1]

        t_pcg = time_cuda(torch, pcg, 3, 1)
        g.close()
        return {"workload": "HPCG 27-point 32^3, b = A*ones: one SpMV, one symmetric GS, "
                            "50 SGS-PCG iterations (FP64)",
                "spmv_us": t_spmv * 1e6, "symgs_us": t_sgs * 1e6, "sgs_pcg_50_ms": t_pcg * 1e3,
                "rel_resid_50": res[0].rel_resid, "bound": "latency (working set in L2)"}

    def cfg4():
        n = 256
        shape = (n, n, n)
        kap = torch.from_numpy(gen.kappa_field(n)).cuda()
        r = {"workload": "variable-kappa 7-point 256^3 (log kappa ~ N(0,1) smoothed, sigma 4), "
                         "b = A*ones, MG-PCG (4 levels) to 1e-10"}
        xs = {}
        for name, pdt in (("fp64", m.DType.F64), ("fp32_precond", m.DType.F32)):
            g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.DIFF7_KAPPA, mg_levels=4, kappa=kap,
                             precond_dtype=pdt)])
            ones = torch.ones(shape, dtype=torch.float64, device="cuda")
            b = torch.empty_like(ones)
            m.m2s_spmv(g.handle, 0, ones, b)
            x = torch.empty_like(ones)
            res = [None]

            def solve():
                res[0] = m.m2s_pcg_solve(g.handle, b, x, max_iters=1000, rtol=1e-10,
                                         fixed_iters=False)[1]

            t = time_cuda(torch, solve, 1, 1)
            if name == "fp64":
                # the 7-point SpMV: read x and the packed kappa record, write y
                sets = [(ones.clone(), torch.empty_like(ones)) for _ in range(3)]
                ts = time_cuda(torch, lambda: [m.m2s_spmv(g.handle, 0, v[0], v[1]) for v in sets],
                               4, 1) / 3
                del sets
                r["spmv7_f64"] = {"ms": ts * 1e3, "alg_GBs": 24.0 * n ** 3 / ts / 1e9,
                                  "hbm_frac": 24.0 * n ** 3 / ts / 1e9 / hbm,
                                  "alg_bytes_note": "24 B/row: x, kappa, y"}
            m.m2s_sweep_timing(g.handle, True)
            solve()
            k, ms, _ = m.m2s_sweep_timing_read(g.handle, 0)
            m.m2s_sweep_timing(g.handle, False)
            xs[name] = x.clone()
            r[name] = {"s": t, "iters": res[0].iters, "rel_resid": res[0].rel_resid,
                       "sweep_ms_256": ms / max(1, k),
                       "max_err_vs_ones": float((x - 1.0).abs().max())}
            g.close()
        r["fp32_precond"]["rel_err_vs_fp64_solution"] = float(
            (xs["fp32_precond"] - xs["fp64"]).abs().max() / xs["fp64"].abs().max())
        r["fp32_precond"]["speedup_vs_fp64"] = r["fp64"]["s"] / r["fp32_precond"]["s"]
        return r

    def cfg3():
        n = 162
        D, L, U, rhs = gen.block_ssor_inputs(n)
        dd, ld, ud = [torch.from_numpy(a).cuda() for a in (D, L, U)]
        del D, L, U
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.BLOCK7_5x5, mg_levels=1, D=dd, L=ld, U=ud)])
        del dd, ld, ud
        b = torch.from_numpy(rhs).cuda()
        u = torch.zeros_like(b)
        m.m2s_ssor_sweep(g.handle, b, u, 1.2, 1)
        u.zero_()
        t = time_cuda(torch, lambda: m.m2s_ssor_sweep(g.handle, b, u, 1.2, 50), 1, 0)
        y = torch.empty_like(b)
        m.m2s_spmv(g.handle, 0, u, y)
        rel = float((b - y).norm() / b.norm())
        pts = n ** 3
        it = t / 50
        g.close()
        return {"workload": "NPB-LU-shaped block SSOR 162^3 x 5 unknowns, omega 1.2, "
                            "50 iterations from u = 0 (FP64)",
                "s_50_iters": t, "ms_per_iter": it * 1e3,
                "alg_GBs": 2440.0 * pts / it / 1e9, "hbm_frac": 2440.0 * pts / it / 1e9 / hbm,
                "alg_bytes_note": "2.44 KB/point/iteration: the fused floor (residual into the "
                                  "lower sweep, update into the upper)",
                "rel_resid_after_50": rel}

    def block_jac_162():
        # NPB-LU-style step: the blocks are formed from u at every step (one
        # pass forms each Jacobian once and scatters its two blocks, a second
        # assembles the residual), then the two block sweeps apply w D^-1
        n = 162
        shape = (n, n, n)
        P, rhs, u0 = gen.block_jac_inputs(shape)
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.BLOCK7_JAC, mg_levels=1, jac=P)])
        b = torch.from_numpy(rhs).cuda()
        u0d = torch.from_numpy(u0).cuda()
        u = u0d.clone()
        m.m2s_ssor_sweep(g.handle, b, u, 1.2, 1)
        u.copy_(u0d)
        steps = 20
        t = time_cuda(torch, lambda: m.m2s_ssor_sweep(g.handle, b, u, 1.2, steps), 1, 0)
        y = torch.empty_like(b)
        m.m2s_spmv(g.handle, 0, u, y)
        rel = float((b - y).norm() / b.norm())
        ta = time_cuda(torch, lambda: m.m2s_spmv(g.handle, 0, u, y), 5, 1)
        g.close()
        pts = n ** 3
        it = t / steps
        # FP64 operations per point: forming pass, residual pass, two sweeps (an
        # FMA one operation; the sweeps' 20 FP64 instructions per lane-step)
        ops_step = 775 + 30 + 2 * 100
        ops_apply = 710 + 175
        return {"workload": "NPB-LU-style block SSOR 162^3 x 5 unknowns with the 5x5 blocks "
                            "formed from u every step (synthetic quadratic-flux Jacobians), "
                            "omega 1.2, %d steps from u0 ~ U(0, 1) (FP64)" % steps,
                "ms_per_step": it * 1e3, "steps": steps,
                "rel_nonlinear_resid_after": rel,
                "apply_ms": ta * 1e3,
                "fp64_ops_per_point": {"step": ops_step, "apply": ops_apply},
                "fp64_op_frac": {"step": ops_step * pts / it / FP64_OPS_PEAK,
                                 "apply": ops_apply * pts / ta / FP64_OPS_PEAK},
                "fp64_ops_note": "per point: the forming pass 775 (D and D u 110, w D^-1 200, "
                                 "three Jacobians with their two blocks and J u 465), the "
                                 "residual pass 30, each sweep 100 (20 per lane-step, 5 lanes); "
                                 "the apply forms all seven blocks itself (710) and applies "
                                 "them (175)",
                "bytes_per_point_step": 80 + 1560 + 240 + 2 * (800 + 80),
                "bytes_note": "the forming pass reads u and b and writes L, U (1200 B), "
                              "w D^-1 (200 B), J u (120 B) and b - D u; the residual pass "
                              "reads those and writes r / w; each sweep reads its 600 B of "
                              "couplings and 200 B of w D^-1; no block outlives its step",
                "parity": "tests/test_gpu_block_jac.py (oracle on ragged and degenerate "
                          "shapes, batches, and one full 162^3 step entry by entry)"}

    def cfg5():
        sides = gen.batch_sides(64)
        kaps = [torch.from_numpy(gen.kappa_field(s_, seed=gen.BASE_SEED + i)).cuda()
                for i, s_ in enumerate(sides)]
        descs = [dict(nx=s_, ny=s_, nz=s_, op=m.Op.DIFF7_KAPPA, mg_levels=3, kappa=k)
                 for s_, k in zip(sides, kaps)]
        g = m.Grid(descs)
        ntot = sum(s_ ** 3 for s_ in sides)
        b = torch.ones(ntot, dtype=torch.float64, device="cuda")
        u = torch.empty_like(b)
        tgt = torch.from_numpy(np.concatenate(
            [gen.target((s_, s_, s_), seed=gen.BASE_SEED + i).ravel()
             for i, s_ in enumerate(sides)])).cuda()
        lam = torch.empty_like(b)
        gk = torch.empty_like(b)
        res = [None, None]

        def fwd():
            res[0] = m.m2s_pcg_solve(g.handle, b, u, max_iters=1000, rtol=1e-10,
                                     fixed_iters=False)[1]

        def adj():
            res[1] = m.m2s_adjoint_solve(g.handle, u, u - tgt, lam, gk, max_iters=1000,
                                         rtol=1e-10)[1]

        tf = time_cuda(torch, fwd, 1, 1)
        ta = time_cuda(torch, adj, 1, 1)
        g.close()
        return {"workload": "64 variable-kappa problems, cube sides from {32,48,64,96,128} by "
                            "seed (%d points), b = 1, MG-PCG (3 levels) to 1e-10, then the "
                            "adjoint solve and dL/dkappa, u_target ~ U(0,1)" % ntot,
                "points": ntot,
                "forward_s": tf, "adjoint_s": ta, "iters_max_forward": res[0].iters,
                "iters_max_adjoint": res[1].iters}

    def symgs_1536():
        n = 1536
        rows = n ** 3
        torch.cuda.empty_cache()
        free, _ = torch.cuda.mem_get_info()
        # b, x (29 GB each) + the grid's Q/26, Q'/26, b/26 (87 GB) + mailboxes (22 GB)
        need = 180 * 2 ** 30
        if free < need:
            return {"skipped": "needs ~170 GB of free device memory (%.0f GB free)"
                               % (free / 2 ** 30)}
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.HPCG27, mg_levels=1)])
        t = {}
        try:
            t["x"] = torch.ones((n, n, n), dtype=torch.float64, device="cuda")
            t["b"] = torch.empty_like(t["x"])
            m.m2s_spmv(g.handle, 0, t["x"], t["b"])
            t["x"].zero_()
            m.m2s_sweep_timing(g.handle, True)
            sec = time_cuda(torch, lambda: m.m2s_symgs(g.handle, 0, t["b"], t["x"], 1), 3, 1)
            k, ms, _ = m.m2s_sweep_timing_read(g.handle, 0)
            m.m2s_sweep_timing(g.handle, False)
            used = torch.cuda.mem_get_info()
        finally:
            g.close()
            t.clear()
            torch.cuda.empty_cache()
        sweep_s = ms / max(1, k) / 1e3
        return {"workload": "HPCG 27-point 1536^3 (%d rows, FP64, 29 GB per vector), b = A*ones: "
                            "symmetric Gauss-Seidel sweeps (forward + backward) from x = 0, the "
                            "paper's SymGS micro-benchmark grid" % rows,
                "ms_per_symgs": sec * 1e3, "ms_per_sweep": sweep_s * 1e3,
                "sweeps_timed": k, "G_point_updates_per_s": 2 * rows / sec / 1e9,
                "alg_GBs": 48.0 * rows / sec / 1e9, "hbm_frac": 48.0 * rows / sec / 1e9 / hbm,
                "alg_bytes_note": "48 B/row per symmetric sweep (read b, x; write x; twice)",
                # the kernel issues ~7.5 FP64 instructions per row and sweep
                # (separable sums: 8 forward, 7 backward), fewer than the
                # definition's 27 operations
                "fp64_pipe_frac_est": 7.5 * rows / sweep_s / FP64_OPS_PEAK,
                "device_GB_held": (used[1] - used[0]) / 2 ** 30,
                "parity": "tests/test_gpu_fullsize.py::test_sweep_1536_f64 (sampled sweep "
                          "identity at this size)"}

    def line_penta_162():
        n, k = 162, 5
        shape = (n, n, n)
        pts = n ** 3
        coefs = [torch.from_numpy(gen.line_penta_inputs(shape, k=k, seed=gen.BASE_SEED + a)[0])
                 .cuda() for a in range(3)]
        _, rhs = gen.line_penta_inputs(shape, k=k, seed=gen.BASE_SEED + 3)
        r = torch.from_numpy(rhs).cuda()
        work = torch.empty(m.m2s_line_penta_work_bytes(n, n, n) // 8, dtype=torch.float64,
                           device="cuda")
        ms = []
        for a in range(3):
            ms.append(time_cuda(torch, lambda: m.m2s_line_penta(coefs[a], r, a, work=work),
                                10, 2) * 1e3)
        t3 = time_cuda(torch, lambda: [m.m2s_line_penta(coefs[a], r, a, work=work)
                                       for a in range(3)], 5, 1)
        ops = (7 + 5 * k) * pts
        return {"workload": "NPB-SP-shaped line solves 162^3 (class C), k = 5 right-hand sides: "
                            "pentadiagonal systems along x, y and z lines (diagonally dominant "
                            "a, e ~ U(-.25,.25), b, d ~ U(-1,1), c ~ U(3,4)), FP64",
                "ms_x": ms[0], "ms_y": ms[1], "ms_z": ms[2], "ms_xyz": t3 * 1e3,
                "alg_GBs_per_axis": [120.0 * pts / (t * 1e-3) / 1e9 for t in ms],
                "alg_bytes_note": "120 B/point per axis solve (read coef, rhs; write v); the "
                                  "kernel also writes and re-reads y and (1/u, u1, e)",
                "fp64_op_frac_per_axis": [ops / (t * 1e-3) / FP64_OPS_PEAK for t in ms],
                "fp64_ops_note": "7 + 5k FP64 operations per point (an FMA is one)",
                "parity": "tests/test_gpu_lines.py (oracle on ragged shapes; sampled equations "
                          "at 162^3)"}

    def line_btri_162():
        n = 162
        shape = (n, n, n)
        pts = n ** 3
        blks = []
        for a in range(3):
            blk, rhs = gen.line_btri_inputs(shape, seed=gen.BASE_SEED + a)
            blks.append(torch.from_numpy(blk).cuda())
            del blk
        r = torch.from_numpy(rhs).cuda()
        work = torch.empty(m.m2s_line_btri_work_bytes(n, n, n) // 8, dtype=torch.float64,
                           device="cuda")
        ms = []
        for a in range(3):
            ms.append(time_cuda(torch, lambda: m.m2s_line_btri(blks[a], r, a, work=work), 5, 1)
                      * 1e3)
        ops = 375.0 * pts
        out_ = {"workload": "NPB-BT-shaped line solves 162^3 (class C): 5x5 block-tridiagonal "
                            "systems along x, y and z lines (B = U(-1,1) + 10 I, A, C ~ "
                            "U(-.25,.25)), 5 unknowns per point, FP64",
                "ms_x": ms[0], "ms_y": ms[1], "ms_z": ms[2],
                "alg_GBs_per_axis": [680.0 * pts / (t * 1e-3) / 1e9 for t in ms],
                "alg_bytes_note": "680 B/point per axis solve (read A, B, C, r; write v); the "
                                  "kernel also writes and re-reads C^ and r^",
                "fp64_op_frac_per_axis": [ops / (t * 1e-3) / FP64_OPS_PEAK for t in ms],
                "fp64_ops_note": "~375 FP64 operations per point (an FMA is one)",
                "parity": "tests/test_gpu_lines.py (oracle on ragged shapes; sampled equations "
                          "at 162^3)"}
        del blks, r, work
        torch.cuda.empty_cache()
        return out_

    def ilu0_256():
        n = 256
        rows = n ** 3
        g = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.HPCG27, mg_levels=1)])
        try:
            t_fac = time_cuda(torch, lambda: m.m2s_ilu0_setup(g.handle), 1, 1)
            gen_t = torch.Generator(device="cuda").manual_seed(5)
            r = torch.rand((n, n, n), dtype=torch.float64, device="cuda", generator=gen_t)
            z = torch.empty_like(r)
            t_app = time_cuda(torch, lambda: m.m2s_ilu0_apply(g.handle, r, z), 5, 2)
        finally:
            g.close()
        hp = (n - 1) * 7 + 1
        return {"workload": "ILU(0) of the HPCG 27-point matrix at 256^3: factorisation and one "
                            "application (forward L, backward U solve), FP64",
                "factor_ms": t_fac * 1e3, "apply_ms": t_app * 1e3,
                "hyperplanes": hp, "launches_per_factor": hp, "launches_per_apply": 2,
                "apply_alg_GBs": 240.0 * rows / t_app / 1e9,
                "apply_hbm_frac": 240.0 * rows / t_app / 1e9 / hbm,
                "alg_bytes_note": "240 B/point per application: the 26 off-diagonal factors and "
                                  "the pivot's reciprocal (216 B), r in, z out, the intermediate y "
                                  "written and re-read",
                "fp64_ops_per_point": 2 * 17,
                "apply_fp64_frac": 34.0 * rows / t_app / FP64_OPS_PEAK,
                "bound_note": "each triangle one persistent wavefront launch (the sweep's "
                              "critical path, 17 FP64 operations per point and triangle); the "
                              "factorisation one launch per hyperplane x + 2y + 4z",
                "parity": "tests/test_gpu_ilu.py (oracle on ragged shapes; sampled (LU)_pq = "
                          "a_pq and L U z = r at 256^3)"}

    guarded("ilu0_256", ilu0_256)
    guarded("line_penta_162x5", line_penta_162)
    guarded("line_btri_162x5", line_btri_162)
    guarded("symgs_1536", symgs_1536)
    guarded("hpcg_32", cfg1)
    guarded("kappa_256", cfg4)
    guarded("block_ssor_162x5", cfg3)
    guarded("block_jac_162x5", block_jac_162)
    guarded("batched_adjoint_64", cfg5)
    return out


def run_reference(args):
    """--impl reference: the serial CPU oracle on the same problem.  A step is
    one iteration of the oracle's MG-PCG solve of the n^3 problem on one host
    core (the oracle as it stands): W iterations untimed, then exactly K
    iterations of a solve from x0 = 0 timed, so ms_per_step x steps is the
    timed run.  value scales the measured time per iteration to the metric,
    seconds per solve to 1e-10, by the oracle's own iteration count for this
    problem (stored by tests/golden/make_hpcg_pcg_history.py)."""
    ws, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    oracle.lib()
    n = args.n
    iters_per_solve, src = oracle_iterations(n)
    if iters_per_solve is None:
        # small grids: the oracle solves the whole problem to count
        _, iters_per_solve, _, _ = oracle.pcg(oracle.HPCG27, oracle.apply(oracle.HPCG27,
                                                                          np.ones((n, n, n))),
                                              4, max_iters=500, rtol=1e-10, fixed_iters=False)
        src = "oracle iteration count of a full oracle solve"
    b = oracle.apply(oracle.HPCG27, np.ones((n, n, n)))
    if args.warmup > 0:
        oracle.pcg(oracle.HPCG27, b, 4, max_iters=args.warmup, fixed_iters=True)
    t0 = time.perf_counter()
    oracle.pcg(oracle.HPCG27, b, 4, max_iters=max(1, args.steps), fixed_iters=True)
    per_iter = (time.perf_counter() - t0) / max(1, args.steps)
    value = per_iter * iters_per_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * 1e3,
        "step": "one iteration of the oracle's MG-PCG solve (%d per solve)" % iters_per_solve,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(n),
        "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": "s",
                         "sample": "%d timed iterations of the oracle's %d^3 MG-PCG solve from "
                                   "x0 = 0 on 1 host core (after %d untimed), x %d iterations "
                                   "per solve (%s)" % (args.steps, n, args.warmup,
                                                       iters_per_solve, src)},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(n):
    return {"workload": "HPCG 27-point operator %d^3 (%d rows), b = A*ones, x0 = 0, FP64 MG-PCG "
                        "(4 levels, 1 pre + 1 post symmetric GS, injection) to rel. residual "
                        "1e-10" % (n, n ** 3),
            "grid": [n, n, n], "mg_levels": 4, "rtol": 1e-10,
            "l2": "inputs larger than L2 (each FP64 vector %d MiB)" % (n ** 3 * 8 >> 20)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--size", "--n", dest="n", type=int, default=256,
                    help="grid points per dimension of the timed problem")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workload configurations (32^3 SGS-PCG, block SSOR, "
                         "variable-kappa, batched adjoint, line solves, 1536^3 SymGS)")
    ap.add_argument("--profile-case", choices=["sweep64", "sweep32", "unit64", "unit32",
                                               "spmv64", "spmv32",
                                               "kappa_sweep64", "block_ssor", "block_jac", "line_penta",
                                               "line_btri", "ilu0"],
                    help="run a few launches of one kernel for an ncu capture and exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args)

    import numpy as np
    import torch

    ws, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2204_13304_gb300 as m

    n = args.n
    shape = (n, n, n)
    stream = torch.cuda.current_stream()
    g64 = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.HPCG27, mg_levels=4, precond_dtype=m.DType.F64)])
    g32 = m.Grid([dict(nx=n, ny=n, nz=n, op=m.Op.HPCG27, mg_levels=4, precond_dtype=m.DType.F32)])
    ones = torch.ones(shape, dtype=torch.float64, device="cuda")
    b = torch.empty_like(ones)
    m.m2s_spmv(g64.handle, 0, ones, b)
    x = torch.empty_like(ones)

    def solve(g):
        st, res = m.m2s_pcg_solve(g.handle, b, x, max_iters=500, rtol=1e-10, fixed_iters=False,
                                  check_every=1)
        return st, res

    # warm-up
    for _ in range(args.warmup):
        st, res64 = solve(g64)
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the sweep kernels of the timed solves are bracketed by CUDA events on
    # the stream they are launched on (the dominant kernel's live timing)
    m.m2s_sweep_timing(g64.handle, True)
    e0.record(stream)
    for _ in range(args.steps):
        st, res64 = solve(g64)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    t64 = e0.elapsed_time(e1) / 1e3 / args.steps
    # whole-job time per solve: the slowest rank's time over all ranks' solves
    value = job_value(ws, t64)
    sweep_lv = [m.m2s_sweep_timing_read(g64.handle, lv) for lv in range(4)]
    m.m2s_sweep_timing(g64.handle, False)
    clk = clocks.stop()
    x64 = x.clone()
    # the fixed-iteration form of the same workload: 50 MG-PCG iterations
    t50 = time_cuda(torch, lambda: m.m2s_pcg_solve(g64.handle, b, x, max_iters=50,
                                                   fixed_iters=True), 1, 1)

    # FP32-preconditioned form on the same problem
    for _ in range(max(1, args.warmup // 2)):
        st32, res32 = solve(g32)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        st32, res32 = solve(g32)
    e1.record(stream)
    torch.cuda.synchronize()
    t32 = e0.elapsed_time(e1) / 1e3 / args.steps
    err32 = float((x - x64).abs().max() / x64.abs().max())
    err64_ones = float((x64 - 1.0).abs().max())
    # both solutions per entry against the oracle's at its stored samples
    osamp = oracle_samples(n)
    eo64 = err_vs_oracle_samples(torch, x64, osamp)
    eo32 = err_vs_oracle_samples(torch, x, osamp)

    # per-kernel timings (CUDA events on the launching stream)
    def time_op(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        c.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(c) / 1e3 / reps

    def time_rotating(fn, sets, reps=12):
        """fn(set) back to back over vector sets taken in turn, more bytes in
        all than the L2 holds: every launch reads its input from DRAM and the
        write-back of the outputs is paid inside the timed launches."""
        for v in sets:
            fn(v)
        torch.cuda.synchronize()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for i in range(reps):
            fn(sets[i % len(sets)])
        c.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(c) / 1e3 / reps

    xs = torch.zeros_like(ones)
    ys = torch.empty_like(ones)
    sets64 = [(x64.clone(), torch.empty_like(x64)) for _ in range(3)]
    t_spmv = time_rotating(lambda v: m.m2s_spmv(g64.handle, 0, v[0], v[1]), sets64)
    del sets64
    # one sweep = (10 symmetric GS - 1 symmetric GS) / 18: removes the
    # one-off old-neighbour-sum kernel that starts m2s_symgs
    t_sweep64 = (time_op(lambda: m.m2s_symgs(g64.handle, 0, b, xs, 10), 2) -
                 time_op(lambda: m.m2s_symgs(g64.handle, 0, b, xs, 1), 2)) / 18
    b32 = b.float()
    xs32 = torch.zeros_like(b32)
    ys32 = torch.empty_like(b32)
    sets32 = [(b32.clone(), torch.empty_like(b32)) for _ in range(4)]
    t_spmv32 = time_rotating(lambda v: m.m2s_spmv(g32.handle, 0, v[0], v[1]), sets32)
    del sets32
    t_sweep32 = (time_op(lambda: m.m2s_symgs(g32.handle, 0, b32, xs32, 10), 2) -
                 time_op(lambda: m.m2s_symgs(g32.handle, 0, b32, xs32, 1), 2)) / 18
    rows = n ** 3
    hbm, peak_kind = peaks()
    kern = {
        "spmv27_f64": {"ms": t_spmv * 1e3, "alg_GBs": 16 * rows / t_spmv / 1e9},
        "symgs_sweep_f64": {"ms": t_sweep64 * 1e3, "alg_GBs": 24 * rows / t_sweep64 / 1e9,
                            "alg_fp64_Gops": 27 * rows / t_sweep64 / 1e9},
        "spmv27_f32": {"ms": t_spmv32 * 1e3, "alg_GBs": 8 * rows / t_spmv32 / 1e9},
        "symgs_sweep_f32": {"ms": t_sweep32 * 1e3, "alg_GBs": 12 * rows / t_sweep32 / 1e9},
    }
    # dominant kernel of the FP64 solve: the Gauss-Seidel sweep on the finest
    # level.  Its roofline is HBM: 24 algorithmic bytes per row (read b and
    # x, write x), the launch duration the live event timing of the sweeps
    # inside the timed solves, against the measured copy bandwidth.  The
    # sweep is bound by its critical path (7(n-1) dependent point updates)
    # and the FP64 issue rate, so the same launch is also stated against the
    # FP64 issue peak on the FP64 operations the kernel executes.
    n_l0, ms_l0, _ = sweep_lv[0]
    t_launch = ms_l0 / 1e3 / max(1, n_l0)
    alg_bytes = 24 * rows
    ach = alg_bytes / t_launch / 1e9
    traffic, traffic_src = sweep_traffic("gs27_cta_kernel_f64_%d" % n)
    fp64_warp_inst, fp64_src = profile_value("gs27_cta_kernel_f64_%d" % n,
                                             "fp64_warp_instructions_per_launch")
    useful = SWEEP_FP64_OPS_PER_ROW * rows
    fp64 = {"useful_fp64_ops_per_row": SWEEP_FP64_OPS_PER_ROW,
            "useful_achieved": useful / t_launch / 1e9,
            "peak": FP64_OPS_PEAK / 1e9, "unit": "G FP64 op/s",
            "useful_frac": useful / t_launch / FP64_OPS_PEAK,
            "issued_lane_slots_frac": (fp64_warp_inst * 32 / t_launch / FP64_OPS_PEAK
                                       if fp64_warp_inst else None),
            "issued_source": fp64_src,
            "note": "FP64 operations the kernel executes per row (separable 3x3x3 sums: 8 in "
                    "a forward sweep, 7 in a backward one), not the definition's 27; the "
                    "issued fraction counts every lane slot of the FP64 warp instructions "
                    "ncu counted (idle halo and ramp lanes included); peak 152 SMs x 2 FP64 "
                    "lanes/clk x 2.07 GHz (derived)"}
    roof = {"kernel": "gs27_cta_kernel (FP64 Gauss-Seidel sweep, %d^3 level)" % n,
            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "traffic": traffic, "traffic_source": traffic_src,
            "alg_bytes_per_launch": alg_bytes,
            "alg_bytes_note": "24 B/row: read b and x, write x (the kernel moves 32 B/row: it "
                              "reads the pre-scaled old-neighbour sums Q/26 and b/26 and writes "
                              "x and the next sweep's Q'/26)",
            "launches_timed": n_l0, "ms_per_launch": t_launch * 1e3,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind,
            "fp64_issue": fp64}
    # the SpMV the metric names: HBM rooflines of the FP64 and FP32 forms
    spmv_roofs = {}
    for tag, t_k, bpr in (("spmv27_f64", t_spmv, 16), ("spmv27_f32", t_spmv32, 8)):
        traf, tsrc = profile_value("st27_tma_kernel_%s_%d" % (tag[-3:], n),
                                   "dram_bytes_per_launch", SPMV_SOURCES)
        a_ = bpr * rows / t_k / 1e9
        spmv_roofs[tag] = {"bound": "hbm", "achieved": a_, "peak": hbm, "unit": "GB/s",
                           "frac": a_ / hbm, "traffic": traf, "traffic_source": tsrc,
                           "ms_per_launch": t_k * 1e3,
                           "alg_bytes_per_launch": bpr * rows,
                           "alg_bytes_note": "%d B/row: read x, write y" % bpr}
    spmv_roofs["spmv27_f64"]["fp64_useful_frac"] = 6.4 * rows / t_spmv / FP64_OPS_PEAK
    # the residual restriction of the V-cycle's finest level (256^3 -> 128^3):
    # read z (8 B/fine row; the 3x3x3 boxes around the even points cover it)
    # and r at the even points, write r_c and r_c/26: ~11 B per fine row
    rc = torch.empty(((n + 1) // 2,) * 3, dtype=torch.float64, device="cuda")
    sets_r = [(b.clone(), x64.clone()) for _ in range(2)]
    t_restrict = time_rotating(lambda v: m.m2s_mg_restrict(g64.handle, 0, v[0], v[1], rc), sets_r)
    del sets_r
    a_r = 11.0 * rows / t_restrict / 1e9
    spmv_roofs["restrict27_f64"] = {"bound": "hbm", "achieved": a_r, "peak": hbm, "unit": "GB/s",
                                    "frac": a_r / hbm, "ms_per_launch": t_restrict * 1e3,
                                    "alg_bytes_note": "11 B per fine row: z, r at the even points, "
                                                      "r_c and r_c/26 written",
                                    "fp64_useful_frac": 28 * rows / 8 / t_restrict / FP64_OPS_PEAK}
    sweep_share = sum(v[1] for v in sweep_lv) / 1e3 / args.steps / t64

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        bh = b.cpu().pin_memory()
        xh = torch.empty(shape, dtype=torch.float64).pin_memory()
        bd = torch.empty_like(b)
        xd = torch.empty_like(b)

        def e2e_step():
            bd.copy_(bh, non_blocking=True)
            m.m2s_pcg_solve(g64.handle, bd, xd, max_iters=500, rtol=1e-10, fixed_iters=False)
            xh.copy_(xd, non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        te = (time.perf_counter() - t0) / args.steps
        e2e = {"value": job_value(ws, te), "unit": "s", "h2d_bytes_per_step": rows * 8,
               "d2h_bytes_per_step": rows * 8}

    # the other workloads are measured on one GPU (rank 0)
    configs = None if (args.no_configs or rank != 0) else other_configs(m, torch, hbm)
    launches = launches_per_solve(res64.iters)
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t64 * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (HPCG operator, b = A*ones)", "config": workload_config(n),
        "iters_fp64": res64.iters, "rel_resid_fp64": res64.rel_resid,
        "fp64_50_iterations_s": t50,
        "max_err_vs_ones_fp64": err64_ones,
        "err_vs_oracle_samples_fp64": eo64,
        "fp32_precond": {"value": t32, "unit": "s", "iters": res32.iters,
                         "rel_resid": res32.rel_resid, "rel_err_vs_fp64_solution": err32,
                         "err_vs_oracle_samples": eo32,
                         "speedup_vs_fp64": t64 / t32},
        "kernels": kern, "sweep_share_of_solve": sweep_share,
        "sweep_ms_per_launch_by_level": [v[1] / max(1, v[0]) for v in sweep_lv],
        "roofline": roof, "roofline_spmv": spmv_roofs, "e2e": e2e, "gpu_launches": launches * args.steps,
        "other_configs": configs,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        per_iter, reps = cpu_baseline(n)
        oit, src = oracle_iterations(n)
        if oit is None:
            oit, src = res64.iters, "iteration count of the GPU solve"
        line["cpu_baseline"] = {"value": per_iter * oit, "unit": "s", "cores": 1,
                                "kind": "oracle",
                                "sample": "the first %d iterations of the oracle's %d^3 MG-PCG "
                                          "solve on one host core, x %d iterations (%s)"
                                          % (reps, n, oit, src)}
        if configs:
            gpu_counts = {}
            try:
                gpu_counts["kappa_iters_fp64"] = configs["kappa_256"]["fp64"]["iters"]
                gpu_counts["kappa_iters_fp32_precond"] = \
                    configs["kappa_256"]["fp32_precond"]["iters"]
            except (KeyError, TypeError):
                pass
            try:
                c5 = configs["batched_adjoint_64"]
                gpu_counts.update(batch_points=c5["points"],
                                  batch_iters_forward=c5["iters_max_forward"],
                                  batch_iters_adjoint=c5["iters_max_adjoint"])
            except (KeyError, TypeError):
                pass
            line["cpu_baseline"]["other_configs"] = oracle_config_times(gpu_counts)
    if rank == 0:
        print(json.dumps(line))
    g64.close()
    g32.close()
    if ws > 1:
        import torch.distributed as dist
        barrier(ws)
        dist.destroy_process_group()
    return 0


def launches_per_solve(iters, levels=4):
    """Kernels of one FP64 MG-PCG solve: setup (r/26, dot, finalize) then per
    iteration the V-cycle (per non-coarsest level 2 + 2 sweeps, restriction,
    fused prolongation; coarsest 2 sweeps), finalize(rho), p-update+SpMV+dot,
    finalize(pq), update+|r|, finalize(rr)."""
    per_v = (levels - 1) * 6 + 2
    return 3 + iters * (per_v + 5)


if __name__ == "__main__":
    sys.exit(main())
