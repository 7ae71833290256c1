"""The multi-GPU path of bench.py on the CPU: two ranks over gloo.  The
solve does not shard (replicas only), so what runs across ranks is the
host logic: the barriers around the timed region, the max over ranks of the
time, and rank 0 alone printing the line (the reference arm included)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_init(None, backend="gloo")
    bench.barrier(w)
    t = 1.0 + r  # rank r "took" 1 + r seconds per solve
    out[r] = (bench.max_over_ranks(w, t), bench.job_value(w, t))
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_ranks_max_and_job_value():
    import torch.multiprocessing as mp
    ws, port = 2, free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    # every rank sees the slowest rank's time; the job value counts both
    # ranks' solves
    assert res[0] == res[1] == (2.0, 1.0)


def test_reference_arm_under_torchrun_prints_once():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--size", "12"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
