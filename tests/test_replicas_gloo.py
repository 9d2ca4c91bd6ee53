"""The multi-process path of bench.py on CPU, world size 2 over gloo.  The path shards nothing (every GPU runs
its own replica of the workload, no data-path collective), so what N > 1 adds is bookkeeping:

* the whole-job figures take the slowest rank's times (max over ranks) and every rank's points (sum);
* every rank runs rank 0's launch-mode choice;
* the reference arm under torchrun prints one line from rank 0, and the other ranks exit 0 without work.
"""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _replica(rank: int, world: int, port: int):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = load_bench()
        # rank r: timed region 10 + r ms, end to end 20 - r ms, 1000 (r + 1) points
        total, e2e, pts = bench.combine_ranks(world, 10.0 + rank, 20.0 - rank, 1000.0 * (rank + 1))
        assert (total, e2e, pts) == (10.0 + world - 1, 20.0, 1000.0 * world * (world + 1) / 2), (total, e2e, pts)
        # rank 0 says yes, the others no: all take yes; and the other way round
        assert bench.rank0_choice(world, rank == 0) is True
        assert bench.rank0_choice(world, rank != 0) is False
    finally:
        torch.distributed.destroy_process_group()


def test_replica_figures_over_gloo():
    mp.start_processes(_replica, args=(2, free_port()), nprocs=2, join=True, start_method="spawn")


def test_one_rank_is_the_local_figures():
    bench = load_bench()
    assert bench.combine_ranks(1, 3.0, 4.0, 5.0) == (3.0, 4.0, 5.0)
    assert bench.rank0_choice(1, False) is False


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference", "--workload", "cfg0",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
