"""The multi-GPU form of bench.py (independent replicas, weak scaling) on
CPU: two gloo ranks, each with its own seeded series, combine their step
times the way bench.py does (max over ranks, whole-job units)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl = bench.workload(rank, n=20000)
    local_ms = 100.0 * (rank + 1)            # rank 1 is the slow one
    value, total = bench.combine(local_ms, 1000, 5, world)
    out[rank] = (value, total, float(wl.series[0, :10].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_bench():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    v0, t0, s0 = out[0]
    v1, t1, s1 = out[1]
    assert t0 == t1 == 200.0                 # max over ranks
    assert v0 == pytest.approx(world * 1000 * 5 / 0.2)
    assert s0 != s1                          # each rank searches its own series


def test_reference_arm_under_torchrun_prints_once():
    # two ranks: rank 0 times the oracle and prints one line, rank 1 exits 0
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] == pytest.approx(d["cpu_baseline"]["value"])
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
