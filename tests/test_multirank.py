"""The N > 1 path of bench.py on CPU: replicas under torchrun, one process
per rank over gloo on 127.0.0.1 (host logic only; no GPU work)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    got = bench.max_over_ranks(values[rank], True)
    dist.barrier()
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"max": got}, f)
    dist.destroy_process_group()


def test_slowest_replica_time_reaches_every_rank(tmp_path):
    world, values = 2, [3.5, 7.25]
    mp.spawn(_rank_main, args=(world, free_port(), values, str(tmp_path)), nprocs=world,
             join=True)
    for r in range(world):
        with open(tmp_path / f"r{r}.json") as f:
            assert json.load(f)["max"] == max(values)


def test_replicas_value_sums_ranks():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, False) == 2.5
    # two ranks, 2^28 characters each in 100 ms: 2 * 268435456 / 0.1 s
    assert bench.replicas_value(1 << 28, 2, 100.0) == pytest.approx(5368.70912)


def test_reference_arm_under_torchrun_prints_once():
    """Rank 0 alone times the oracle and prints one line; the other rank
    exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
