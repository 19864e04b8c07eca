"""The N > 1 path of bench.py on CPU processes (gloo, world size 2): the
timed region is reduced to its maximum over ranks and the whole-job rate
counts every rank's replica; under a two-rank launch the reference arm
prints one JSON line from rank 0 and the other rank exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist)
    rate = bench.whole_job_rate(1000, world, ms / 4)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms, "rate": rate}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    # both ranks see the slower rank's 20 ms; 2 replicas x 1000 evals per 5 ms step
    assert [g["ms"] for g in got] == [20.0, 20.0]
    assert [g["rate"] for g in got] == [400000.0, 400000.0]
    import bench
    assert bench.max_over_ranks(7.5) == 7.5


def test_reference_arm_under_two_rank_launch():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    for key in ("metric", "value", "unit", "ms_per_step", "higher_is_better", "scaling",
                "dtype", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
