"""The N > 1 path of bench.py on CPU (gloo, world size 2): replicas only, the
job time is the slowest rank's, the value counts every rank's work, only rank
0 prints, and the reference arm runs on rank 0 alone."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    r, w = bench.dist_init(world)
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
    t = bench.max_over_ranks(local_ms, w)
    v = bench.job_value(w, 1000.0, t)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": t, "value": v}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    got = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for g in got:
        assert g["max"] == 15.0                       # both ranks see the slowest time
        assert abs(g["value"] - 2 * 1000.0 / 15e-3) < 1e-6


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_init(1) == (0, 1)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(1, 2e6, 2.0) == pytest.approx(1e9)
