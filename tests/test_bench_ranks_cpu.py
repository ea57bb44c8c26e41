"""The multi-GPU form of bench.py is "replicas only" (one cell does not
shard): each rank solves its own replica and the job's figures are the
slowest rank's time and all ranks' voxel-iterations.  These checks run the
rank logic as two gloo processes on the CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, vox = bench.combine_ranks(10.0 * (rank + 1), 100.0 * (rank + 1), world)
    out[rank] = (ms, vox)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_takes_the_slowest_time_and_all_work():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (20.0, 300.0)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_profiling_shape_names_its_workload_and_drops_traffic():
    """--shape runs a box-shaped regeneration under its own workload name; the
    committed per-launch traffic belongs to the 256^3 workload only."""
    import argparse
    import bench
    a = argparse.Namespace(n=256, cells=200, shape="256,128,128", gpus=1)
    cfg = bench._config(a)
    assert cfg["workload"] == "voronoi200-256x128x128" and cfg["n"] == [256, 128, 128]
    assert bench._traffic("pass_a", cfg["workload"]) is None
    b = argparse.Namespace(n=256, cells=200, shape=None, gpus=1)
    assert bench._config(b)["workload"] == "voronoi200-256^3"
