"""The multi-GPU form of the bench is replicas: each rank times its own batch and the job's
figure is the slowest rank's time and all ranks' frames (frames are independent, so there is no
data-path collective).  The aggregation runs here on two CPU ranks over gloo."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_info()
    assert (r, w) == (rank, world)
    # rank k's batch took 100 + 50 k ms for 256 frames x 4 steps
    job_ms, fps = bench.job_throughput(100.0 + 50.0 * rank, 256 * 4, world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{job_ms} {fps}\n")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replica_throughput_takes_the_slowest_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for rank in range(world):
        job_ms, fps = map(float, open(tmp_path / f"rank{rank}.txt").read().split())
        assert job_ms == 150.0  # the slower rank
        assert fps == pytest.approx(world * 256 * 4 / 0.150)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(200.0, 512, 1) == (200.0, pytest.approx(2560.0))


def test_reference_arm_prints_on_rank_zero_only():
    # a non-zero rank of the reference arm exits 0 without work or output
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
