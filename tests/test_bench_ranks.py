"""The bench's multi-rank bookkeeping (replicas, no data-path collective) with two
gloo ranks on the CPU: the step time is the slowest rank's, the value counts every
rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 2.0 + rank          # rank 1 is the slower replica
        slowest = bench.max_over_ranks(ms)
        out[rank] = (slowest, bench.job_value(1000.0, world, slowest), bench.dist_env())
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        slowest, value, env = out[r]
        assert slowest == 3.0
        assert value == pytest.approx(2 * 1000.0 / 3e-3)
        assert env == (r, r, world)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.job_value(10.0, 1, 2.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the oracle timing (the reference arm) runs on rank 0 only;
    the other ranks exit 0 without output."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
