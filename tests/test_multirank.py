"""The multi-rank host logic of the bench on CPU (gloo, world size 2): the path does not
shard, so N ranks run N replicas, and the whole-job numbers are the slowest rank's time
and the units of all ranks together."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, units, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.aggregate(ms[rank], units[rank], world, torch.device("cpu"))
        out[rank] = (t, u)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks_max_time_sum_units():
    ms, units = [12.5, 17.25], [3.0e6, 5.0e6]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, _free_port(), ms, units, out), nprocs=2,
                           start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        assert res[r] == (17.25, 8.0e6)


def test_aggregate_single_rank_is_identity():
    assert bench.aggregate(3.5, 7.0, 1, None) == (3.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle on the host cores) runs on rank 0;
    the other ranks exit 0 without work or output."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120, cwd=root)
    assert r.returncode == 0 and r.stdout.strip() == ""
