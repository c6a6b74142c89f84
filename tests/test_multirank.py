"""The multi-rank path of bench.py on CPU: two gloo ranks.

On N GPUs every rank runs an independent replica (the solve does not shard),
and bench.py reports the units of all ranks over the slowest rank's time.
These tests run that host logic with world size 2 on the gloo backend: the
cross-rank aggregation, and the reference arm's rule that only rank 0 works
and prints.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _aggregate_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]                     # rank 1 is the slow one
        units = [1000, 3000][rank]
        t, u = bench.aggregate_over_ranks(ms, units)
        out.put((rank, t, u))
    finally:
        dist.destroy_process_group()


def test_aggregate_over_ranks_max_time_sum_units_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_aggregate_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time and the units of both
    assert res == [(0, 20.0, 4000.0), (1, 20.0, 4000.0)]
    # whole-job throughput as bench.py reports it
    assert 4000.0 / (20.0 / 1e3) == 200000.0


def test_aggregate_without_process_group_is_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(7.0, 123) == (7.0, 123.0)


def test_reference_arm_only_rank0_prints(tmp_path):
    """`bench.py --impl reference` under torchrun: rank 1 exits 0 without work
    or output (rank 0 would time the oracle, which this test does not run)."""
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
