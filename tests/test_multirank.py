"""Host logic of the N-process benchmark, on two gloo ranks on the CPU:
the pose partition, the max-over-ranks time and the whole-job rate.  The
path shards by independent frames (replicas, no data-path collective), so
these are the only cross-rank steps."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    poses = [bench.rank_pose(k, world, rank, 20) for k in range(40)]
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    dist.barrier()
    q.put((rank, poses, t))
    dist.destroy_process_group()


def test_pose_partition_single_rank():
    assert [bench.rank_pose(k, 1, 0, 20) for k in range(25)] == [k % 20 for k in range(25)]
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(100, 1, 200.0) == pytest.approx(500.0)


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict((r, (poses, t)) for r, poses, t in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time
    assert out[0][1] == out[1][1] == 15.0
    # per step the two ranks render different poses, and each covers half the orbit per cycle
    for k in range(40):
        assert out[0][0][k] != out[1][0][k]
    assert set(out[0][0][:10]) | set(out[1][0][:10]) == set(range(20))
    assert bench.whole_job_rate(1000, world, 2000.0) == pytest.approx(1000.0)
