"""The benchmark's multi-rank path on CPU (gloo, world size 2): replicas with
no data-path collective; the job's time is the slowest rank's (max over
ranks) and the job's throughput counts every rank's rays."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, lr = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    dist.barrier()
    # rank-dependent "timed region": rank 1 is the slower replica
    seconds = 0.5 + 0.25 * r
    slowest = bench.max_over_ranks(seconds, dist, "cpu")
    rate = bench.job_rate(1000.0, w, slowest)
    out[r] = (r, w, lr, slowest, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_count_all_rays():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        rank, w, lr, slowest, rate = out[r]
        assert (rank, w, lr) == (r, world, r)
        assert slowest == pytest.approx(0.75)
        assert rate == pytest.approx(2 * 1000.0 / 0.75)


def test_single_process_defaults():
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.job_rate(10.0, 1, 2.0) == 5.0
