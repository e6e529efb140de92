"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): every
rank reconstructs its own scan (replicas, no data-path collective); the job's
time per scan is the slowest rank's time over all ranks' scans."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slower one
    t = bench.job_seconds_per_scan(local_ms, 5, world, dist, "cpu")
    out[rank] = (t, bench.rank_noise_seed(4, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_time_is_max_over_ranks_and_scans_differ():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    t0, seed0 = out[0]
    t1, seed1 = out[1]
    assert t0 == t1 == pytest.approx(200.0 / 1e3 / (5 * 2))
    assert seed0 == 4 and seed1 != seed0


def test_single_rank_needs_no_collective():
    import bench
    assert bench.job_seconds_per_scan(500.0, 5, 1) == pytest.approx(0.1)
