"""The N > 1 benchmark path on CPU: two gloo ranks, each a replica with its
own view; the only collective is the max of the timed region, and the
whole-job throughput counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2203_11484_gb300 import workloads as W
        ws, r, _ = bench._dist()
        seed = bench.replica_seed(1, r)
        cam = W.room200k_workload(width=64, height=64, seed=seed).views[0].camera
        my_ms = 100.0 + 50.0 * r                      # rank 1 is slower
        slowest = bench.max_over_ranks(my_ms, "cpu")
        out[r] = (ws, seed, tuple(cam.eye), slowest, bench.job_throughput(1000, 4, ws, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2
    assert res[0][1] != res[1][1] and res[0][2] != res[1][2]      # different views
    assert res[0][3] == res[1][3] == 150.0                        # both see the slowest rank
    assert res[0][4] == res[1][4] == 1000 * 4 * 2 / 0.15
