"""The N > 1 host logic of bench.py on CPU: world_size-2 gloo ranks, each
with its own (replica) point set; the job value uses the slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank: a replica problem with its own seed and its own step time
    w = dict(bench.WORKLOADS["uniform2d_10k"])
    P = bench.gen_points(w, seed_offset=rank)
    ms = 10.0 + 5.0 * rank
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    q.put((rank, float(P[0, 0]), ms_max, bench.job_value(w["n"], world, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] != out[1][1]                       # replicas draw different points
    assert out[0][2] == out[1][2] == 15.0               # max over ranks
    assert out[0][3] == pytest.approx(2 * 10_000 / 0.015 / 1e6)
