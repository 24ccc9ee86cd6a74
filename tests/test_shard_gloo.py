"""The sharded divide-and-conquer bookkeeping (partition owners, the point
all-to-all, the occupancy OR, the border gather into the root) on CPU with
two gloo ranks.  Each rank holds half of the points; the triangulation steps
on the ranks are the oracle's (this is a test of the data movement), and the
root's merge must reproduce DT(P) exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1902_07554_gb300 import shard


def test_assign_partitions_balanced_and_deterministic():
    sizes = np.array([50, 10, 40, 40, 30, 30, 20, 5])
    own = shard.assign_partitions(sizes, 3)
    assert own.tolist() == shard.assign_partitions(sizes, 3).tolist()
    load = np.bincount(own, weights=sizes, minlength=3)
    assert load.sum() == sizes.sum() and load.max() - load.min() <= sizes.max()
    # largest first onto the lightest rank: 50 -> 0, 40 -> 1, 40 -> 2, 30 -> 1, 30 -> 2, 20 -> 0, 10 -> 0, 5 -> 1
    assert own.tolist() == [0, 0, 1, 2, 1, 2, 0, 1]
    order, counts = shard.route(np.array([3, 0, 7, 2, 0]), own, 3)
    assert counts.tolist() == [2, 2, 1] and order.tolist() == [1, 4, 2, 3, 0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    import pointsets
    from oracle import divide as dv
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, D, k = 1200, 2, 5
        P = pointsets.uniform(n, D, 77)
        local = np.arange(rank * n // world, (rank + 1) * n // world)
        # the same sample, sample graph and blocks on every rank
        ids = dv.sample_ids(n, dv.sample_size(n, 0.03, D), 1)
        PS = P[ids]
        E, w = dv.sample_graph(PS, ids)
        block = dv.partition(PS, E, w, k)
        lab_local = dv.labels(P, PS, ids, block, idx=local)
        sizes = shard.partition_sizes(dist, lab_local, k)
        owner = shard.assign_partitions(sizes, world)
        coords, gids, labs = shard.exchange_points(dist, P[local], local, lab_local, owner)
        full = dv.labels(P, PS, ids, block)
        mine = np.nonzero(owner[full] == rank)[0]
        exchange_ok = (sorted(gids.tolist()) == mine.tolist() and np.array_equal(coords, P[gids])
                       and np.array_equal(labs, full[gids]) and np.array_equal(sizes, np.bincount(full, minlength=k)))
        # occupancy of an 8 x 8 grid by partition (bit i = partition i), OR over ranks
        cell = np.minimum((coords * 8).astype(np.int64), 7) @ np.array([1, 8])
        masks = np.zeros(64, dtype=np.int64)
        np.bitwise_or.at(masks, cell, np.left_shift(1, labs))
        occ = shard.allreduce_occupancy(dist, masks)
        want_occ = np.zeros(64, dtype=np.int64)
        np.bitwise_or.at(want_occ, np.minimum((P * 8).astype(np.int64), 7) @ np.array([1, 8]),
                         np.left_shift(1, full))
        occ_ok = np.array_equal(occ, want_occ)
        # each rank: its partitions' DTs and exact border simplices (Alg. 1)
        keep, brows, vb = [], [], []
        for i in sorted(set(labs.tolist())):
            pid = np.sort(gids[labs == i])
            others = np.nonzero(full != i)[0]
            _, v, _ = oracle.delaunay(P[pid], pid, mesh=True)
            for row in v:
                fin = tuple(sorted(int(pid[x]) for x in row if x >= 0))
                if dv._is_border(P, pid, row, others):
                    vb.extend(fin)
                    if len(fin) == D + 1:
                        brows.append(fin)
                elif len(fin) == D + 1:
                    keep.append(fin)
        keep_all = shard.gather_to_root(dist, np.array(keep, dtype=np.int64).reshape(-1, D + 1))
        b_all = shard.gather_to_root(dist, np.array(brows, dtype=np.int64).reshape(-1, D + 1))
        vb_all = shard.gather_to_root(dist, np.unique(np.array(vb, dtype=np.int64)))
        merged_ok = None
        if rank == 0:
            VB = np.unique(vb_all)
            Bset = {tuple(r) for r in b_all.tolist()}
            rows = {tuple(r) for r in keep_all.tolist()}
            for s in oracle.delaunay(P[VB], VB).tolist():
                if len(set(full[s].tolist())) > 1 or tuple(s) in Bset:
                    rows.add(tuple(s))
            got = np.array(sorted(rows), dtype=np.int64)
            merged_ok = bool(np.array_equal(got, oracle.delaunay(P))) and len(VB) > 0
        q.put((rank, exchange_ok, occ_ok, merged_ok, len(gids)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_exchange_gather_merge():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(o[1] for o in out), "points did not reach their partitions' owners"
    assert all(o[2] for o in out), "occupancy OR"
    assert out[0][3] is True, "the root's merge of the gathered border did not reproduce DT(P)"
    assert out[0][4] + out[1][4] == 1200 and min(out[0][4], out[1][4]) > 0
