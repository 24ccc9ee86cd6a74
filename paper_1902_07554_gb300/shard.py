"""Host-side bookkeeping of the divide-and-conquer path sharded over G GPUs.

The k partitions of Alg. 1 are independent until the merge, so the path
shards by partition (one process per GPU, torch.distributed):

1. every rank holds a slice of P (its global index range) and draws the same
   sample (the sample indices depend only on n, eta and the seed); the sample
   points are all-gathered, and every rank triangulates and partitions the
   sample itself (a few thousand points: cheaper than shipping the result);
2. every rank labels its slice (Alg. 2, assignment of the points);
3. partitions are assigned to ranks (`assign_partitions`, about k / G each,
   balanced by point count) and the points go to their partition's owner in
   one all-to-all (`exchange_points`); each rank receives its points with
   their global indices, so the perturbation ranks stay global;
4. every rank triangulates its partitions and detects their border simplices;
   the grid occupancy the border test needs is the bitwise OR of every rank's
   own partitions' cells (`allreduce_occupancy`);
5. vertices(B) are gathered into the root rank's own memory
   (`gather_to_root`: every copy lands in the receiver's buffers, no remote
   reads), the root triangulates them, and the hash merge runs on global ids:
   every rank keeps its T_i minus B, the root adds the kept border simplices.

The functions here move only host tensors through the process group (gloo
on CPU, NCCL on GPUs); the triangulation steps are the library's calls on
each rank's own GPU.  Covered on CPU by world_size-2 gloo tests.
"""
from __future__ import annotations

import numpy as np


def assign_partitions(sizes, world: int) -> np.ndarray:
    """Owner rank of every partition: partitions in decreasing size (ties:
    smaller id) go one by one to the rank with the fewest points so far
    (ties: smaller rank).  Deterministic, so every rank computes the same
    plan from the all-reduced partition sizes."""
    sizes = np.asarray(sizes, dtype=np.int64)
    k = len(sizes)
    owner = np.zeros(k, dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    for i in sorted(range(k), key=lambda j: (-int(sizes[j]), j)):
        r = int(np.argmin(load))           # first minimum: the smaller rank on ties
        owner[i] = r
        load[r] += sizes[i]
    return owner


def route(labels, owner, world: int):
    """Order of this rank's points for the all-to-all (stable by destination
    rank) and the number of points for each destination."""
    dest = np.asarray(owner)[np.asarray(labels, dtype=np.int64)]
    order = np.argsort(dest, kind="stable")
    counts = np.bincount(dest, minlength=world).astype(np.int64)
    return order, counts


def exchange_points(dist, coords, gids, labels, owner):
    """All-to-all of this rank's points to their partitions' owners.
    Returns (coords, global ids, labels) of the points this rank owns, in
    the order of the sending ranks (each sender's points in its own order)."""
    import torch
    world = dist.get_world_size()
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    order, send = route(labels, owner, world)
    recv = torch.empty(world, dtype=torch.int64)
    dist.all_to_all_single(recv, torch.from_numpy(send))
    recv = recv.numpy()
    dim = coords.shape[1]
    cin = torch.from_numpy(np.ascontiguousarray(coords[order]).reshape(-1))
    cout = torch.empty(int(recv.sum()) * dim, dtype=torch.float64)
    dist.all_to_all_single(cout, cin, [int(x) * dim for x in recv], [int(x) * dim for x in send])
    meta_in = torch.from_numpy(np.stack([np.asarray(gids, dtype=np.int64)[order],
                                         np.asarray(labels, dtype=np.int64)[order]], axis=1).reshape(-1))
    meta_out = torch.empty(int(recv.sum()) * 2, dtype=torch.int64)
    dist.all_to_all_single(meta_out, meta_in, [int(x) * 2 for x in recv], [int(x) * 2 for x in send])
    meta = meta_out.numpy().reshape(-1, 2)
    return cout.numpy().reshape(-1, dim), meta[:, 0], meta[:, 1]


def partition_sizes(dist, labels, k: int) -> np.ndarray:
    """Points per partition over all ranks (all-reduced)."""
    import torch
    t = torch.from_numpy(np.bincount(np.asarray(labels, dtype=np.int64), minlength=k).astype(np.int64))
    dist.all_reduce(t)
    return t.numpy()


def allreduce_occupancy(dist, cells) -> np.ndarray:
    """Bitwise OR over ranks of the per-cell partition masks (int64, bit i =
    partition i occupies the cell), the grid the border test reads."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(cells, dtype=np.int64).copy())
    dist.all_reduce(t, op=dist.ReduceOp.BOR)
    return t.numpy()


def gather_to_root(dist, rows, root: int = 0):
    """Variable-length rows (int64 or float64, any row width) from every rank
    into the root's own memory: sizes first, then one gather of rows padded to
    the largest count.  Returns the concatenation in rank order on the root,
    None elsewhere."""
    import torch
    world = dist.get_world_size()
    rows = np.ascontiguousarray(rows)
    width = rows.shape[1] if rows.ndim == 2 else 1
    n = torch.tensor([len(rows)], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    m = max(counts) if counts else 0
    pad = np.zeros((m, width), dtype=rows.dtype)
    pad[:len(rows)] = rows.reshape(len(rows), width)
    t = torch.from_numpy(pad)
    bufs = [torch.empty_like(t) for _ in range(world)] if dist.get_rank() == root else None
    dist.gather(t, gather_list=bufs, dst=root)
    if dist.get_rank() != root:
        return None
    out = np.concatenate([b.numpy()[:c] for b, c in zip(bufs, counts)])
    return out if rows.ndim == 2 else out.reshape(-1)
