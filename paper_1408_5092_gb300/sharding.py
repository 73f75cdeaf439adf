"""Partitioned MPS-PT across ranks, one process per GPU.

The virtual-pair partitions P = (a, b), a <= b, are independent first-order
problems (H0 conserves every virtual occupation, so E2 = sum_P E2_P exactly;
the paper notes this parallelism over pairs of virtual orbitals).  Each rank
solves its share of the partitions with ``mpspt_minimize_partitioned`` on its
own GPU; one float64 all-reduce then gathers the partition energies, which
every rank sums in partition order (a, then b).  No collective runs inside a
partition's sweep.

Assignment is longest-processing-time first on the estimated cost M_P^3 (the
sigma contractions scale with the cube of the bond dimension), so that the
slowest rank's load stays within one partition of the mean.
"""
import numpy as np

from . import _lib


def partition_cost(Ms):
    """Estimated relative cost of each partition (bond dimension cubed)."""
    return np.asarray(Ms, dtype=np.float64) ** 3


def assign(Ms, world):
    """Partition indices per rank: longest first, each to the least-loaded
    rank (ties to the lower rank, equal costs in index order).  Every index
    appears exactly once; each rank's list is sorted."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    cost = partition_cost(Ms)
    order = sorted(range(len(cost)), key=lambda i: (-cost[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += cost[i]
    return [np.array(sorted(x), dtype=np.int64) for x in out]


def minimize_partitioned_sharded(ctx, h0, pairs, Ms, n_streams=0, group=None, solve=None):
    """E2 over all partitions with the partitions spread over the ranks of
    ``group`` (default: the default process group; a single process when
    torch.distributed is not initialised).

    ctx: this rank's mpspt context (integrals and reference loaded).
    solve: optional callable (pairs_subset, Ms_subset) -> energies, used in
    place of the library call (host-side tests of the sharding logic).
    Returns (E2_total, per-partition E2 in partition order); every rank
    returns the same values."""
    import torch
    import torch.distributed as dist

    pairs = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    Ms = np.asarray(Ms, dtype=np.int32).reshape(-1)
    if len(pairs) != len(Ms):
        raise ValueError("pairs and Ms differ in length")
    dist_on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if dist_on else 1
    rank = dist.get_rank(group) if dist_on else 0
    mine = assign(Ms, world)[rank]
    dev = "cpu"
    if dist_on and dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.zeros(len(Ms), dtype=torch.float64, device=dev)
    if len(mine):
        if solve is None:
            _, ep, _ = _lib.mpspt_minimize_partitioned(ctx, h0, pairs[mine], Ms[mine], n_streams)
        else:
            ep = np.asarray(solve(pairs[mine], Ms[mine]), dtype=np.float64)
        e[torch.as_tensor(mine, device=dev)] = torch.as_tensor(ep, dtype=torch.float64, device=dev)
    if world > 1:
        # each entry is non-zero on exactly one rank, so the sum is exact
        dist.all_reduce(e, group=group)
    ep = e.cpu().numpy()
    total = 0.0
    for v in ep:
        total += float(v)
    return total, ep
