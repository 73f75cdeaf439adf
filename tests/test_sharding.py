"""Host logic of the partitioned mode across ranks: the longest-first
assignment, and a world-size-2 gloo run on CPU whose per-rank solver is the
oracle's uncontracted partition energy.  The sharded sum must equal the
serial sum bit for bit and, since E2* = sum_P E2*_P, the brute-force E2*."""
import os
import socket

import numpy as np
import pytest

import synthetic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_assign_covers_each_partition_once_and_balances():
    from paper_1408_5092_gb300.sharding import assign, partition_cost
    rng = np.random.default_rng(7)
    Ms = rng.choice([32, 64, 128, 256, 512], size=1830)
    for world in (1, 2, 3, 8):
        parts = assign(Ms, world)
        allidx = np.concatenate(parts)
        assert sorted(allidx.tolist()) == list(range(len(Ms)))
        cost = partition_cost(Ms)
        loads = [cost[p].sum() for p in parts]
        # LPT: the heaviest rank exceeds the lightest by at most one partition
        assert max(loads) - min(loads) <= cost.max() + 1e-9
    assert assign([], 2)[0].size == 0
    with pytest.raises(ValueError):
        assign(Ms, 0)


def _problem():
    from oracle.operators import Problem
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    return Problem(h, L, c["k_act"], c["n_elec"], ci, h0="fock")


def _exact_solver(prob):
    from oracle.partition import ExactPartition, SubProblem

    def solve(pairs, Ms):
        return [ExactPartition(SubProblem(prob, int(a), int(b))).e2() for a, b in pairs]
    return solve


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    from oracle.partition import partitions
    from paper_1408_5092_gb300.sharding import minimize_partitioned_sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        prob = _problem()
        pairs = partitions(prob.k_virt)
        Ms = [4 + (3 * a + 5 * b) % 9 for a, b in pairs]
        tot, ep = minimize_partitioned_sharded(None, "fock", pairs, Ms, solve=_exact_solver(prob))
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([[tot], ep]))
    finally:
        dist.destroy_process_group()


def test_sharded_sum_equals_serial_and_brute_force(tmp_path):
    import torch.multiprocessing as mp
    from oracle.brute import ExactFirstOrder
    from oracle.partition import partitions
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    assert np.array_equal(res[0], res[1])           # every rank holds the same result
    prob = _problem()
    solve = _exact_solver(prob)
    serial = solve(partitions(prob.k_virt), None)
    assert np.array_equal(res[0][1:], np.array(serial))
    total = 0.0
    for v in serial:
        total += v
    assert res[0][0] == total
    assert abs(total - ExactFirstOrder(prob).e2()) < 1e-10
