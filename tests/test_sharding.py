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


def _serial(prob):
    from oracle.partition import partitions
    pairs = partitions(prob.k_virt)
    return pairs, np.array(_exact_solver(prob)(pairs, None))


def test_checkpoint_resume_skips_recorded_partitions(tmp_path):
    from paper_1408_5092_gb300.sharding import load_checkpoint, minimize_partitioned_sharded
    prob = _problem()
    pairs, serial = _serial(prob)
    Ms = [4 + (3 * a + 5 * b) % 9 for a, b in pairs]
    ck = str(tmp_path / "run")
    exact = _exact_solver(prob)
    calls = []

    def crashing(p, m):
        if len(calls) == 3:
            raise RuntimeError("node lost")
        calls.append(len(p))
        return exact(p, m)

    with pytest.raises(RuntimeError):
        minimize_partitioned_sharded(None, "fock", pairs, Ms, solve=crashing, checkpoint=ck, chunk=2)
    done = load_checkpoint(ck, "fock", pairs, Ms)
    assert len(done) == 6 and all(done[i] == serial[i] for i in done)
    # a write cut short leaves a partial last line, which is ignored
    with open(ck + ".rank0.jsonl", "a") as f:
        f.write('{"p": 7, "a": ')
    solved = []

    def counting(p, m):
        solved.extend(map(tuple, np.asarray(p).tolist()))
        return exact(p, m)

    tot, ep = minimize_partitioned_sharded(None, "fock", pairs, Ms, solve=counting, checkpoint=ck, chunk=5)
    assert len(solved) == len(pairs) - 6
    assert np.array_equal(ep, serial)
    total = 0.0
    for v in serial:
        total += v
    assert tot == total
    # records of another partition list are refused
    with pytest.raises(ValueError):
        load_checkpoint(ck, "fock", pairs, [m + 1 for m in Ms])
    with pytest.raises(ValueError):
        load_checkpoint(ck, "dyall", pairs, Ms)


def _resume_worker(rank, world, port, out_dir, ck):
    import torch.distributed as dist
    from paper_1408_5092_gb300.sharding import minimize_partitioned_sharded
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        prob = _problem()
        from oracle.partition import partitions
        pairs = partitions(prob.k_virt)
        Ms = [4 + (3 * a + 5 * b) % 9 for a, b in pairs]
        seen = []
        exact = _exact_solver(prob)

        def solve(p, m):
            seen.extend(map(tuple, np.asarray(p).tolist()))
            return exact(p, m)
        tot, ep = minimize_partitioned_sharded(None, "fock", pairs, Ms, solve=solve, checkpoint=ck, chunk=3)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([[tot, len(seen)], ep]))
    finally:
        dist.destroy_process_group()


def test_sharded_resume_over_two_ranks(tmp_path):
    """A previous run (other world size) recorded every third partition; two
    gloo ranks solve only the rest and agree bit for bit with the serial
    energies."""
    import torch.multiprocessing as mp
    from paper_1408_5092_gb300.sharding import load_checkpoint
    from paper_1408_5092_gb300.sharding import _append_checkpoint
    prob = _problem()
    pairs, serial = _serial(prob)
    Ms = [4 + (3 * a + 5 * b) % 9 for a, b in pairs]
    ck = str(tmp_path / "run")
    prev = list(range(0, len(pairs), 3))
    _append_checkpoint(ck + ".rank5.jsonl", "fock", np.asarray(pairs), Ms, prev, serial[prev])
    mp.spawn(_resume_worker, args=(2, _free_port(), str(tmp_path), ck), nprocs=2, join=True)
    res = [np.load(tmp_path / f"rank{r}.npy") for r in range(2)]
    assert np.array_equal(res[0][2:], res[1][2:]) and res[0][0] == res[1][0]
    assert np.array_equal(res[0][2:], serial)
    assert res[0][1] + res[1][1] == len(pairs) - len(prev)
    assert len(load_checkpoint(ck, "fock", pairs, Ms)) == len(pairs)


def _elastic_worker(rank, port, out_dir, die_on_call):
    import datetime
    import time as _t
    import torch.distributed as dist
    from oracle.partition import partitions
    from paper_1408_5092_gb300.sharding import minimize_partitioned_elastic
    store = dist.TCPStore("127.0.0.1", port, is_master=False, timeout=datetime.timedelta(seconds=60))
    prob = _problem()
    pairs = partitions(prob.k_virt)
    Ms = [4 + (3 * a + 5 * b) % 9 for a, b in pairs]
    exact = _exact_solver(prob)
    calls = [0]

    def solve(p, m):
        calls[0] += 1
        if calls[0] == die_on_call:
            os._exit(3)                      # the process disappears with its claims unfinished
        _t.sleep(0.05 * len(p))
        return exact(p, m)
    tot, ep, mine, taken = minimize_partitioned_elastic(None, "fock", pairs, Ms, store, rank, solve=solve,
                                                        batch=2, timeout=3.0, heartbeat=0.2, poll=0.05,
                                                        deadline=120.0)
    np.save(os.path.join(out_dir, f"elastic{rank}.npy"), np.concatenate([[tot], ep]))
    np.save(os.path.join(out_dir, f"mine{rank}.npy"), np.asarray(mine))
    np.save(os.path.join(out_dir, f"taken{rank}.npy"), np.asarray(taken, dtype=np.int64))


def test_elastic_run_survives_a_dead_rank(tmp_path):
    """Three ranks claim partitions through a store served by this process;
    rank 1 exits after claiming its second batch.  The other two take over
    its unfinished claims once its heartbeat stops and return the serial
    energies bit for bit."""
    import datetime
    import multiprocessing
    import torch.distributed as dist
    prob = _problem()
    pairs, serial = _serial(prob)
    port = _free_port()
    store = dist.TCPStore("127.0.0.1", port, is_master=True, wait_for_workers=False,
                          timeout=datetime.timedelta(seconds=60))
    ctx = multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_elastic_worker, args=(r, port, str(tmp_path), 2 if r == 1 else 0))
             for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    codes = [p.exitcode for p in procs]
    assert codes == [0, 3, 0], codes
    res = [np.load(tmp_path / f"elastic{r}.npy") for r in (0, 2)]
    assert np.array_equal(res[0], res[1])
    assert np.array_equal(res[0][1:], serial)
    total = 0.0
    for v in serial:
        total += v
    assert res[0][0] == total
    # rank 1 stored at most its first batch; the survivors solved the rest,
    # including its orphaned second batch
    mine = [set(np.load(tmp_path / f"mine{r}.npy").tolist()) for r in (0, 2)]
    taken = [set(np.load(tmp_path / f"taken{r}.npy").tolist()) for r in (0, 2)]
    assert len(mine[0] | mine[1]) >= len(pairs) - 2
    assert taken[0] | taken[1], "nobody took over the dead rank's claims"
    # a partition is solved twice only through a takeover: the overlap of the
    # survivors' work is made of taken-over claims (a live rank starved of CPU
    # past the timeout can have a claim taken over; the energy is the same),
    # and no more than the dead rank's batch plus one batch per survivor is
    # solved twice
    dup = mine[0] & mine[1]
    assert dup <= (taken[0] | taken[1]), (dup, taken)
    assert len(dup) <= 2 + 2 * 2, dup
    del store
