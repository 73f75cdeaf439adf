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

Two host-side services sit around the partition solves:

* checkpoint / resume: finished partition energies are appended to one
  JSON-lines file per rank; a later run reads every rank's file, skips the
  recorded partitions and solves only the rest;
* elastic recovery (``minimize_partitioned_elastic``): ranks claim
  partitions through a key-value store instead of a fixed assignment, keep
  a heartbeat counter there, and take over the unfinished claims of a rank
  whose heartbeat stops.  No collective is used, so a rank that dies does
  not block the others.
"""
import glob
import json
import os
import threading
import time

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


def _solver(ctx, h0, n_streams, solve):
    if solve is not None:
        return lambda p, m: np.asarray(solve(p, m), dtype=np.float64)

    def run(p, m):
        _, ep, _ = _lib.mpspt_minimize_partitioned(ctx, h0, p, m, n_streams)
        return np.asarray(ep, dtype=np.float64)
    return run


def _checkpoint_files(checkpoint):
    return sorted(glob.glob(glob.escape(checkpoint) + ".rank*.jsonl"))


def load_checkpoint(checkpoint, h0, pairs, Ms):
    """Partition energies recorded under ``checkpoint`` (every rank's file):
    {partition index: E2_P}.  A record whose pair, bond dimension or H0
    differs from this request raises ValueError; an incomplete last line (a
    write cut short) is ignored."""
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    Ms = np.asarray(Ms, dtype=np.int64).reshape(-1)
    done = {}
    for path in _checkpoint_files(checkpoint):
        with open(path) as f:
            lines = f.read().split("\n")
        for n, line in enumerate(lines):
            if not line.strip():
                continue
            try:
                r = json.loads(line)
            except json.JSONDecodeError:
                if n == len(lines) - 1 or not any(x.strip() for x in lines[n + 1:]):
                    continue          # the last record of a rank that stopped mid-write
                raise ValueError(f"{path}: corrupt record on line {n + 1}")
            i = int(r["p"])
            if not (0 <= i < len(Ms)) or [r["a"], r["b"]] != pairs[i].tolist() or r["M"] != int(Ms[i]) \
                    or r["h0"] != h0:
                raise ValueError(f"{path}: record {r} does not belong to this partition list")
            done[i] = float(r["e2"])
    return done


def _append_checkpoint(path, h0, pairs, Ms, idx, energies):
    with open(path, "a") as f:
        for i, e in zip(idx, energies):
            f.write(json.dumps({"p": int(i), "a": int(pairs[i][0]), "b": int(pairs[i][1]), "M": int(Ms[i]),
                                "h0": h0, "e2": float(e)}) + "\n")
        f.flush()
        os.fsync(f.fileno())


def minimize_partitioned_sharded(ctx, h0, pairs, Ms, n_streams=0, group=None, solve=None,
                                 checkpoint=None, chunk=0):
    """E2 over all partitions with the partitions spread over the ranks of
    ``group`` (default: the default process group; a single process when
    torch.distributed is not initialised).

    ctx: this rank's mpspt context (integrals and reference loaded).
    solve: optional callable (pairs_subset, Ms_subset) -> energies, used in
    place of the library call (host-side tests of the sharding logic).
    checkpoint: optional path prefix.  Partitions already recorded under it
    are not solved again; each rank appends what it finishes to
    ``<checkpoint>.rank<r>.jsonl`` after every ``chunk`` partitions (0: once,
    after all of its partitions).
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
    done = load_checkpoint(checkpoint, h0, pairs, Ms) if checkpoint else {}
    if checkpoint and world > 1:
        dist.barrier(group=group)     # every rank has read the records before any rank appends
    todo = np.array([i for i in range(len(Ms)) if i not in done], dtype=np.int64)
    mine = todo[assign(Ms[todo], world)[rank]] if len(todo) else todo
    dev = "cpu"
    if dist_on and dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    e = torch.zeros(len(Ms), dtype=torch.float64, device=dev)
    run = _solver(ctx, h0, n_streams, solve)
    step = len(mine) if chunk <= 0 else chunk
    for c0 in range(0, len(mine), max(step, 1)):
        part = mine[c0:c0 + step]
        ep = run(pairs[part], Ms[part])
        e[torch.as_tensor(part, device=dev)] = torch.as_tensor(ep, dtype=torch.float64, device=dev)
        if checkpoint:
            _append_checkpoint(f"{checkpoint}.rank{rank}.jsonl", h0, pairs, Ms, part, ep)
    if world > 1:
        # each entry is non-zero on exactly one rank, so the sum is exact
        dist.all_reduce(e, group=group)
    ep = e.cpu().numpy()
    for i, v in done.items():
        ep[i] = v
    total = 0.0
    for v in ep:
        total += float(v)
    return total, ep


class _Heartbeat:
    """Increments ``<prefix>/hb/<rank>`` in the store every ``interval``
    seconds from a daemon thread until stopped (or the process ends)."""

    def __init__(self, store, lock, key, interval):
        self.store, self.lock, self.key, self.interval = store, lock, key, interval
        self.stop_ev = threading.Event()
        with self.lock:
            self.store.add(self.key, 1)
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        while not self.stop_ev.wait(self.interval):
            try:
                with self.lock:
                    self.store.add(self.key, 1)
            except Exception:
                return

    def stop(self):
        self.stop_ev.set()
        self.th.join()


def minimize_partitioned_elastic(ctx, h0, pairs, Ms, store, rank, n_streams=0, solve=None, batch=1,
                                 timeout=60.0, heartbeat=1.0, poll=0.2, deadline=None, prefix="mpspt"):
    """E2 over all partitions, solved by whichever ranks are alive.

    store: a torch.distributed Store shared by the ranks that must outlive
    them (for example the launcher's rendezvous store, or a TCPStore served
    by a process that does not solve).  rank: this process's id.
    Each rank walks the partitions longest first and claims unclaimed ones
    atomically (compare-and-set of ``<prefix>/claim/<i>``), ``batch`` at a
    time, solves them and stores the energies.  When nothing is left to
    claim it waits for the missing energies; a claim whose owner's
    heartbeat has not advanced for ``timeout`` seconds (this rank's clock)
    is taken over and solved again.  Partition energies do not depend on
    who solves them, and the total is summed in partition order, so every
    surviving rank returns the same values.
    deadline: optional limit in seconds on the whole call (TimeoutError).
    Returns (E2_total, per-partition E2, indices this rank solved, indices
    it took over from a rank whose heartbeat had stopped)."""
    pairs = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    Ms = np.asarray(Ms, dtype=np.int32).reshape(-1)
    if len(pairs) != len(Ms):
        raise ValueError("pairs and Ms differ in length")
    n = len(Ms)
    me = str(int(rank))
    t_start = time.monotonic()
    lock = threading.Lock()
    run = _solver(ctx, h0, n_streams, solve)
    cost = partition_cost(Ms)
    order = sorted(range(n), key=lambda i: (-cost[i], i))
    ekey = lambda i: f"{prefix}/e/{i}"          # noqa: E731
    ckey = lambda i: f"{prefix}/claim/{i}"      # noqa: E731
    solved = []
    taken = []

    def have(i):
        with lock:
            return store.check([ekey(i)])

    def solve_and_store(idx):
        idx = np.asarray(idx, dtype=np.int64)
        ep = run(pairs[idx], Ms[idx])
        with lock:
            for i, v in zip(idx, ep):
                store.set(ekey(int(i)), repr(float(v)))
        solved.extend(int(i) for i in idx)

    def check_deadline():
        if deadline is not None and time.monotonic() - t_start > deadline:
            raise TimeoutError(f"rank {me}: partitions still missing after {deadline} s")

    hb = _Heartbeat(store, lock, f"{prefix}/hb/{me}", heartbeat)
    try:
        # claim phase: every index ends up claimed by some rank
        mine = []
        for i in order:
            if have(i):
                continue
            with lock:
                owner = store.compare_set(ckey(i), "", me).decode()
            if owner == me:
                mine.append(i)
                if len(mine) == batch:
                    solve_and_store(mine)
                    mine = []
        if mine:
            solve_and_store(mine)
        # recovery phase: wait for the others, take over the claims of dead ranks
        seen = {}                                  # owner -> (last heartbeat value, when it last changed)
        while True:
            missing = [i for i in order if not have(i)]
            if not missing:
                break
            check_deadline()
            now = time.monotonic()
            take = []
            for i in missing:
                with lock:
                    owner = store.get(ckey(i)).decode()
                    beat = int(store.add(f"{prefix}/hb/{owner}", 0))
                last = seen.get(owner)
                if last is None or last[0] != beat:
                    seen[owner] = (beat, now)
                elif owner != me and now - last[1] > timeout:
                    with lock:
                        if store.compare_set(ckey(i), owner, me).decode() == me:
                            take.append(i)
            taken.extend(take)
            for c0 in range(0, len(take), batch):
                solve_and_store(take[c0:c0 + batch])
            if not take:
                time.sleep(poll)
    finally:
        hb.stop()
    ep = np.empty(n)
    with lock:
        for i in range(n):
            ep[i] = float(store.get(ekey(i)).decode())
    total = 0.0
    for v in ep:
        total += float(v)
    return total, ep, sorted(solved), sorted(taken)
