"""Writes the stored oracle energies used by the GPU parity tests.

Calls only oracle/ (and the seeded inputs of synthetic/).  Run from the repo
root:
    python tests/golden/make_golden.py [tiny|medium_partitions|medium<M> [fock|dyall [sweeps]]] [--threads T]
(medium<M>: the sweep history at bond dimension M; the tests compare E2 per
sweep).  The medium reference vector is the stored one
(synthetic.config_reference), so the GPU machine starts from the same bits.  The
BLAS thread count is fixed (default 2) and recorded: it changes the summation
order of the oracle's matrix products.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synthetic  # noqa: E402
from oracle.brute import ExactFirstOrder  # noqa: E402
from oracle.mps import HylleraasSweep, third_order  # noqa: E402
from oracle.operators import Problem  # noqa: E402


def tiny():
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    out = {"config": "tiny", "seed": synthetic.integrals.EVAL_SEED if hasattr(synthetic.integrals, "EVAL_SEED") else 1408, "h0": {}}
    for h0 in ("fock", "dyall"):
        p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
        ex = ExactFirstOrder(p)
        ranks = ex.schmidt_ranks()
        d = {"E_ref": p.E_ref, "E0": p.E0, "E1": p.E1, "E2_exact": ex.e2(), "E3_exact": ex.e3(),
             "M_exact": max(ranks), "runs": {}}
        for M in (16, 32, max(ranks)):
            t = time.time()
            sw = HylleraasSweep(p, M)
            e2 = sw.run()
            d["runs"][str(M)] = {"E2": e2, "E3": third_order(sw), "sweeps": len(sw.history),
                                 "history": sw.history, "oracle_s": time.time() - t}
            print(h0, M, e2, flush=True)
        out["h0"][h0] = d
    return out


def tiny_extrapolation(Ms=(20, 26, 32, 36)):
    """E2(M), discarded weights and the extrapolated E2 (oracle/extrapolate.py)
    on the tiny system, both H0."""
    from oracle.extrapolate import extrapolate_e2
    h, L, c = synthetic.config_integrals("tiny")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    out = {"config": "tiny", "Ms": list(Ms), "h0": {}}
    for h0 in ("fock", "dyall"):
        p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
        a, b, e2, w = extrapolate_e2(p, Ms)
        out["h0"][h0] = {"E2_extrap": a, "slope": b, "E2": e2, "w": w}
        print(h0, a, b, flush=True)
    return out


def medium_partitions(M, h0, pairs):
    """Per-partition E2 of a few virtual-pair partitions of the medium system."""
    from oracle.partition import SubProblem
    h, L, c, ci = synthetic.config_reference("medium")
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    out = {"config": "medium", "h0": h0, "M": M, "parts": []}
    for a, b in pairs:
        t = time.time()
        sub = SubProblem(p, a, b)
        e2 = HylleraasSweep(sub, M, allowed=sub.allowed).run()
        out["parts"].append({"a": a, "b": b, "E2": e2, "oracle_s": time.time() - t})
        print(a, b, e2, flush=True)
    return out


def medium_partition_e3(M, h0, pairs):
    """E3 of the sum of a few medium partitions' MPS-PT2 solutions (Eq. 5 over
    partitions, transfer route of oracle/partition.py), with every partition's
    E2, E3 and the pair elements <Psi1^i|H|Psi1^j>."""
    from oracle.mpo import build_mpo
    from oracle.partition import partition_e3_mps, partition_psi1
    h, L, c, ci = synthetic.config_reference("medium")
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    t = time.time()
    sp = partition_psi1(p, pairs, lambda a, b: M)
    t_sweeps = time.time() - t
    WH = build_mpo(p.hamiltonian_terms(), p.k, k_split=p.k_act)
    t = time.time()
    e3, diag, cross, hh = partition_e3_mps(p, [(s, m) for s, _, m in sp], WH=WH)
    out = {"config": "medium", "h0": h0, "M": M, "pairs": [list(x) for x in pairs],
           "E2_part": [e for _, e, _ in sp], "E3": e3, "E3_part": diag, "E3_cross": cross,
           "H_pair": [[i, j, v] for (i, j), v in sorted(hh.items())],
           "oracle_sweeps_s": t_sweeps, "oracle_e3_s": time.time() - t, "blas_threads": THREADS}
    print(out, flush=True)
    return out


def medium(M, h0, sweeps, out_name):
    """Sweep history at bond dimension M; the file is rewritten after every
    sweep (with E3 of the state at that point), so a long run leaves usable
    values while it goes on."""
    h, L, c, ci = synthetic.config_reference("medium")
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    t = time.time()
    sw = HylleraasSweep(p, M, tol_e=1e-10, max_sweeps=sweeps, verbose=True)
    res = {"config": "medium", "h0": h0, "M": M, "E_ref": p.E_ref, "E0": p.E0, "E1": p.E1,
           "tol_e": 1e-10, "blas_threads": THREADS, "history": [], "E3_history": [],
           "max_discarded": [], "cg_iters": [], "sweep_s": []}
    prev = None
    for n in range(sweeps):
        t1 = time.time()
        sw.discarded = []
        e = sw.sweep()
        sw.history.append(e)
        e3 = third_order(sw)
        res["history"].append(e)
        res["E3_history"].append(e3)
        res["max_discarded"].append(max(sw.discarded))
        res["cg_iters"].append(sw.cg_iters)
        res["sweep_s"].append(time.time() - t1)
        res.update({"E2": e, "E3": e3, "sweeps": len(sw.history), "oracle_s": time.time() - t,
                    "converged": prev is not None and abs(e - prev) < 1e-10})
        print(f"sweep {n}: E2 = {e:.12f} E3 = {e3:.12f} max discarded {max(sw.discarded):.3e} "
              f"({time.time() - t1:.0f} s)", flush=True)
        with open(os.path.join(HERE, out_name), "w") as f:
            json.dump(res, f, indent=1)
        if res["converged"]:
            break
        prev = e
    return res


THREADS = 2

if __name__ == "__main__":
    if "--threads" in sys.argv:
        k = sys.argv.index("--threads")
        THREADS = int(sys.argv[k + 1])
        del sys.argv[k:k + 2]
    from threadpoolctl import threadpool_limits
    threadpool_limits(THREADS)
    what = sys.argv[1] if len(sys.argv) > 1 else "tiny"
    if what == "tiny":
        res = tiny()
        name = "oracle_tiny.json"
    elif what == "tiny_extrapolation":
        res = tiny_extrapolation()
        name = "oracle_tiny_extrapolation.json"
    elif what == "medium_partitions":
        res = medium_partitions(16, "fock", [(0, 0), (3, 17), (23, 23)])
        name = "oracle_medium_partitions_fock_M16.json"
    elif what == "medium_partition_e3":
        res = medium_partition_e3(16, "fock", [(0, 0), (0, 1), (1, 5), (5, 5), (23, 23)])
        name = "oracle_medium_partition_e3_fock_M16.json"
    else:
        M = int(what.replace("medium", ""))
        h0 = sys.argv[2] if len(sys.argv) > 2 else "fock"
        name = f"oracle_medium_{h0}_M{M}.json"
        res = medium(M, h0, int(sys.argv[3]) if len(sys.argv) > 3 else 3, name)
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", name)
