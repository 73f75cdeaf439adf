"""Writes the stored oracle energies used by the GPU parity tests.

Calls only oracle/ (and the seeded inputs of synthetic/).  Run from the repo
root:  python tests/golden/make_golden.py [tiny|medium_partitions|medium64 [fock|dyall [sweeps]]]
(medium: the first sweeps of the M = 64 run; the tests compare E2 per sweep).
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


def medium_partitions(M, h0, pairs):
    """Per-partition E2 of a few virtual-pair partitions of the medium system."""
    from oracle.partition import SubProblem
    h, L, c = synthetic.config_integrals("medium")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    out = {"config": "medium", "h0": h0, "M": M, "parts": []}
    for a, b in pairs:
        t = time.time()
        sub = SubProblem(p, a, b)
        e2 = HylleraasSweep(sub, M, allowed=sub.allowed).run()
        out["parts"].append({"a": a, "b": b, "E2": e2, "oracle_s": time.time() - t})
        print(a, b, e2, flush=True)
    return out


def medium(M, h0, sweeps):
    h, L, c = synthetic.config_integrals("medium")
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    t = time.time()
    sw = HylleraasSweep(p, M, tol_e=1e-9, max_sweeps=sweeps, verbose=True)
    e2 = sw.run()
    e3 = third_order(sw)
    print("E3", e3, flush=True)
    return {"config": "medium", "h0": h0, "M": M, "E_ref": p.E_ref, "E0": p.E0, "E1": p.E1,
            "E2": e2, "E3": e3, "sweeps": len(sw.history), "history": sw.history, "tol_e": 1e-9,
            "oracle_s": time.time() - t}


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "tiny"
    if what == "tiny":
        res = tiny()
        name = "oracle_tiny.json"
    elif what == "medium_partitions":
        res = medium_partitions(16, "fock", [(0, 0), (3, 17), (23, 23)])
        name = "oracle_medium_partitions_fock_M16.json"
    else:
        M = int(what.replace("medium", ""))
        h0 = sys.argv[2] if len(sys.argv) > 2 else "fock"
        res = medium(M, h0, int(sys.argv[3]) if len(sys.argv) > 3 else 3)
        name = f"oracle_medium_{h0}_M{M}.json"
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(res, f, indent=1)
    print("wrote", name)
