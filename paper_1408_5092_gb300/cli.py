"""Run one MPS-PT minimisation on a seeded synthetic system from the shell.

    python -m paper_1408_5092_gb300.cli --config medium --M 256 --h0 dyall \
        --prec mixed [--sweeps 64] [--e_tol 1e-7] [--e3] [--verbose 1]
    python -m paper_1408_5092_gb300.cli --config medium --partitions 300 \
        [--streams 8] [--M 0]      (partitioned mode, uneven seeded M_P)

Prints one JSON line: E2 (and E3), the per-sweep energies and device times,
the local-solver counters and the kernel launch count; in partitioned mode
the total E2, the partitions per second and the wall time.  The system comes
from the seeded generator in synthetic/ (run from the repository root).
"""
import argparse
import json
import sys
import time

from . import _lib as L


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--config", default="medium", choices=["tiny", "medium", "partitions", "large"])
    ap.add_argument("--seed", type=int, default=None, help="integral seed (default: the evaluation seed)")
    ap.add_argument("--M", type=int, default=64)
    ap.add_argument("--h0", default="dyall", choices=["dyall", "fock"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--sweeps", type=int, default=64)
    ap.add_argument("--e_tol", type=float, default=1e-7)
    ap.add_argument("--eig_fp64_only", type=int, default=0)
    ap.add_argument("--e3", action="store_true")
    ap.add_argument("--verbose", type=int, default=0)
    ap.add_argument("--partitions", type=int, default=0,
                    help="partitioned mode: the first N virtual pairs (a <= b, a then b)")
    ap.add_argument("--streams", type=int, default=8)
    a = ap.parse_args(argv)
    import synthetic
    seed = synthetic.EVAL_SEED if a.seed is None else a.seed
    h, Lc, c = synthetic.config_integrals(a.config, seed=seed)
    ci, _ = synthetic.fci_reference(h, Lc, c["k_act"], c["n_elec"])
    o = L.mpspt_default_options()
    o.prec = L.PREC[a.prec]
    o.max_sweeps = a.sweeps
    o.e_tol = a.e_tol
    o.verbose = a.verbose
    o.eig_fp64_only = a.eig_fp64_only
    ctx = L.mpspt_create(o)
    try:
        L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
        L.mpspt_set_reference_ci(ctx, ci)
        if a.partitions > 0:
            kv = h.shape[0] - c["k_act"]
            pairs = [(x, y) for x in range(kv) for y in range(x, kv)][: a.partitions]
            Ms = synthetic.partition_bond_dims(len(pairs)) if a.M <= 0 else [a.M] * len(pairs)
            t = time.time()
            tot, ep, rep = L.mpspt_minimize_partitioned(ctx, a.h0, pairs, Ms, n_streams=a.streams)
            wall = time.time() - t
            print(json.dumps({"config": a.config, "h0": a.h0, "prec": a.prec, "partitions": len(pairs),
                              "M_part": "seeded from {32,...,512}" if a.M <= 0 else a.M, "E2": tot,
                              "wall_s": wall, "partitions_per_s": len(pairs) / wall, "streams": a.streams,
                              "cg_iters": rep.cg_iters, "kernel_launches": rep.kernel_launches}), flush=True)
            return 0
        t = time.time()
        e2, psi, rep = L.mpspt_minimize_hylleraas(ctx, a.h0, a.M, want_psi1=a.e3)
        wall = time.time() - t
        out = {"config": a.config, "M": a.M, "h0": a.h0, "prec": a.prec, "E2": e2, "wall_s": wall,
               "sweeps": rep.n_sweeps, "e2_per_sweep": [rep.e2_per_sweep[s] for s in range(rep.n_sweeps)],
               "sweep_ms": [rep.sweep_ms[s] for s in range(rep.n_sweeps)], "cg_iters": rep.cg_iters,
               "sigma_ms": rep.sigma_ms, "sigma_gflop": rep.sigma_flops / 1e9, "sigma64_ms": rep.sigma64_ms,
               "max_bond_dim": rep.max_bond_dim, "max_discarded_weight": rep.max_discarded_weight,
               "kernel_launches": rep.kernel_launches}
        if a.e3:
            out["E3"] = L.mpspt_third_order(ctx, a.h0, psi)
            L.mpspt_mps_free(psi)
        print(json.dumps(out), flush=True)
    finally:
        L.mpspt_destroy(ctx)
    return 0


if __name__ == "__main__":
    sys.exit(main())
