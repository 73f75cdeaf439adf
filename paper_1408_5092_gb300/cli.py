"""Run one MPS-PT minimisation on a seeded synthetic system from the shell.

    python -m paper_1408_5092_gb300.cli --config medium --M 256 --h0 dyall \
        --prec mixed [--sweeps 64] [--e_tol 1e-7] [--e3] [--verbose 1]
    python -m paper_1408_5092_gb300.cli --config medium --partitions 300 \
        [--streams 8] [--M 0] [--e3]   (partitioned mode, uneven seeded M_P;
                                        --e3 adds E3 with the cross-partition terms)
    python -m paper_1408_5092_gb300.cli --config partitions --dmrg 256 \
        --partitions 1830 --M 0    (reference by the library's DMRG at M0)

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
    ap.add_argument("--config", default="medium",
                    choices=["tiny", "medium", "partitions", "large"])
    ap.add_argument("--seed", type=int, default=None, help="integral seed (default: the evaluation seed)")
    ap.add_argument("--M", type=int, default=64)
    ap.add_argument("--h0", default="dyall", choices=["dyall", "fock"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "mixed", "mixed_fp16"])
    ap.add_argument("--sweeps", type=int, default=64)
    ap.add_argument("--e_tol", type=float, default=1e-7)
    ap.add_argument("--eig_fp64_only", type=int, default=0)
    ap.add_argument("--e3", action="store_true")
    ap.add_argument("--verbose", type=int, default=0)
    ap.add_argument("--partitions", type=int, default=0,
                    help="partitioned mode: the first N virtual pairs (a <= b, a then b)")
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--chunk", type=int, default=0, help="partitions per call (progress lines between calls)")
    ap.add_argument("--dmrg", type=int, default=0,
                    help="build the reference with the library's ground-state DMRG at this M0 "
                         "(S^2 penalty 1) instead of the FCI vector")
    ap.add_argument("--dmrg_sweeps", type=int, default=0, help="sweep cap of the reference DMRG (0: --sweeps)")
    ap.add_argument("--s2_penalty", type=float, default=1.0,
                    help="lambda of the DMRG's lambda S^2 term (0: lowest Sz = 0 state of any spin)")
    ap.add_argument("--autotune", type=int, default=0)
    ap.add_argument("--graphs", type=int, default=0, help="capture CG chunks in CUDA graphs")
    ap.add_argument("--autotune_cache", default=None)
    a = ap.parse_args(argv)
    import synthetic
    seed = synthetic.EVAL_SEED if a.seed is None else a.seed
    if a.dmrg > 0:
        h, Lc, c = synthetic.config_integrals(a.config, seed=seed)
        ci = None
    else:
        h, Lc, c, ci = synthetic.config_reference(a.config, seed=seed)
    o = L.mpspt_default_options()
    o.autotune = a.autotune
    o.cuda_graphs = a.graphs
    if a.autotune_cache:
        o.autotune_cache = a.autotune_cache.encode()
    o.prec = L.PREC[a.prec]
    o.max_sweeps = a.sweeps
    o.e_tol = a.e_tol
    o.verbose = a.verbose
    o.eig_fp64_only = a.eig_fp64_only
    ctx = L.mpspt_create(o)
    try:
        L.mpspt_set_integrals(ctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
        ref_info = {}
        if ci is None:
            # the reference comes from the library's DMRG in its own context
            # (its own sweep cap) and enters this one as an MPS
            t = time.time()
            od = L.mpspt_default_options()
            od.max_sweeps = a.dmrg_sweeps if a.dmrg_sweeps > 0 else a.sweeps
            od.e_tol = a.e_tol
            od.verbose = a.verbose
            gctx = L.mpspt_create(od)
            L.mpspt_set_integrals(gctx, c["k_act"], h.shape[0] - c["k_act"], c["n_elec"], h, Lc)
            e_ref, psi0, grep = L.mpspt_ground_state(gctx, a.dmrg, s2_penalty=a.s2_penalty, want_psi0=True)
            tensors, labels = L.mpspt_mps_export(psi0)
            L.mpspt_mps_free(psi0)
            L.mpspt_destroy(gctx)
            L.mpspt_set_reference(ctx, tensors, labels)
            e0, e1, eref2 = L.mpspt_energies(ctx, a.h0)
            ref_info = {"reference": f"DMRG M0={a.dmrg}, S^2 penalty {a.s2_penalty}", "E_ref": e_ref, "E_ref_installed": eref2, "E0": e0,
                        "E1": e1, "dmrg_sweeps": grep.n_sweeps, "dmrg_s": time.time() - t}
            print(json.dumps(ref_info), flush=True)
        else:
            L.mpspt_set_reference_ci(ctx, ci)
        if a.partitions > 0:
            kv = h.shape[0] - c["k_act"]
            pairs = [(x, y) for x in range(kv) for y in range(x, kv)][: a.partitions]
            Ms = synthetic.partition_bond_dims(len(pairs)) if a.M <= 0 else [a.M] * len(pairs)
            t = time.time()
            if a.e3:
                # E3 over the listed partitions needs all of them at once
                e2, e3, ex, ep_, e3p, _, rep = L.mpspt_third_order_partitioned(ctx, a.h0, pairs, Ms,
                                                                               n_streams=a.streams)
                print(json.dumps({"config": a.config, "h0": a.h0, "prec": a.prec, "partitions": len(pairs),
                                  "M_part": "seeded from {32,...,512}" if a.M <= 0 else a.M, "E2": e2,
                                  "E3": e3, "E3_cross": ex, "E3_diag": e3 - ex, "wall_s": time.time() - t,
                                  "e2_phase_s": rep.wall_ms / 1e3, "e3_setup_s": rep.e3_setup_ms / 1e3,
                                  "e3_transfers_s": rep.e3_ms / 1e3,
                                  "e3_transfers": rep.e3_transfers, "e3_lane_wait_s": rep.e3_wait_ms / 1e3,
                                  "e3_gflop": rep.e3_flops / 1e9, "e3_plan_mb": rep.e3_plan_bytes / 1e6,
                                  "e3_fp64_tflops": rep.e3_flops / max(rep.e3_ms * 1e-3, 1e-9) / 1e12,
                                  "transfers_per_s": rep.e3_transfers / max(rep.e3_ms / 1e3, 1e-9),
                                  "streams": a.streams, "kernel_launches": rep.kernel_launches, **ref_info}),
                      flush=True)
                return 0
            step = a.chunk if a.chunk > 0 else len(pairs)
            eps, cg, launches, wait = [], 0, 0, 0.0
            for c0 in range(0, len(pairs), step):   # chunks: a progress line after each
                _, ep_c, rep = L.mpspt_minimize_partitioned(ctx, a.h0, pairs[c0:c0 + step], Ms[c0:c0 + step],
                                                            n_streams=a.streams)
                eps.extend(float(v) for v in ep_c)
                cg += rep.cg_iters
                launches += rep.kernel_launches
                wait += rep.host_wait_ms / 1e3
                if step < len(pairs):
                    print(json.dumps({"done": len(eps), "of": len(pairs), "wall_s": time.time() - t}), flush=True)
            wall = time.time() - t
            tot = 0.0
            for v in eps:       # pair order
                tot += v
            rep.cg_iters, rep.kernel_launches, rep.host_wait_ms = cg, launches, wait * 1e3
            hist = {}
            for m in Ms:
                hist[m] = hist.get(m, 0) + 1
            print(json.dumps({"config": a.config, "h0": a.h0, "prec": a.prec, "partitions": len(pairs),
                              "M_part": "seeded from {32,...,512}" if a.M <= 0 else a.M,
                              "M_part_counts": {str(k): v for k, v in sorted(hist.items())}, "E2": tot,
                              "wall_s": wall, "partitions_per_s": len(pairs) / wall, "streams": a.streams,
                              "cg_iters": rep.cg_iters, "kernel_launches": rep.kernel_launches,
                              "host_wait_s": rep.host_wait_ms / 1e3, **ref_info}),
                  flush=True)
            return 0
        t = time.time()
        e2, psi, rep = L.mpspt_minimize_hylleraas(ctx, a.h0, a.M, want_psi1=a.e3)
        wall = time.time() - t
        out = {"config": a.config, "M": a.M, "h0": a.h0, "prec": a.prec, "E2": e2, "wall_s": wall,
               "sweeps": rep.n_sweeps, "e2_per_sweep": [rep.e2_per_sweep[s] for s in range(rep.n_sweeps)],
               "sweep_ms": [rep.sweep_ms[s] for s in range(rep.n_sweeps)], "cg_iters": rep.cg_iters,
               "sigma_ms": rep.sigma_ms, "sigma_gflop": rep.sigma_flops / 1e9, "sigma64_ms": rep.sigma64_ms,
               "max_bond_dim": rep.max_bond_dim, "max_discarded_weight": rep.max_discarded_weight,
               "kernel_launches": rep.kernel_launches, **ref_info}
        if a.e3:
            out["E3"] = L.mpspt_third_order(ctx, a.h0, psi)
            L.mpspt_mps_free(psi)
        print(json.dumps(out), flush=True)
    finally:
        L.mpspt_destroy(ctx)
    return 0


if __name__ == "__main__":
    sys.exit(main())
