"""Benchmark: time-to-E2 of the MPS-PT Hylleraas sweep on one GB300.

A step is one call of mpspt_minimize_hylleraas on the medium workload (8
electrons in 8 active orbitals + 24 virtual orbitals, seeded integrals,
Cholesky rank 60, exact FCI reference), run from the seeded initial Psi1 to
convergence.  Time-to-E2 is the device time (CUDA events recorded by the
library at the end of every sweep) until the reported E2 first lies within
1e-6 Eh of the converged float64 E2 and stays there.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--h0 dyall|fock] [--M 64] [--prec fp64]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-E2 at 1e-6 Eh and σ TFLOP/s on 1 GB300: mixed+batched vs plain FP64"
NOMINAL_FP64_TFLOPS = 1.25      # GB300 dense FP64 (nominal)
NOMINAL_BF16_TFLOPS = 2250.0    # GB300 dense BF16 (nominal)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _clock_sampler():
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        p = subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, f.name


def _clock_summary(p, path, device):
    if p is not None:
        p.terminate()
        try:
            p.wait(timeout=5)
        except Exception:
            p.kill()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device):
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
    except OSError:
        pass
    os.unlink(path) if os.path.exists(path) else None
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


def _inputs(name):
    import synthetic
    h, L, c, ci = synthetic.config_reference(name)
    return h, L, c, ci


def _time_to_e2(rep, e2_ref, tol=1e-6):
    n = rep.n_sweeps
    hist = [rep.e2_per_sweep[s] for s in range(n)]
    first = None
    for s in range(n):
        if all(abs(hist[t] - e2_ref) < tol for t in range(s, n)):
            first = s
            break
    if first is None:
        return None, None
    return rep.sweep_ms[first] / 1e3, first


def _workload(args):
    c = {"tiny": "4e/4o + 8 virtual", "medium": "8e/8o + 24 virtual"}.get(args.config, args.config)
    return f"{args.config}: {c}, M={args.M}, {args.h0} H0"


class _OracleCosts:
    """Measured oracle (CPU) unit costs on the workload's own shapes.

    Tensors carry the bond dimensions of the initial-state rule at bond
    dimension M and the real MPOs; entries are random (the oracle's dense
    contractions cost the same for any values).  Measured: one sigma
    application (Fig. 1C, H0 - E0 term) at an active-region bond and at a
    virtual-region bond, and the once-per-bond-step work at the virtual bond
    (RHS, Jacobi diagonal, truncation, two environment updates).  The
    active-region sigma is the expensive piece (tens of seconds at M = 256)
    and is timed once; the cheap pieces are re-timed at every step."""

    def __init__(self, name, h0, M):
        import numpy as np
        from oracle.mps import random_mps, reference_mps, two_site_mask
        from oracle.mpo import build_mpo
        from oracle.operators import Problem
        import synthetic
        h, L, c, ci = synthetic.config_reference(name)
        p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
        self.p, self.M = p, M
        self.WA = build_mpo(p.h0_terms(), p.k, k_split=p.k_act)
        self.WV = build_mpo(p.rhs_terms(), p.k, k_split=p.k_act)
        N = p.n_elec
        self.allowed = {p.k_act: {N - 1, N - 2}}
        self.psi = random_mps(p.k, (N, 0), self.allowed, M, 1408)
        self.psi0 = reference_mps(p.ci, p.k_act, p.k_virt)
        self.rng = np.random.default_rng(0)
        self.ia = max(1, p.k_act // 2)
        self.iv = p.k_act + (p.k_virt // 2)
        self.two_site_mask = two_site_mask
        self.ts_a = self._sigma(self.ia)[0]

    def _sigma(self, i):
        import time as _t
        from oracle.mps import two_site_apply
        psi, WA = self.psi, self.WA
        Dl, Dr = len(psi.q[i]), len(psi.q[i + 2])
        La = self.rng.normal(size=(WA.dims[i], Dl, Dl))
        Ra = self.rng.normal(size=(WA.dims[i + 2], Dr, Dr))
        mask = self.two_site_mask(psi.q[i], psi.q[i + 2], self.allowed.get(i + 1))
        x = self.rng.normal(size=mask.shape) * mask
        t0 = _t.perf_counter()
        two_site_apply(La, WA.W[i], WA.W[i + 1], Ra, x, WA.dims[i + 1])
        return _t.perf_counter() - t0, (La, Ra, x, Dl, Dr)

    def step(self):
        """Re-times the virtual-bond sigma and the once-per-step work; returns
        (t_sigma_active, t_sigma_virtual, t_once)."""
        import time as _t
        import numpy as np
        from oracle.mps import env_left, truncate, two_site_apply, two_site_diag
        ts_v, (La, Ra, x, Dl, Dr) = self._sigma(self.iv)
        i, psi, psi0, WA, WV = self.iv, self.psi, self.psi0, self.WA, self.WV
        D0l, D0r = len(psi0.q[i]), len(psi0.q[i + 2])
        Lv = self.rng.normal(size=(WV.dims[i], Dl, D0l))
        Rv = self.rng.normal(size=(WV.dims[i + 2], Dr, D0r))
        p0 = np.einsum("lsm,mtr->lstr", psi0.A[i], psi0.A[i + 1])
        t0 = _t.perf_counter()
        two_site_apply(Lv, WV.W[i], WV.W[i + 1], Rv, p0, WV.dims[i + 1])
        two_site_diag(La, WA.W[i], WA.W[i + 1], Ra, x.shape, WA.dims[i + 1])
        Al, Ar, lab, w = truncate(x, psi.q[i], psi.q[i + 2], self.M, "LR", self.allowed.get(i + 1))
        env_left(La, Al, WA.W[i], Al, WA.dims[i + 1])
        env_left(Lv, Al, WV.W[i], psi0.A[i], WV.dims[i + 1])
        return self.ts_a, ts_v, _t.perf_counter() - t0

    def extrapolate(self, costs, n_sigma, n_steps):
        """Seconds the oracle needs for n_sigma sigma applications over
        n_steps bond steps, with sigma applications and steps spread over the
        chain's bonds in proportion to their number (k_act - 1 of the k - 1
        bonds lie in the active region, where sigma is largest)."""
        ts_a, ts_v, t_once = costs
        p = self.p
        frac_a = (p.k_act - 1) / (p.k - 1)
        t_sig = frac_a * ts_a + (1 - frac_a) * ts_v
        return n_sigma * t_sig + n_steps * t_once, (
            f"oracle (NumPy float64, dense) unit costs measured on random tensors of the workload's shapes at "
            f"M={self.M}: sigma {ts_a:.3f} s at active-region bond {self.ia}, {ts_v:.3f} s at virtual-region "
            f"bond {self.iv}; once-per-step work (RHS, diagonal, truncation, two environment updates) "
            f"{t_once:.3f} s at bond {self.iv}; scaled by {n_sigma} sigma applications over {n_steps} bond "
            f"steps (the float64 GPU run's counts until E2), bonds weighted by region "
            f"({p.k_act - 1} of {p.k - 1} active); the once-per-step work of active bonds is priced at the "
            f"virtual bond's, so the total is a lower bound")


def _counts_path(args):
    return os.path.join(ROOT, "profiles", f"bench_counts_{args.config}_M{args.M}_{args.h0}.json")


def _fp64_roofline(reps, peaks, src):
    """The float64 sigma of the refinement (same grouped GEMM kernel as the
    RHS and environment updates) against the float64 peak (the measured bf16
    burst scaled by the nominal float64 / bf16 ratio of GB300)."""
    flops = sum(r.sigma64_flops for r in reps)
    ms = sum(r.sigma64_ms for r in reps)
    peak = peaks["bf16_tflops"] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
    ach = flops / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    return {"bound": "fp64_alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if peak else None, "traffic": None,
            "peak_source": f"{src} bf16 burst x nominal fp64/bf16 ratio",
            "kernel": "k_gemm<64, 64, double> (float64 refinement sigma)"}


def run_reference(args):
    """The oracle arm: the CPU oracle as it stands on this machine's host cores.
    A real oracle run to E2 at this size takes hours, so each step times the
    oracle's unit costs (see _OracleCosts) and scales them by the counts the
    float64 GPU sweep needed to reach E2 on the same workload (recorded by
    the GPU arm in profiles/bench_counts_<workload>.json)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    counts = None
    try:
        counts = json.load(open(_counts_path(args)))
    except (OSError, ValueError):
        counts = None
    oc = _OracleCosts(args.config, args.h0, args.M)
    vals, sample = [], ""
    for s_ in range(args.warmup + args.steps):
        costs = oc.step()
        if counts:
            v, sample = oc.extrapolate(costs, counts["sigma_calls_to_e2"], counts["bond_steps_to_e2"])
        else:   # no GPU record for this workload: one sigma per step over one sweep
            n = 2 * (oc.p.k - 1)
            v, sample = oc.extrapolate(costs, n, n)
            sample += " (no GPU count record: one sweep, one sigma per step)"
        vals.append(v)
    value = statistics.median(vals[args.warmup:])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": _workload(args), "h0": args.h0, "M": args.M},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": sample + (f"; counts from {os.path.basename(_counts_path(args))}"
                                                 if counts else "")},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import numpy as np
    import torch
    from paper_1408_5092_gb300 import _lib as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    L.load()
    h, Lc, c, ci = _inputs(args.config)
    k = h.shape[0]
    stream = torch.cuda.current_stream()
    o = L.mpspt_default_options()
    o.device = local
    o.stream = stream.cuda_stream
    o.prec = L.PREC[args.prec]
    o.e_tol = args.e_tol
    o.max_sweeps = args.max_sweeps
    # tuned GEMM tiles for the mixed arm: the warm-up context tunes, its table
    # goes to a cache file when it is destroyed, and the end-to-end contexts
    # read it back (the plain float64 arm keeps the default tiles)
    import tempfile
    tune_dir = tempfile.mkdtemp(prefix="mpspt_tiles_")
    tune_cache = os.path.join(tune_dir, "tiles.txt").encode()
    o.autotune = 1 if args.autotune else 0
    o.autotune_cache = tune_cache if args.autotune else None
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], k - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference_ci(ctx, ci)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one(c=None):
        flush.zero_()
        torch.cuda.synchronize()
        e2, psi, rep = L.mpspt_minimize_hylleraas(c or ctx, args.h0, args.M, want_psi1=False)
        return e2, rep

    # warm-up 1: the plain float64 sweep converged tightly; it fixes E2_ref
    # (the float64 E2 at this M, within 1e-8 of the oracle by the parity tests)
    def ctx_for(prec, e_tol):
        oo = L.mpspt_default_options()
        oo.device = local
        oo.stream = stream.cuda_stream
        oo.prec = prec
        oo.e_tol = e_tol
        oo.max_sweeps = args.max_sweeps
        cx = L.mpspt_create(oo)
        L.mpspt_set_integrals(cx, c["k_act"], k - c["k_act"], c["n_elec"], h, Lc)
        L.mpspt_set_reference_ci(cx, ci)
        return cx
    ctx64 = ctx_for(L.MPSPT_FP64, args.ref_e_tol)
    e2_ref, rep_ref = one(ctx64)
    L.mpspt_destroy(ctx64)
    hist_ref = [rep_ref.e2_per_sweep[s] for s in range(rep_ref.n_sweeps)]
    # the plain float64 arm: same stopping rule as the mixed arm, its own
    # warm-up (the run above) and fp64_steps timed repeats (median)
    ctx64 = ctx_for(L.MPSPT_FP64, args.e_tol)
    fp64_runs = []
    for s_ in range(max(1, min(args.steps, args.fp64_steps))):
        _, r64 = one(ctx64)
        t_, s64_ = _time_to_e2(r64, e2_ref)
        fp64_runs.append((t_ if t_ is not None else r64.wall_ms / 1e3, s64_, r64))
    L.mpspt_destroy(ctx64)
    t64 = statistics.median([x[0] for x in fp64_runs])
    rep64 = fp64_runs[0][2]
    s64 = fp64_runs[0][1]
    for w in range(max(0, args.warmup - 1)):
        one()
    sampler, cpath = _clock_sampler() if rank == 0 else (None, None)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")     # lets a profiler capture the timed steps only
    t0 = time.perf_counter()
    reps, tte, e2s = [], [], []
    for s in range(args.steps):
        e2, rep = one()
        reps.append(rep)
        e2s.append(e2)
        t, _ = _time_to_e2(rep, e2_ref)
        tte.append(t if t is not None else rep.wall_ms / 1e3)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    clocks = _clock_summary(sampler, cpath, local) if rank == 0 else None
    value = statistics.median(tte)
    ms_per_step = 1e3 * wall / args.steps
    if dist:
        t = torch.tensor([value, ms_per_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        value, ms_per_step = float(t[0]), float(t[1])
        dist.barrier()
    L.mpspt_destroy(ctx)      # writes the tuned tile table for the end-to-end contexts
    ctx = None
    # end to end through the public API: wall clock from mpspt_create to the
    # return of mpspt_minimize_hylleraas (integrals and CI vector copied from
    # host buffers, E2 read back), median of e2e_steps runs
    e2e_times = []
    for s_ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx2 = L.mpspt_create(o)
        L.mpspt_set_integrals(ctx2, c["k_act"], k - c["k_act"], c["n_elec"], h, Lc)
        L.mpspt_set_reference_ci(ctx2, ci)
        e2, _, rep = L.mpspt_minimize_hylleraas(ctx2, args.h0, args.M, want_psi1=False)
        e2e_times.append(time.perf_counter() - t1)
        L.mpspt_destroy(ctx2)
    e2e = statistics.median(e2e_times) if e2e_times else None
    if dist and e2e is not None:
        t = torch.tensor([e2e], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = float(t[0])
    flops = sum(r.sigma_flops for r in reps)
    sms = sum(r.sigma_ms for r in reps)
    achieved = flops / (sms * 1e-3) / 1e12 if sms > 0 else 0.0
    peaks, src = _peaks()
    if args.prec == "fp64":
        peak = peaks["bf16_tflops"] * NOMINAL_FP64_TFLOPS / NOMINAL_BF16_TFLOPS
        peak_note = f"fp64 = {src} bf16 burst x nominal fp64/bf16 ratio"
    else:
        peak = peaks["bf16_tflops"]
        peak_note = f"{src} bf16 burst"
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "sigma_gemm_traffic.json")
    if os.path.exists(tpath):
        try:
            tj = json.load(open(tpath))
            if tj.get("prec") == args.prec and tj.get("M") == args.M and tj.get("h0") == args.h0:
                traffic = tj.get("bytes_per_launch")
        except Exception:
            traffic = None
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "bf16x3+f64", "mixed_fp16": "f16x3+f64"}[args.prec],
        "data": "synthetic",
        "config": {"workload": _workload(args), "h0": args.h0, "M": args.M, "prec": args.prec, "l2_flush": True,
                   "tuned_tiles": bool(args.autotune),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "E2": statistics.median(e2s), "E2_ref": e2_ref,
        "sweeps": [r.n_sweeps for r in reps],
        "fp64": {"time_to_e2_s": t64, "runs_s": [x[0] for x in fp64_runs],
                 "sweeps_to_e2": (s64 + 1) if s64 is not None else None,
                 "sweeps": rep64.n_sweeps, "sigma_tflops": (rep64.sigma_flops / (rep64.sigma_ms * 1e-3) / 1e12)
                 if rep64.sigma_ms > 0 else None, "e2_ref_history": hist_ref,
                 "note": "plain float64 sweep on the same inputs and stopping rule: one untimed converged run "
                         "(E2_ref, e_tol ref_e_tol) then fp64_steps timed repeats, median"},
        "speedup_vs_fp64": (t64 / value) if (t64 and value) else None,
        "sigma_tflops": achieved,
        "roofline": {"bound": "fp64_alu" if args.prec == "fp64" else "tensor", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                     "traffic": traffic, "peak_source": peak_note,
                     "kernel": "k_gemm (sigma grouped block GEMM)"},
        "roofline_fp64_sigma": _fp64_roofline(reps, peaks, src),
        "e2e": {"value": e2e, "unit": "s", "runs": args.e2e_steps,
                "what": "wall clock mpspt_create -> set_integrals -> set_reference_ci -> minimize_hylleraas "
                        "(to the e_tol stop) -> return, host buffers"
                        + (", tile table read from the warm-up context's cache file" if args.autotune else ""),
                "h2d_bytes_per_step": int(h.nbytes + Lc.nbytes + ci.nbytes), "d2h_bytes_per_step": 8},
        "gpu_launches": int(sum(r.kernel_launches for r in reps)),
        "clocks": clocks,
    }
    # counts of the float64 run until E2 (they scale the oracle's unit costs)
    n_sig = int(rep64.sigma_calls_cum[s64]) if s64 is not None else int(rep64.sigma_calls_cum[rep64.n_sweeps - 1])
    n_steps = 2 * (k - 1) * ((s64 + 1) if s64 is not None else rep64.n_sweeps)
    line["fp64"]["sigma_calls_to_e2"] = n_sig
    line["fp64"]["bond_steps_to_e2"] = n_steps
    if rank == 0 and world == 1 and args.write_counts:
        with open(_counts_path(args), "w") as f:
            json.dump({"workload": _workload(args), "sigma_calls_to_e2": n_sig, "bond_steps_to_e2": n_steps,
                       "from": "float64 GPU sweep of bench.py (plain arm), same inputs"}, f, indent=1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oc = _OracleCosts(args.config, args.h0, args.M)
        val, sample = oc.extrapolate(oc.step(), n_sig, n_steps)
        line["cpu_baseline"] = {"value": val, "unit": "s", "cores": len(os.sched_getaffinity(0)),
                                "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="medium")
    ap.add_argument("--h0", default="dyall", choices=["dyall", "fock"])
    ap.add_argument("--M", type=int, default=256)
    ap.add_argument("--prec", default="mixed", choices=["fp64", "fp32", "mixed", "mixed_fp16"])
    ap.add_argument("--e_tol", type=float, default=1e-7)
    ap.add_argument("--ref_e_tol", type=float, default=1e-9)
    ap.add_argument("--e2e_steps", type=int, default=3)
    ap.add_argument("--autotune", type=int, default=1,
                    help="tuned GEMM tiles in the mixed arm (tuned during warm-up, cached for the e2e runs)")
    ap.add_argument("--fp64_steps", type=int, default=3,
                    help="timed repeats of the plain float64 arm (at most --steps)")
    ap.add_argument("--write_counts", action="store_true",
                    help="record the float64 run's counts for the oracle arm (profiles/bench_counts_*.json)")
    ap.add_argument("--no_cpu_baseline", action="store_true")
    ap.add_argument("--max_sweeps", type=int, default=64,
                    help="sweep cap of every minimisation (a smaller workload, e.g. for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
