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
    h, L, c = synthetic.config_integrals(name)
    ci, _ = synthetic.fci_reference(h, L, c["k_act"], c["n_elec"])
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


def _oracle_sample(name, h0, M, cg_per_step, bonds_active, bonds_virtual):
    """Bounded oracle (CPU) sample of the same workload.

    The oracle's own sweep would spend minutes just building environments at
    this size, so the sample times its kernels once each on tensors with the
    workload's shapes (bond dimensions from the initial-state rule, the real
    MPOs): sigma at an active-region bond and at a virtual-region bond, and
    the once-per-step work (RHS, Jacobi diagonal, truncation, two environment
    updates) at the virtual-region bond.  Seconds per bond step are then
    (cg + 2) x sigma + once-per-step work; the active-region once-per-step
    work (larger RHS) is not included, so the estimate is a lower bound."""
    import numpy as np
    from oracle.mps import (HylleraasSweep, env_left, random_mps, reference_mps, truncate,
                            two_site_apply, two_site_diag, two_site_mask)
    from oracle.mpo import build_mpo
    from oracle.operators import Problem
    h, L, c, ci = _inputs(name)
    p = Problem(h, L, c["k_act"], c["n_elec"], ci, h0=h0)
    WA = build_mpo(p.h0_terms(), p.k, k_split=p.k_act)
    WV = build_mpo(p.rhs_terms(), p.k, k_split=p.k_act)
    N = p.n_elec
    allowed = {p.k_act: {N - 1, N - 2}}
    psi = random_mps(p.k, (N, 0), allowed, M, 1408)
    psi0 = reference_mps(p.ci, p.k_act, p.k_virt)
    rng = np.random.default_rng(0)

    def t_sigma(i):
        Dl, Dr = len(psi.q[i]), len(psi.q[i + 2])
        La = rng.normal(size=(WA.dims[i], Dl, Dl))
        Ra = rng.normal(size=(WA.dims[i + 2], Dr, Dr))
        mask = two_site_mask(psi.q[i], psi.q[i + 2], allowed.get(i + 1))
        x = rng.normal(size=mask.shape) * mask
        t0 = time.perf_counter()
        two_site_apply(La, WA.W[i], WA.W[i + 1], Ra, x, WA.dims[i + 1])
        return time.perf_counter() - t0, (La, Ra, x, mask, Dl, Dr)

    ia = max(1, p.k_act // 2)
    iv = p.k_act + (p.k_virt // 2)
    ts_a, _ = t_sigma(ia)
    ts_v, (La, Ra, x, mask, Dl, Dr) = t_sigma(iv)
    i = iv
    D0l, D0r = len(psi0.q[i]), len(psi0.q[i + 2])
    Lv = rng.normal(size=(WV.dims[i], Dl, D0l))
    Rv = rng.normal(size=(WV.dims[i + 2], Dr, D0r))
    p0 = np.einsum("lsm,mtr->lstr", psi0.A[i], psi0.A[i + 1])
    t0 = time.perf_counter()
    two_site_apply(Lv, WV.W[i], WV.W[i + 1], Rv, p0, WV.dims[i + 1])
    two_site_diag(La, WA.W[i], WA.W[i + 1], Ra, x.shape, WA.dims[i + 1])
    Al, Ar, lab, w = truncate(x, psi.q[i], psi.q[i + 2], M, "LR", allowed.get(i + 1))
    env_left(La, Al, WA.W[i], Al, WA.dims[i + 1])
    env_left(Lv, Al, WV.W[i], psi0.A[i], WV.dims[i + 1])
    t_once = time.perf_counter() - t0
    per_a = (cg_per_step + 2) * ts_a + t_once
    per_v = (cg_per_step + 2) * ts_v + t_once
    sample = (f"oracle kernels timed once each on random tensors of the workload's shapes (M={M}): "
              f"sigma {ts_a:.3f}s at active bond {ia}, {ts_v:.3f}s at virtual bond {iv}; "
              f"once-per-step work {t_once:.3f}s at bond {iv}; x {cg_per_step:.1f} CG iterations per step "
              f"over {bonds_active} active and {bonds_virtual} virtual bond steps (lower bound)")
    return per_a * bonds_active + per_v * bonds_virtual, sample


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
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    c = {"medium": (8, 24)}.get(args.config, (8, 24))
    bonds = 2 * (c[0] + c[1] - 1) * args.ref_sweeps
    frac_a = c[0] / (c[0] + c[1] - 1)
    vals = []
    sample = ""
    for _ in range(args.warmup + args.steps):
        v, sample = _oracle_sample(args.config, args.h0, args.M, args.ref_cg, bonds * frac_a, bonds * (1 - frac_a))
        vals.append(v)
    value = statistics.median(vals[args.warmup:])
    sample += f"; {args.ref_sweeps} sweeps assumed"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.config}: 8e/8o + 24 virtual, M={args.M}, {args.h0} H0",
                       "h0": args.h0, "M": args.M},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
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
    ctx = L.mpspt_create(o)
    L.mpspt_set_integrals(ctx, c["k_act"], k - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference(ctx, ci)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one(c=None):
        flush.zero_()
        torch.cuda.synchronize()
        e2, psi, rep = L.mpspt_minimize_hylleraas(c or ctx, args.h0, args.M, want_psi1=False)
        return e2, rep

    # warm-up 1: the plain float64 sweep converged tightly; it fixes E2_ref
    # (the float64 E2 at this M) and gives the float64 time-to-E2
    o64 = L.mpspt_default_options()
    o64.device = local
    o64.stream = stream.cuda_stream
    o64.prec = L.MPSPT_FP64
    o64.e_tol = args.ref_e_tol
    o64.max_sweeps = args.max_sweeps
    ctx64 = L.mpspt_create(o64)
    L.mpspt_set_integrals(ctx64, c["k_act"], k - c["k_act"], c["n_elec"], h, Lc)
    L.mpspt_set_reference(ctx64, ci)
    e2_ref, rep64 = one(ctx64)
    L.mpspt_destroy(ctx64)
    hist64 = [rep64.e2_per_sweep[s] for s in range(rep64.n_sweeps)]
    t64, s64 = _time_to_e2(rep64, e2_ref)
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
    # end to end through the public API with host buffers
    e2e_times = []
    for s in range(args.e2e_steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ctx2 = L.mpspt_create(o)
        L.mpspt_set_integrals(ctx2, c["k_act"], k - c["k_act"], c["n_elec"], h, Lc)
        L.mpspt_set_reference(ctx2, ci)
        t_setup = time.perf_counter() - t1
        e2, _, rep = L.mpspt_minimize_hylleraas(ctx2, args.h0, args.M, want_psi1=False)
        tt, _ = _time_to_e2(rep, e2_ref)
        e2e_times.append(t_setup + (tt if tt is not None else rep.wall_ms / 1e3))
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
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "mixed": "bf16x3+f64"}[args.prec],
        "data": "synthetic",
        "config": {"workload": f"{args.config}: 8e/8o + 24 virtual, M={args.M}, {args.h0} H0, {args.prec}",
                   "h0": args.h0, "M": args.M, "prec": args.prec, "l2_flush": True,
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "E2": statistics.median(e2s), "E2_ref": e2_ref,
        "sweeps": [r.n_sweeps for r in reps],
        "fp64": {"time_to_e2_s": t64, "sweeps_to_e2": (s64 + 1) if s64 is not None else None,
                 "sweeps": rep64.n_sweeps, "sigma_tflops": (rep64.sigma_flops / (rep64.sigma_ms * 1e-3) / 1e12)
                 if rep64.sigma_ms > 0 else None, "e2_history": hist64},
        "speedup_vs_fp64": (t64 / value) if (t64 and value) else None,
        "sigma_tflops": achieved,
        "roofline": {"bound": "fp64_alu" if args.prec == "fp64" else "tensor", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                     "traffic": traffic, "peak_source": peak_note,
                     "kernel": "k_gemm (sigma grouped block GEMM)"},
        "roofline_fp64_sigma": _fp64_roofline(reps, peaks, src),
        "e2e": {"value": e2e, "unit": "s",
                "h2d_bytes_per_step": int(h.nbytes + Lc.nbytes + ci.nbytes), "d2h_bytes_per_step": 8},
        "gpu_launches": int(sum(r.kernel_launches for r in reps)),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle needs as many bond steps as the float64 GPU run took to reach E2
        ka, kv = c["k_act"], k - c["k_act"]
        nb = 2 * (k - 1) * ((s64 + 1) if s64 is not None else rep64.n_sweeps)
        cg_ps = rep64.cg_iters / max(1, 2 * (k - 1) * rep64.n_sweeps)
        frac_a = ka / (k - 1)
        val, sample = _oracle_sample(args.config, args.h0, args.M, cg_ps, nb * frac_a, nb * (1 - frac_a))
        line["cpu_baseline"] = {"value": val, "unit": "s", "cores": len(os.sched_getaffinity(0)),
                                "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    L.mpspt_destroy(ctx)
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
    ap.add_argument("--prec", default="mixed", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--e_tol", type=float, default=1e-7)
    ap.add_argument("--ref_e_tol", type=float, default=1e-9)
    ap.add_argument("--e2e_steps", type=int, default=1)
    ap.add_argument("--ref_sweeps", type=int, default=10)
    ap.add_argument("--ref_cg", type=float, default=6.0)
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
