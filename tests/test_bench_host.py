"""Host-side parts of bench.py, without a GPU: the time-to-E2 rule, the
clock-record parser, the float64 roofline arithmetic, and the JSON line of
the oracle arm (--impl reference), which runs on the host cores only."""
import json
import os
import subprocess
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _rep(hist, ms):
    return SimpleNamespace(n_sweeps=len(hist), e2_per_sweep=list(hist), sweep_ms=list(ms))


def test_time_to_e2_takes_first_sweep_that_stays_within_tolerance():
    ref = -1.0
    ms = [100.0, 200.0, 300.0, 400.0, 500.0]
    # within 1e-6 at sweep 1, out again at sweep 2, back from sweep 3 on
    rep = _rep([-0.9, -1.0 + 5e-7, -1.0 + 3e-6, -1.0 + 2e-7, -1.0], ms)
    t, s = bench._time_to_e2(rep, ref)
    assert s == 3 and t == pytest.approx(0.4)
    # never within tolerance at the end
    assert bench._time_to_e2(_rep([-0.9, -0.99], ms[:2]), ref) == (None, None)
    # converged from the first sweep
    assert bench._time_to_e2(_rep([-1.0, -1.0], ms[:2]), ref) == (pytest.approx(0.1), 0)


def test_clock_summary_reads_only_its_device(tmp_path):
    p = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2050, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "1, 1000, 2070, 300.0, 0x0, Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    p.write_text("\n".join(rows) + "\n")
    c = bench._clock_summary(None, str(p), 0)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]     # device 1's hw_slowdown is not ours
    assert c["samples"] == 3
    assert not p.exists()


def test_fp64_roofline_arithmetic():
    reps = [SimpleNamespace(sigma64_flops=2e12, sigma64_ms=1000.0),
            SimpleNamespace(sigma64_flops=1e12, sigma64_ms=500.0)]
    r = bench._fp64_roofline(reps, {"bf16_tflops": 1800.0}, "measured")
    assert r["achieved"] == pytest.approx(2.0)            # 3e12 flop in 1.5 s
    assert r["peak"] == pytest.approx(1800.0 * 1.25 / 2250.0)
    assert r["frac"] == pytest.approx(2.0 / r["peak"])
    assert r["unit"] == "TFLOP/s" and r["bound"] == "fp64_alu"


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--M", "16", "--config", "tiny"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return [l for l in out.stdout.splitlines() if l.strip()]


def test_reference_arm_prints_one_contract_line():
    lines = _run_reference({"RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "s" and d["higher_is_better"] is False and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["ms_per_step"] == pytest.approx(d["value"] * 1e3)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"] and d["config"]["M"] == 16


def test_reference_arm_other_ranks_exit_quietly():
    assert _run_reference({"RANK": "1"}) == []
